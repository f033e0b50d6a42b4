"""Truth solves x(mu) = A(mu)^{-1} f(mu) of eq. 1.

`sparse_direct` factors the sparse matrix with SuperLU (scipy), the library
step standing in for "a standard linear solver" of Alg. 1 step 3.  `cg` is
textbook (preconditioned) conjugate gradients, Hestenes-Stiefel form, used
for large grids and as the plain-CG baseline the paper compares against.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import problem as pb


def sparse_direct(prob, mu, b=None) -> np.ndarray:
    A = pb.assemble_csr(prob, mu).tocsc()
    rhs = pb.load(prob, mu) if b is None else b
    return spla.spsolve(A, rhs)


def cg(prob, mu, b=None, tol: float = 1e-13, max_iter: int = 100000, precond=None,
       x0=None, history: bool = False):
    """Textbook PCG on A(mu) x = b; stops when ||r|| < tol ||b||.

    Returns (x, iterations, residual-norm history).  `precond(r)` returns
    M^{-1} r (identity if None).
    """
    b = pb.load(prob, mu) if b is None else np.asarray(b, dtype=np.float64)
    A = lambda v: pb.apply(prob, mu, v)
    M = (lambda r: r.copy()) if precond is None else precond
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    r = b - A(x) if x0 is not None else b.copy()
    bn = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bn]
    it = 0
    if hist[-1] < tol:
        return x, it, hist
    z = M(r)
    p = z.copy()
    rz = r @ z
    while it < max_iter:
        q = A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        if hist[-1] < tol:
            break
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist
