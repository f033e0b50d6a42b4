"""The smoother z = S(A, b, y) of eq. 8: iterate on A z = b starting from y.

The paper names Jacobi or Gauss-Seidel (Section 3.1) and uses Gauss-Seidel for
every method (Section 3.3).  Lexicographic Gauss-Seidel is sequential; the
oracle's default is the red-black ordering (colour (i_x + i_y + i_z) mod 2,
colour 0 first), which is a Gauss-Seidel method with a different point order.
The lexicographic form is kept to compare iteration counts.

Every sweep updates a point as z_i <- z_i + (b_i - (A z)_i) / a_ii using the
newest values; in the red-black form all points of one colour are mutually
uncoupled, so updating them at once is the same as updating them one by one.
"""
from __future__ import annotations

import numpy as np

from . import problem as pb


def red_black_gs(prob, mu, b, y, sweeps: int = 1) -> np.ndarray:
    D = pb.diagonal(prob, mu)
    col = pb.colour(prob)
    z = np.array(y, dtype=np.float64, copy=True)
    for _ in range(sweeps):
        for c in (0, 1):
            upd = z + (b - pb.apply(prob, mu, z)) / D
            z[col == c] = upd[col == c]
    return z


def lexicographic_gs(prob, mu, b, y, sweeps: int = 1) -> np.ndarray:
    """Point-by-point Gauss-Seidel in the flat index order (pure Python; tiny grids only)."""
    A = pb.assemble_csr(prob, mu)
    z = np.array(y, dtype=np.float64, copy=True)
    for _ in range(sweeps):
        for i in range(prob.n_dof):
            lo, hi = A.indptr[i], A.indptr[i + 1]
            cols, vals = A.indices[lo:hi], A.data[lo:hi]
            s, aii = b[i], 0.0
            for j, a in zip(cols, vals):
                if j == i:
                    aii = a
                else:
                    s -= a * z[j]
            z[i] = s / aii
    return z


def jacobi(prob, mu, b, y, sweeps: int = 1, omega: float = 2.0 / 3.0) -> np.ndarray:
    D = pb.diagonal(prob, mu)
    z = np.array(y, dtype=np.float64, copy=True)
    for _ in range(sweeps):
        z = z + omega * (b - pb.apply(prob, mu, z)) / D
    return z


def smooth(kind: str, prob, mu, b, y, sweeps: int = 1, omega: float = 2.0 / 3.0) -> np.ndarray:
    if kind == "none" or sweeps == 0:
        return np.array(y, dtype=np.float64, copy=True)
    if kind == "rbgs":
        return red_black_gs(prob, mu, b, y, sweeps)
    if kind == "lexgs":
        return lexicographic_gs(prob, mu, b, y, sweeps)
    if kind == "jacobi":
        return jacobi(prob, mu, b, y, sweeps, omega)
    raise ValueError(kind)
