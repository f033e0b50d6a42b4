"""Independent constructions the oracle is pinned to (no oracle code used here).

* `incidence_operator`: A(mu) = G^T diag(kappa_f / h_f^2) G, with G the
  face-node incidence matrix (one row per face, boundary faces included).  This
  is the energy form v^T A v = sum_f kappa_f (v_i - v_j)^2 / h^2 of the same
  finite-difference operator, assembled by loops over nodes instead of by
  array slicing.
* `laplace_closed_form`: at equal coefficients mu_p = c the operator is c times
  the Dirichlet Laplacian, diagonalised by the discrete sine transform:
  v_k(i) = prod_d sin(k_d pi (i_d + 1) h_d), lambda_k = sum_d 4/h_d^2 sin^2(k_d pi h_d / 2),
  ||v_k||^2 = prod_d (m_d + 1)/2.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def _block_of(i1: int, m: int, nb: int) -> int:
    # 1-based node index i1 in 1..m: floor((i1 - 1) nb / m)
    return ((i1 - 1) * nb) // m


def incidence_operator(dims, blocks, mu) -> np.ndarray:
    dim = len(dims)
    n = int(np.prod(dims))
    strides = [int(np.prod(dims[:d])) for d in range(dim)]
    bstr = [int(np.prod(blocks[:d])) for d in range(dim)]

    def node_mu(idx):
        p = sum(_block_of(idx[d] + 1, dims[d], blocks[d]) * bstr[d] for d in range(dim))
        return mu[p]

    rows_G, w = [], []
    for idx in itertools.product(*[range(m) for m in reversed(dims)]):
        idx = tuple(reversed(idx))            # (ix, iy, iz)
        i = sum(idx[d] * strides[d] for d in range(dim))
        for d in range(dim):
            inv_h2 = (dims[d] + 1) ** 2
            # face towards -d: to the boundary if idx[d] == 0 (interior faces are added from the lower node)
            if idx[d] == 0:
                g = np.zeros(n); g[i] = 1.0
                rows_G.append(g); w.append(node_mu(idx) * inv_h2)
            if idx[d] == dims[d] - 1:
                g = np.zeros(n); g[i] = 1.0
                rows_G.append(g); w.append(node_mu(idx) * inv_h2)
            else:
                nb_idx = list(idx); nb_idx[d] += 1
                j = i + strides[d]
                g = np.zeros(n); g[i] = 1.0; g[j] = -1.0
                rows_G.append(g); w.append(0.5 * (node_mu(idx) + node_mu(tuple(nb_idx))) * inv_h2)
    G = np.array(rows_G)
    return G.T @ (np.array(w)[:, None] * G)


def dst_matrix(m: int) -> np.ndarray:
    h = 1.0 / (m + 1)
    k = np.arange(1, m + 1)[:, None]
    i = np.arange(m)[None, :]
    return np.sin(k * math.pi * (i + 1) * h)


def laplace_closed_form(dims, c: float, f: np.ndarray) -> np.ndarray:
    """Solution of c L_h x = f for the Dirichlet Laplacian L_h, via the DST eigenbasis."""
    dim = len(dims)
    F = np.asarray(f, dtype=np.float64).reshape(tuple(reversed(dims)))
    S = [dst_matrix(m) for m in dims]
    # forward transform along every axis: coefficient <v_k, f>
    Fh = F
    for d in range(dim):
        ax = dim - 1 - d
        Fh = np.moveaxis(np.tensordot(S[d], Fh, axes=([1], [ax])), 0, ax)
    lam = np.zeros(Fh.shape)
    norm2 = 1.0
    for d in range(dim):
        ax = dim - 1 - d
        m = dims[d]
        h = 1.0 / (m + 1)
        ld = 4.0 / h ** 2 * np.sin(np.arange(1, m + 1) * math.pi * h / 2.0) ** 2
        shape = [1] * dim; shape[ax] = m
        lam = lam + ld.reshape(shape)
        norm2 *= (m + 1) / 2.0
    Xh = Fh / (c * lam * norm2)
    X = Xh
    for d in range(dim):
        ax = dim - 1 - d
        X = np.moveaxis(np.tensordot(S[d].T, X, axes=([1], [ax])), 0, ax)
    return X.reshape(-1)


def red_black_permutation(dims) -> np.ndarray:
    """Flat indices ordered colour 0 first, then colour 1, each in natural order."""
    dim = len(dims)
    idx = np.indices(tuple(reversed(dims))).reshape(dim, -1)
    col = idx.sum(axis=0) % 2
    n = int(np.prod(dims))
    flat = np.arange(n)
    return np.concatenate([flat[col == 0], flat[col == 1]])


def textbook_gs(A: np.ndarray, b, x, sweeps=1, order=None) -> np.ndarray:
    """x <- x + (D - L)^{-1} (b - A x) in the given point order (Gauss-Seidel)."""
    import scipy.linalg as sla
    n = A.shape[0]
    perm = np.arange(n) if order is None else np.asarray(order)
    Ap = A[np.ix_(perm, perm)]
    xp = np.asarray(x, dtype=np.float64)[perm].copy()
    bp = np.asarray(b, dtype=np.float64)[perm]
    DL = np.tril(Ap)
    for _ in range(sweeps):
        xp = xp + sla.solve_triangular(DL, bp - Ap @ xp, lower=True)
    out = np.empty(n)
    out[perm] = xp
    return out
