"""The parametrized SPD system A(mu) x = f(mu) (eq. 1) and its affine form (eq. 12).

Discretisation (finite differences; the paper's own experiments use P1 finite
elements, Section 5):
  * unknowns are the interior nodes i_d = 0..m_d-1 of a uniform grid on the
    unit square / cube, h_d = 1/(m_d + 1), node coordinate (i_d + 1) h_d;
    vectors are flat with x fastest (numpy shape (mz, my, mx) or (my, mx));
  * (A(mu) v)_i = sum over the 2*dim faces of node i of kappa_f (v_i - v_j)/h_d^2,
    with v_j = 0 outside the grid (homogeneous Dirichlet);
  * block map b_d(i) = floor(i * nb_d / m_d), node block
    p = b_x + nb_x (b_y + nb_y b_z), node coefficient mu_p;
  * kappa_f = (mu_p(i) + mu_p(j)) / 2 on a face between two nodes and
    kappa_f = mu_p(i) on a face to the boundary.  The arithmetic mean keeps
    A(mu) = sum_p mu_p A_p affine in mu (eq. 12 with Theta_q(mu) = mu_q, Q = P).
  * f(mu) = sum_r phi_r(mu) f_r (eq. 12), phi_r = 1 or mu[param_r];
    f_r = 1 (const) or exp(-|x - c_r|^2 / (2 sigma_r^2)) at the nodes.
  * Coefficient fields (the paper's Section 5 cases): the node coefficient is
    kappa(i) = sum_q mu_q F_q(i) with given node values F_q, the face rule is the
    same, so A(mu) = sum_q mu_q A_q with A_q the operator of kappa = F_q.
  * Non-zero Dirichlet data g (the paper's Case 2): in the row of a node i next
    to the boundary, the face to the boundary node j carries kappa(i) and the
    known value g(j) moves to the right-hand side, kappa(i) g(j) / h_d^2.  With
    kappa = sum_q mu_q F_q the lift is affine: a "boundary" load term is
    sum over the boundary faces of F_q(i) g(j) / h_d^2 for one field q.
    (In block problems F_q is the indicator of block q.)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads import Problem


def grid_shape(prob: Problem):
    """numpy shape of a grid vector: reversed dims so that x is the fastest axis."""
    return tuple(reversed(prob.dims))


def block_index(m: int, nb: int) -> np.ndarray:
    """b(i) = floor(i * nb / m), i = 0..m-1."""
    i = np.arange(m)
    return (i * nb) // m


def node_block(prob: Problem) -> np.ndarray:
    """Block id p of every node, as a grid-shaped integer array."""
    p = np.zeros(grid_shape(prob), dtype=np.int64)
    stride = 1
    for d in range(prob.dim):
        ax = prob.dim - 1 - d
        b = block_index(prob.dims[d], prob.blocks[d])
        shape = [1] * prob.dim
        shape[ax] = prob.dims[d]
        p = p + stride * b.reshape(shape)
        stride *= prob.blocks[d]
    return p


def node_fields(prob: Problem) -> np.ndarray:
    """[P][grid] the fields F_q at the nodes: the given fields, or the block indicators."""
    F = prob.field_values()
    if F is not None:
        return np.asarray(F, dtype=np.float64).reshape((prob.P,) + grid_shape(prob))
    blk = node_block(prob)
    return np.stack([(blk == q).astype(np.float64) for q in range(prob.P)])


def node_coefficient(prob: Problem, mu) -> np.ndarray:
    """kappa at every node (grid-shaped): mu_p(i) on blocks, sum_q mu_q F_q(i) with fields."""
    mu = np.asarray(mu, dtype=np.float64)
    if prob.coefficient == "blocks":
        return mu[:prob.P][node_block(prob)]
    F = node_fields(prob)
    K = np.zeros(grid_shape(prob))
    for q in range(prob.P):
        K += mu[q] * F[q]
    return K


def _sl(ndim, ax, s):
    idx = [slice(None)] * ndim
    idx[ax] = s
    return tuple(idx)


def apply(prob: Problem, mu, v) -> np.ndarray:
    """A(mu) v by summing the flux of every face (definition above)."""
    K = node_coefficient(prob, mu)
    V = np.asarray(v, dtype=np.float64).reshape(grid_shape(prob))
    out = np.zeros_like(V)
    nd = prob.dim
    for d in range(nd):
        ax = nd - 1 - d
        m = prob.dims[d]
        inv_h2 = float(m + 1) ** 2
        lo, hi = _sl(nd, ax, slice(0, m - 1)), _sl(nd, ax, slice(1, m))
        # faces between node k and node k+1 along this axis
        kf = 0.5 * (K[lo] + K[hi])
        flux = kf * (V[lo] - V[hi]) * inv_h2
        out[lo] += flux
        out[hi] -= flux
        # faces from the first and the last node to the boundary
        first, last = _sl(nd, ax, slice(0, 1)), _sl(nd, ax, slice(m - 1, m))
        out[first] += K[first] * V[first] * inv_h2
        out[last] += K[last] * V[last] * inv_h2
    return out.reshape(-1)


def diagonal(prob: Problem, mu) -> np.ndarray:
    """a_ii = sum over the faces of node i of kappa_f / h_d^2."""
    K = node_coefficient(prob, mu)
    D = np.zeros_like(K)
    nd = prob.dim
    for d in range(nd):
        ax = nd - 1 - d
        m = prob.dims[d]
        inv_h2 = float(m + 1) ** 2
        lo, hi = _sl(nd, ax, slice(0, m - 1)), _sl(nd, ax, slice(1, m))
        kf = 0.5 * (K[lo] + K[hi]) * inv_h2
        D[lo] += kf
        D[hi] += kf
        first, last = _sl(nd, ax, slice(0, 1)), _sl(nd, ax, slice(m - 1, m))
        D[first] += K[first] * inv_h2
        D[last] += K[last] * inv_h2
    return D.reshape(-1)


def assemble_csr(prob: Problem, mu) -> sp.csr_matrix:
    """A(mu) as a sparse matrix, built face by face from the same definition."""
    n = prob.n_dof
    K = node_coefficient(prob, mu).reshape(-1)
    idx = np.arange(n).reshape(grid_shape(prob))
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    nd = prob.dim
    for d in range(nd):
        ax = nd - 1 - d
        m = prob.dims[d]
        inv_h2 = float(m + 1) ** 2
        i = idx[_sl(nd, ax, slice(0, m - 1))].reshape(-1)
        j = idx[_sl(nd, ax, slice(1, m))].reshape(-1)
        kf = 0.5 * (K[i] + K[j]) * inv_h2
        rows += [i, j]
        cols += [j, i]
        vals += [-kf, -kf]
        np.add.at(diag, i, kf)
        np.add.at(diag, j, kf)
        for s in (slice(0, 1), slice(m - 1, m)):
            b = idx[_sl(nd, ax, s)].reshape(-1)
            np.add.at(diag, b, K[b] * inv_h2)
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def affine_term(prob: Problem, q: int, v) -> np.ndarray:
    """A_q v, the q-th affine term: A(mu) with mu = e_q (Theta_q(mu) = mu_q)."""
    e = np.zeros(prob.n_mu)
    e[q] = 1.0
    return apply(prob, e, v)


def node_coordinates(prob: Problem):
    """Per-direction coordinate arrays (x, y[, z]) broadcastable to the grid shape."""
    coords = []
    for d in range(prob.dim):
        ax = prob.dim - 1 - d
        m = prob.dims[d]
        shape = [1] * prob.dim
        shape[ax] = m
        coords.append(((np.arange(m) + 1.0) / (m + 1.0)).reshape(shape))
    return coords


def boundary_lift(prob: Problem, F, G) -> np.ndarray:
    """sum over the boundary faces of node i of F(i) g(j) / h_d^2 (flat), with F grid-shaped
    and G the Dirichlet data on the grid extended by the boundary layer (shape + 2 per axis)."""
    nd = prob.dim
    out = np.zeros(grid_shape(prob))
    inner = tuple(slice(1, -1) for _ in range(nd))
    for d in range(nd):
        ax = nd - 1 - d
        m = prob.dims[d]
        inv_h2 = float(m + 1) ** 2
        for node, ghost in ((0, 0), (m - 1, m + 1)):
            sel = list(inner)
            sel[ax] = slice(ghost, ghost + 1)
            g = G[tuple(sel)]                               # boundary nodes facing this layer
            lay = _sl(nd, ax, slice(node, node + 1))
            out[lay] += F[lay] * g * inv_h2
    return out.reshape(-1)


def load_term(prob: Problem, r: int) -> np.ndarray:
    """f_r at the nodes (flat)."""
    ld = prob.loads[r]
    shape = grid_shape(prob)
    if ld.kind == "const":
        return np.ones(prob.n_dof)
    if ld.kind == "array":
        return np.asarray(prob.load_values(r), dtype=np.float64).copy()
    if ld.kind == "boundary":
        G = np.asarray(prob.load_values(r), dtype=np.float64).reshape(tuple(s + 2 for s in shape))
        return boundary_lift(prob, node_fields(prob)[ld.field], G)
    coords = node_coordinates(prob)
    d2 = np.zeros(shape)
    for d in range(prob.dim):
        d2 = d2 + (coords[d] - ld.center[d]) ** 2
    return np.exp(-d2 / (2.0 * ld.sigma ** 2)).reshape(-1)


def load_weight(prob: Problem, r: int, mu) -> float:
    """phi_r(mu)."""
    p = prob.loads[r].param
    return 1.0 if p < 0 else float(mu[p])


def load(prob: Problem, mu) -> np.ndarray:
    """f(mu) = sum_r phi_r(mu) f_r (eq. 12)."""
    f = np.zeros(prob.n_dof)
    for r in range(len(prob.loads)):
        f += load_weight(prob, r, mu) * load_term(prob, r)
    return f


def colour(prob: Problem) -> np.ndarray:
    """Red-black colour of every node: (i_x + i_y [+ i_z]) mod 2 with 0-based indices (flat)."""
    s = np.zeros(grid_shape(prob), dtype=np.int64)
    for d in range(prob.dim):
        ax = prob.dim - 1 - d
        shape = [1] * prob.dim
        shape[ax] = prob.dims[d]
        s = s + np.arange(prob.dims[d]).reshape(shape)
    return (s % 2).reshape(-1)
