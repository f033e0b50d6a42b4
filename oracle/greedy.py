"""Greedy construction of the RB space: Alg. 1, the adaptive variant Alg. 4 and the
multi-fidelity construction of Section 4.2 (last paragraph).

Steps, per N = 1..N_max (Section 2.2):
  3. solve A(mu_N) x(mu_N) = f(mu_N) (sparse direct or CG for Alg. 1; RBCG with
     W_{N-1} for Alg. 4, plain smoother-preconditioned CG when N = 1);
  4. W_N = MGS(W_{N-1}, x(mu_N)): modified Gram-Schmidt against the previous
     columns, done twice (one re-orthogonalisation pass) so that W^T W = I
     holds to round-off; the R factor of the snapshots X = W R is kept;
  5. grow A_{N,q} = W^T A_q W and f_{N,r} = W^T f_r by the new row and column
     (eq. 12c) and solve A_N(mu) x_N(mu) = f_N(mu) for every mu in Xi_train;
  6. mu_{N+1} = argmax over Xi_train of the L1 norm of the RB coefficients.

Readings of the paper:
  * mu_1 "randomly in Xi_train": the first entry of the seeded training set;
  * the L1 score of step 6 is taken on the coefficients of x_hat(mu) in the
    snapshot basis, c = R^{-1} x_N(mu) (so x_hat = X c and a selected mu_j
    scores exactly 1).  With orthonormal W the literal sum of |x_{N,n}(mu)|
    keeps the largest solution on top and would select the same mu again;
    `score="literal"` keeps that form as an option;
  * already selected parameters are excluded; ties go to the lowest index;
    a candidate whose snapshot leaves an MGS residual below 1e-10 ||x|| is
    dropped and the next best candidate is taken.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import direct
from . import problem as pb
from . import rb


def mgs_twice(W: np.ndarray, x: np.ndarray):
    """Two passes of modified Gram-Schmidt of x against the columns of W.

    Returns (v, coeffs, norm) with x = W coeffs + v, v orthogonal to W, norm = ||v||.
    """
    v = np.array(x, dtype=np.float64, copy=True)
    coeffs = np.zeros(W.shape[1])
    for _ in range(2):
        for j in range(W.shape[1]):
            c = W[:, j] @ v
            v = v - c * W[:, j]
            coeffs[j] += c
    return v, coeffs, np.linalg.norm(v)


def scores(basis: rb.Basis, train_mu: np.ndarray, kind: str = "snapshot") -> np.ndarray:
    """Step 6 criterion for every training parameter."""
    out = np.empty(len(train_mu))
    for i, mu in enumerate(train_mu):
        a = rb.rb_coefficients(basis, mu)
        if kind == "snapshot":
            c = sla.solve_triangular(basis.R, a, lower=False)
        elif kind == "literal":
            c = a
        else:
            raise ValueError(kind)
        out[i] = np.abs(c).sum()
    return out


def truth_solve(prob, mu, method: str, basis: rb.Basis | None, tol: float):
    if method == "direct":
        return direct.sparse_direct(prob, mu)
    if method == "cg":
        return direct.cg(prob, mu, tol=tol)[0]
    if method == "rbcg":      # Alg. 4 step 3: RBCG with W_{N-1} (N = 1: no basis)
        return rb.rbcg(basis, mu, tol=tol, max_iter=100000).x
    raise ValueError(method)


def grow(prob, basis: rb.Basis, x: np.ndarray, candidate: int, drop_tol: float = 1e-10):
    """Steps 4-5 for one snapshot x: modified Gram-Schmidt (twice) against W, the new column of
    W, the snapshot factor R and the new row and column of A_{N,q}, f_{N,r} (eq. 12c).
    Returns the grown basis, or None when x lies inside span(W) (remainder below drop_tol ||x||)."""
    Q, R = prob.P, len(prob.loads)
    v, coeffs, nrm = mgs_twice(basis.W, x)
    if nrm < drop_tol * np.linalg.norm(x):
        return None
    N = basis.N + 1
    w = v / nrm
    W = np.concatenate([basis.W, w[:, None]], axis=1)
    Rf = np.zeros((N, N))
    Rf[:N - 1, :N - 1] = basis.R
    Rf[:N - 1, N - 1] = coeffs
    Rf[N - 1, N - 1] = nrm
    ANq = np.zeros((Q, N, N))
    ANq[:, :N - 1, :N - 1] = basis.ANq
    for q in range(Q):
        col = W.T @ pb.affine_term(prob, q, w)
        ANq[q, :, N - 1] = col
        ANq[q, N - 1, :] = col
    fNr = np.zeros((R, N))
    fNr[:, :N - 1] = basis.fNr
    for r in range(R):
        fNr[r, N - 1] = w @ pb.load_term(prob, r)
    return rb.Basis(prob, W, ANq, fNr, Rf, basis.selected + [candidate])


def empty_basis(prob) -> rb.Basis:
    return rb.Basis(prob, np.zeros((prob.n_dof, 0)), np.zeros((prob.P, 0, 0)), np.zeros((len(prob.loads), 0)),
                    np.zeros((0, 0)), [])


def multi_fidelity(prob, coarse, train_mu: np.ndarray, n_max: int, truth: str = "direct",
                   score: str = "snapshot", truth_tol: float = 1e-13, drop_tol: float = 1e-10) -> rb.Basis:
    """Section 4.2, last paragraph: the greedy runs on the coarse grid and selects the parameter
    sample S_N; the snapshots of S_N are then solved on the fine grid (`prob`) and enter the fine
    basis in the selection order (a snapshot inside the span of the earlier ones is skipped).
    The coarse problem has the fine one's blocks, loads and parameters."""
    sample = greedy(coarse, train_mu, n_max, truth, score, truth_tol, drop_tol).selected
    basis = empty_basis(prob)
    for j in sample:
        x = truth_solve(prob, train_mu[j], truth, basis, truth_tol)
        grown = grow(prob, basis, x, j, drop_tol)
        if grown is not None:
            basis = grown
    return basis


def greedy(prob, train_mu: np.ndarray, n_max: int, truth: str = "direct",
           score: str = "snapshot", truth_tol: float = 1e-13, drop_tol: float = 1e-10) -> rb.Basis:
    """Alg. 1 (truth = "direct" or "cg") or Alg. 4 (truth = "rbcg")."""
    basis = empty_basis(prob)
    excluded = set()
    candidate = 0                              # step 0: mu_1 = Xi_train[0]
    last_scores = None
    while basis.N < n_max:
        mu = train_mu[candidate]
        x = truth_solve(prob, mu, truth, basis, truth_tol)
        grown = grow(prob, basis, x, candidate, drop_tol)
        excluded.add(candidate)
        if grown is None:
            if last_scores is None:
                raise RuntimeError("first snapshot is zero")
            s = last_scores.copy()
            s[list(excluded)] = -np.inf
            if not np.isfinite(s.max()):
                break
            candidate = int(np.argmax(s))
            continue
        basis = grown
        if basis.N == n_max:
            break
        last_scores = scores(basis, train_mu, score)
        s = last_scores.copy()
        s[list(excluded)] = -np.inf
        if not np.isfinite(s.max()):
            break
        candidate = int(np.argmax(s))
    return basis
