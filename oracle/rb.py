"""Reduced-basis approximation (Section 2.1, 2.3), RBI (Alg. 2) and RBCG (Alg. 3).

Notation follows the paper: W = W_N (N_dof x N, orthonormal columns), the
precomputed affine blocks A_{N,q} = W^T A_q W and f_{N,r} = W^T f_r (eq. 12c),
the online reduced system A_N(mu) = sum_q Theta_q(mu) A_{N,q},
f_N(mu) = sum_r Phi_r(mu) f_{N,r} (eq. 12b), factored by Cholesky (Section 2.1).

Readings of the paper (where it is silent or loose):
  * the stopping test ||r|| < eps is taken relative, ||r|| < tol ||f(mu)||
    (the relative residual of eq. relerr); it is applied to the recurrence
    residual, and at exit the true residual f - A x is recomputed: if it is
    not below tol either, the residual is replaced by the true one and the
    iteration restarts from the current x (counted in the same budget) with
    the same stopping test.  `restart_factor` < 1 makes the restarted cycles
    aim at restart_factor * tol instead (a solver policy, not the paper's);
  * the adaptive choice of N at the end of Section 4.1: when the residual
    falls by less than a factor gamma in one iteration,
    ||r_k|| / ||r_{k+1}|| < gamma, the next preconditioner application uses
    one more basis vector (N <- N + 1, at most the basis size).  W_N is nested
    in W_{N+1}, so the reduced matrix of size N is the leading block of the
    full A_N(mu); the starting N is not given in the paper (argument
    `adaptive_n`, off when 0);
  * Alg. 3 step 1 writes A without mu; it is A(mu).  With x_0 = 0 the first
    residual is f itself, so no matrix-vector product is spent on it;
  * RBI(A, r, W, 1) inside Alg. 3 starts from x = 0, so its own residual is r:
    y = W A_N^{-1} W^T r followed by the smoother on A y = r;
  * beta is the printed Fletcher-Reeves form y_{k+1}^T r_{k+1} / y_k^T r_k;
    the Polak-Ribiere form y_{k+1}^T (r_{k+1} - r_k) / y_k^T r_k is an option
    (the RBI preconditioner is not symmetric).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg as sla

from . import problem as pb
from . import smoothers


@dataclasses.dataclass
class Basis:
    prob: object
    W: np.ndarray            # N_dof x N, orthonormal columns
    ANq: np.ndarray          # Q x N x N, A_{N,q} = W^T A_q W
    fNr: np.ndarray          # R x N,     f_{N,r} = W^T f_r
    R: Optional[np.ndarray] = None   # N x N upper triangular, snapshots X = W R
    selected: Optional[List[int]] = None

    @property
    def N(self) -> int:
        return self.W.shape[1]

    def truncated(self, N: int) -> "Basis":
        """The nested basis W_N taken from the first N columns (W_N in W_{N+1})."""
        R = None if self.R is None else self.R[:N, :N].copy()
        sel = None if self.selected is None else list(self.selected[:N])
        return Basis(self.prob, self.W[:, :N].copy(), self.ANq[:, :N, :N].copy(),
                     self.fNr[:, :N].copy(), R, sel)


def affine_blocks(prob, W: np.ndarray):
    """A_{N,q} = W^T A_q W and f_{N,r} = W^T f_r for all q, r (eq. 12c)."""
    Q, R = prob.P, len(prob.loads)
    N = W.shape[1]
    ANq = np.zeros((Q, N, N))
    for q in range(Q):
        AqW = np.stack([pb.affine_term(prob, q, W[:, j]) for j in range(N)], axis=1)
        ANq[q] = W.T @ AqW
    fNr = np.stack([W.T @ pb.load_term(prob, r) for r in range(R)], axis=0)
    return ANq, fNr


def reduced_system(basis: Basis, mu):
    """A_N(mu) and f_N(mu) by eq. 12b (Theta_q(mu) = mu_q)."""
    prob = basis.prob
    A_N = np.zeros((basis.N, basis.N))
    for q in range(prob.P):
        A_N += mu[q] * basis.ANq[q]
    f_N = np.zeros(basis.N)
    for r in range(len(prob.loads)):
        f_N += pb.load_weight(prob, r, mu) * basis.fNr[r]
    return A_N, f_N


def reduced_factor(basis: Basis, mu):
    """Cholesky factor of A_N(mu) (lower), raising if A_N(mu) is not SPD."""
    A_N, _ = reduced_system(basis, mu)
    return sla.cho_factor(A_N, lower=True)


def rb_coefficients(basis: Basis, mu) -> np.ndarray:
    """a_N(mu) solving A_N(mu) a_N = f_N(mu) (eq. 2)."""
    A_N, f_N = reduced_system(basis, mu)
    return sla.cho_solve(sla.cho_factor(A_N, lower=True), f_N)


def rb_approximation(basis: Basis, mu) -> np.ndarray:
    """x_hat(mu) = W a_N(mu) (eq. 3)."""
    return basis.W @ rb_coefficients(basis, mu)


def rbi_step(basis: Basis, mu, factor, x, b, smoother="rbgs", nu=1, omega=2.0 / 3.0):
    """One pass of Alg. 2 steps 2, 4-7 on A(mu) x = b: returns (x_new, r)."""
    prob = basis.prob
    r = b - pb.apply(prob, mu, x)
    if basis.N > 0:
        e_N = sla.cho_solve(factor, basis.W.T @ r)
        x = x + basis.W @ e_N
    return smoothers.smooth(smoother, prob, mu, b, x, nu, omega), r


def rbi_precondition(basis: Basis, mu, factor, r, smoother="rbgs", nu=1, omega=2.0 / 3.0):
    """y = RBI(A(mu), r, W_N, 1) from x = 0: y = W A_N^{-1} W^T r, then S(A, r, y)."""
    prob = basis.prob
    y = np.zeros_like(r)
    if basis.N > 0:
        y = basis.W @ sla.cho_solve(factor, basis.W.T @ r)
    return smoothers.smooth(smoother, prob, mu, r, y, nu, omega)


@dataclasses.dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    rel_res: float                 # true ||f - A x|| / ||f|| at exit
    converged: bool
    history: List[float]           # relative residual after each iteration
    restarts: int = 0
    n_history: Optional[List[int]] = None   # RBCG: basis size N of each preconditioner application


def rbi(basis: Basis, mu, tol=1e-10, max_iter=1000, smoother="rbgs", nu=1,
        omega=2.0 / 3.0, x0=None, b=None) -> SolveResult:
    """Alg. 2.  x <- 0; repeat: r = b - A x; stop if ||r|| < tol ||b||;
    e_N = A_N^{-1} W^T r; x += W e_N; x = S(A, b, x)."""
    prob = basis.prob
    b = pb.load(prob, mu) if b is None else np.asarray(b, dtype=np.float64)
    bn = np.linalg.norm(b)
    factor = reduced_factor(basis, mu) if basis.N > 0 else None
    x = np.zeros(prob.n_dof) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    hist = []
    it = 0
    while True:
        r = b - pb.apply(prob, mu, x)
        rel = np.linalg.norm(r) / bn
        hist.append(rel)
        if rel < tol or it >= max_iter:
            return SolveResult(x, it, rel, rel < tol, hist)
        if basis.N > 0:
            x = x + basis.W @ sla.cho_solve(factor, basis.W.T @ r)
        x = smoothers.smooth(smoother, prob, mu, b, x, nu, omega)
        it += 1


def leading_factor(basis: Basis, mu, k: int):
    """Cholesky factor of the leading k x k block of A_N(mu): the reduced matrix of the
    nested basis W_k (the first k columns of W)."""
    A_N, _ = reduced_system(basis, mu)
    return sla.cho_factor(A_N[:k, :k], lower=True)


def rbcg(basis: Basis, mu, tol=1e-10, max_iter=5000, smoother="rbgs", nu=1,
         omega=2.0 / 3.0, beta="fr", x0=None, b=None, apply_counter=None,
         restart_factor=1.0, adaptive_n=0, gamma=10.0) -> SolveResult:
    """Alg. 3, with the readings listed in the module docstring.

    adaptive_n = 0 uses the whole basis in every preconditioner application;
    adaptive_n = k >= 1 starts with W_k and grows N by one after every
    iteration whose residual ratio ||r_k|| / ||r_{k+1}|| is below gamma (end of
    Section 4.1).  The N of each application is recorded in `n_history`.
    """
    prob = basis.prob
    b = pb.load(prob, mu) if b is None else np.asarray(b, dtype=np.float64)
    bn = np.linalg.norm(b)

    def A(v):
        if apply_counter is not None:
            apply_counter[0] += 1
        return pb.apply(prob, mu, v)

    n_cur = basis.N if adaptive_n <= 0 else min(adaptive_n, basis.N)
    nested = {}

    def Minv(r):
        """RBI(A, r, W_N, 1) with the current N (the nested basis W_N = first N columns)."""
        n_hist.append(n_cur)
        if n_cur not in nested:
            sub = basis if n_cur == basis.N else basis.truncated(n_cur)
            nested[n_cur] = (sub, reduced_factor(sub, mu) if n_cur > 0 else None)
        sub, factor = nested[n_cur]
        return rbi_precondition(sub, mu, factor, r, smoother, nu, omega)

    n_hist: List[int] = []
    if x0 is None:
        x = np.zeros(prob.n_dof)
        r = b.copy()
    else:
        x = np.array(x0, dtype=np.float64, copy=True)
        r = b - A(x)
    hist = [np.linalg.norm(r) / bn]
    it, restarts = 0, 0
    target = tol
    while True:
        y = Minv(r) if hist[-1] >= target else None
        p = None if y is None else y.copy()
        rho = None if y is None else r @ y
        while y is not None and it < max_iter:
            q = A(p)
            alpha = rho / (p @ q)
            x = x + alpha * p
            r_old = r
            r = r - alpha * q
            it += 1
            hist.append(np.linalg.norm(r) / bn)
            if hist[-1] < target:
                break
            if adaptive_n > 0 and n_cur < basis.N and hist[-2] < gamma * hist[-1]:
                n_cur += 1            # ||r_k|| / ||r_{k+1}|| < gamma
            y = Minv(r)
            rho_new = r @ y
            if beta == "fr":
                bet = rho_new / rho
            elif beta == "pr":
                bet = (rho_new - r_old @ y) / rho
            else:
                raise ValueError(beta)
            p = y + bet * p
            rho = rho_new
        # the recurrence said converged (or the budget ran out): check the true residual
        r_true = b - pb.apply(prob, mu, x)
        rel = np.linalg.norm(r_true) / bn
        if rel < tol or it >= max_iter:
            return SolveResult(x, it, rel, rel < tol, hist, restarts, n_hist)
        r = r_true
        hist[-1] = rel
        restarts += 1
        target = restart_factor * tol
