"""Error basis of the learned warm start (test infrastructure only, FP64).

Any starting vector in span(W) is sent by the first RB correction of Alg. 3
(y = W A_N^{-1} W^T r plus smoothing) to about the same iterate, so a network
that predicts coefficients in span(W) gains at most the Galerkin step.  A start
that can gain must leave span(W): x_0 = x_hat(mu) + V z(mu), with x_hat the RB
approximation of eq. 3 (exact and cheap, eq. 2) and V an orthonormal basis of
the errors e(mu) = x(mu) - x_hat(mu) of training solutions (proper orthogonal
decomposition: the leading left singular vectors of E = [e_1 .. e_S]).  The
network predicts the coefficients z = V^T e.

  error_basis(basis, mus, X, m)   V, Z = V^T E and the singular values, by SVD
  error_basis_gram(...)           the same subspace by the method of snapshots
                                  (eigenvectors of E^T E), the route the CUDA
                                  library takes
  warm_start(basis, V, mu, z)     x_0 = x_hat(mu) + V z
"""
from __future__ import annotations

import numpy as np

from . import rb


def errors(basis: rb.Basis, mus, X) -> np.ndarray:
    """E = [x_s - x_hat(mu_s)] as columns (N_dof x S)."""
    X = np.asarray(X, dtype=np.float64)
    return np.stack([X[s] - rb.rb_approximation(basis, mus[s]) for s in range(len(mus))], axis=1)


def error_basis(basis: rb.Basis, mus, X, m: int):
    """POD of the errors by the thin SVD E = U diag(sigma) V^T: the first m left singular
    vectors, Z = V^T E ([m][S]) and the m leading singular values."""
    E = errors(basis, mus, X)
    U, sig, _ = np.linalg.svd(E, full_matrices=False)
    V = U[:, :m]
    return V, V.T @ E, sig[:m]


def error_basis_gram(basis: rb.Basis, mus, X, m: int):
    """The same by the method of snapshots: E^T E = Phi diag(lambda) Phi^T, V = E Phi_m
    diag(lambda_m)^{-1/2}, Z = diag(lambda_m)^{1/2} Phi_m^T, sigma = lambda^{1/2}."""
    E = errors(basis, mus, X)
    lam, Phi = np.linalg.eigh(E.T @ E)
    order = np.argsort(lam)[::-1][:m]
    lam, Phi = lam[order], Phi[:, order]
    sig = np.sqrt(np.maximum(lam, 0.0))
    V = (E @ Phi) / sig
    return V, sig[:, None] * Phi.T, sig


def warm_start(basis: rb.Basis, V, mu, z) -> np.ndarray:
    """x_0 = x_hat(mu) + V z."""
    return rb.rb_approximation(basis, mu) + np.asarray(V) @ np.asarray(z)
