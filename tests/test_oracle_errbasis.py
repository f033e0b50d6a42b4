"""Pins of the oracle's error basis of the learned warm start (oracle/errbasis.py)."""
import numpy as np
import pytest

import workloads as wl
from oracle import direct, errbasis, greedy, rb


@pytest.fixture(scope="module")
def case():
    w = wl.small((24, 20), (2, 2), n_basis=4, n_train=30, bumps=True)
    basis = greedy.greedy(w.problem, w.train_mu(), w.n_basis)
    mus = wl.mlp_train_mu(w, 12)
    X = np.stack([direct.sparse_direct(w.problem, m) for m in mus])
    return w, basis, mus, X


def test_errors_are_orthogonal_to_the_galerkin_residual_space(case):
    """e = x - x_hat satisfies W^T A(mu) e = 0 (Galerkin orthogonality, Lemma 3): the errors are
    A-orthogonal to span(W), a fact independent of how the basis V is formed."""
    w, B, mus, X = case
    from oracle import problem as pb
    E = errbasis.errors(B, mus, X)
    for s in range(len(mus)):
        Ae = pb.apply(w.problem, mus[s], E[:, s])
        assert np.abs(B.W.T @ Ae).max() <= 1e-10 * np.abs(pb.apply(w.problem, mus[s], X[s]) @ B.W).max()


@pytest.mark.parametrize("m", [1, 3, 6])
def test_pod_is_optimal_and_orthonormal(case, m):
    """Eckart-Young: ||E - V V^T E||_F^2 equals the sum of the discarded squared singular values
    (computed independently as the eigenvalues of E^T E), and no other orthonormal basis of the same
    size (random ones tried) does better."""
    w, B, mus, X = case
    E = errbasis.errors(B, mus, X)
    V, Z, sig = errbasis.error_basis(B, mus, X, m)
    assert np.abs(V.T @ V - np.eye(m)).max() < 1e-12
    np.testing.assert_allclose(Z, V.T @ E, rtol=0, atol=1e-14 * np.abs(E).max())
    lam = np.sort(np.linalg.eigvalsh(E.T @ E))[::-1]
    res = np.linalg.norm(E - V @ Z) ** 2
    assert abs(res - lam[m:].sum()) <= 1e-8 * lam.sum()
    rng = np.random.default_rng(3)
    for _ in range(5):
        Q, _ = np.linalg.qr(rng.standard_normal((E.shape[0], m)))
        assert np.linalg.norm(E - Q @ (Q.T @ E)) ** 2 >= res * (1 - 1e-12)


def test_method_of_snapshots_spans_the_same_space(case):
    """The Gram-matrix route the CUDA library takes gives the same singular values and, mode by
    mode up to sign, the same basis while the singular values are separated."""
    w, B, mus, X = case
    V1, Z1, s1 = errbasis.error_basis(B, mus, X, 4)
    V2, Z2, s2 = errbasis.error_basis_gram(B, mus, X, 4)
    np.testing.assert_allclose(s2, s1, rtol=1e-8)
    signs = np.sign(np.sum(V1 * V2, axis=0))
    assert np.abs(V2 * signs - V1).max() < 1e-6
    np.testing.assert_allclose(Z2 * signs[:, None], Z1, rtol=0, atol=1e-6 * np.abs(Z1).max())


def test_full_rank_basis_reproduces_the_training_solutions(case):
    """With as many modes as snapshots the start x_hat + V z(mu_s) is the training solution itself."""
    w, B, mus, X = case
    S = len(mus)
    V, Z, sig = errbasis.error_basis(B, mus, X, S)
    for s in range(S):
        x0 = errbasis.warm_start(B, V, mus[s], Z[:, s])
        assert np.linalg.norm(x0 - X[s]) <= 1e-10 * np.linalg.norm(X[s])
