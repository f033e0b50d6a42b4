"""Pins of the oracle's truth solves and smoothers (eq. 1, eq. 8)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as wl
from oracle import direct, smoothers
from oracle import problem as pb
from tests import pins


def _prob(dims, blocks, bumps=False):
    return wl.small(dims, blocks, n_basis=1, bumps=bumps).problem


def _mu(prob, seed=5):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(0.1), np.log(10.0), prob.n_mu))


@pytest.mark.parametrize("dims,blocks", [((6, 5), (2, 2)), ((4, 3, 5), (2, 1, 3))])
def test_sparse_direct_matches_dense_solve(dims, blocks):
    prob = _prob(dims, blocks, bumps=True)
    mu = _mu(prob)
    A = pins.incidence_operator(dims, blocks, mu)
    f = pb.load(prob, mu)
    np.testing.assert_allclose(direct.sparse_direct(prob, mu), np.linalg.solve(A, f), rtol=1e-12)


@pytest.mark.parametrize("dims", [(64, 64), (300, 257), (32, 32, 32), (17, 9, 12)])
@pytest.mark.parametrize("bumps", [False, True])
def test_truth_matches_closed_form_at_equal_coefficients(dims, bumps):
    blocks = (3,) * len(dims)
    prob = _prob(dims, blocks, bumps=bumps)
    c = 2.75
    mu = np.full(prob.n_mu, c)
    mu[prob.P:] = [0.4, 0.9][: prob.n_mu - prob.P]
    f = pb.load(prob, mu)
    x_cf = pins.laplace_closed_form(dims, c, f)
    x = direct.sparse_direct(prob, mu)
    assert np.linalg.norm(x - x_cf) <= 1e-12 * np.linalg.norm(x_cf)


def test_cg_matches_direct_and_jacobi_pcg_matches_library():
    prob = _prob((24, 20), (3, 2), bumps=True)
    mu = _mu(prob, 11)
    xs = direct.sparse_direct(prob, mu)
    x, it, hist = direct.cg(prob, mu, tol=1e-12)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert hist[-1] < 1e-12 and all(h >= 1e-12 for h in hist[:-1])
    # Jacobi-preconditioned CG: same iterates as scipy's PCG
    D = pb.diagonal(prob, mu)
    A = pb.assemble_csr(prob, mu)
    f = pb.load(prob, mu)
    xj, itj, _ = direct.cg(prob, mu, tol=1e-8, precond=lambda r: r / D)
    lib_it = [0]
    xl, info = spla.cg(A, f, rtol=1e-8, atol=0.0, M=spla.LinearOperator(A.shape, matvec=lambda r: r / D),
                       maxiter=10000, callback=lambda xk: lib_it.__setitem__(0, lib_it[0] + 1))
    assert info == 0
    assert abs(itj - lib_it[0]) <= 1
    assert np.linalg.norm(xj - xl) <= 1e-6 * np.linalg.norm(xl)


@pytest.mark.parametrize("dims,blocks", [((5, 4), (2, 2)), ((3, 4, 3), (1, 2, 1))])
def test_red_black_gs_is_textbook_gs_in_red_black_order(dims, blocks):
    prob = _prob(dims, blocks)
    mu = _mu(prob, 9)
    A = pins.incidence_operator(dims, blocks, mu)
    rng = np.random.default_rng(3)
    b, y = rng.standard_normal((2, prob.n_dof))
    order = pins.red_black_permutation(dims)
    for sweeps in (1, 3):
        np.testing.assert_allclose(smoothers.red_black_gs(prob, mu, b, y, sweeps),
                                   pins.textbook_gs(A, b, y, sweeps, order), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(smoothers.lexicographic_gs(prob, mu, b, y, sweeps),
                                   pins.textbook_gs(A, b, y, sweeps), rtol=1e-12, atol=1e-12)
    Dm = np.diag(A)
    np.testing.assert_allclose(smoothers.jacobi(prob, mu, b, y, 1, 0.8), y + 0.8 * (b - A @ y) / Dm,
                               rtol=1e-13, atol=1e-13)


def test_gs_contracts_the_energy_norm():
    prob = _prob((16, 12), (2, 2))
    mu = _mu(prob, 2)
    xs = direct.sparse_direct(prob, mu)
    f = pb.load(prob, mu)
    y = np.random.default_rng(4).standard_normal(prob.n_dof)
    enorm = lambda e: np.sqrt(e @ pb.apply(prob, mu, e))
    prev = enorm(y - xs)
    for _ in range(5):
        y = smoothers.red_black_gs(prob, mu, f, y)
        cur = enorm(y - xs)
        assert cur < prev
        prev = cur
