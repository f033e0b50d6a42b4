"""Pins of the oracle's operator, load and colouring (eq. 1, eq. 12)."""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import problem as pb
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_solutions.txt")

SMALL = [((4, 4), (2, 2)), ((5, 7), (3, 2)), ((3, 3, 3), (2, 2, 2)), ((4, 3, 5), (2, 1, 3)),
         ((6,  1), (2, 1)), ((1, 1, 1), (1, 1, 1))]


def _prob(dims, blocks, bumps=False):
    return wl.small(dims, blocks, n_basis=1, bumps=bumps).problem


def _mu(prob, seed=7):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(0.1), np.log(10.0), prob.n_mu))


@pytest.mark.parametrize("dims,blocks", SMALL)
def test_apply_matches_incidence_form(dims, blocks):
    prob = _prob(dims, blocks)
    mu = _mu(prob)
    A = pins.incidence_operator(dims, blocks, mu)
    v = np.random.default_rng(1).standard_normal(prob.n_dof)
    np.testing.assert_allclose(pb.apply(prob, mu, v), A @ v, rtol=1e-13, atol=1e-13 * np.abs(A).max())
    np.testing.assert_allclose(pb.assemble_csr(prob, mu).toarray(), A, rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(pb.diagonal(prob, mu), np.diag(A), rtol=1e-14)


@pytest.mark.parametrize("dims,blocks", SMALL[:4])
def test_symmetric_positive_affine(dims, blocks):
    prob = _prob(dims, blocks)
    mu = _mu(prob, 3)
    rng = np.random.default_rng(2)
    v, w = rng.standard_normal((2, prob.n_dof))
    Av, Aw = pb.apply(prob, mu, v), pb.apply(prob, mu, w)
    assert abs(w @ Av - v @ Aw) <= 1e-12 * abs(w @ Av) + 1e-9
    assert v @ Av > 0
    affine = sum(mu[q] * pb.affine_term(prob, q, v) for q in range(prob.P))
    np.testing.assert_allclose(affine, Av, rtol=1e-12, atol=1e-10)


def test_hand_derived_solutions():
    """Tiny grids whose solution is worked out by hand (tests/golden/hand_solutions.txt)."""
    n_cases = 0
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        name, dims, blocks, mu, f, x, _ = [s.strip() for s in line.split("|")]
        dims = tuple(int(t) for t in dims.split(","))
        blocks = tuple(int(t) for t in blocks.split(","))
        mu = np.array([float(t) for t in mu.split(",")])
        x = np.array([float(t) for t in x.split(",")])
        prob = _prob(dims, blocks)
        A = pb.assemble_csr(prob, mu).toarray()
        np.testing.assert_allclose(np.linalg.solve(A, np.full(prob.n_dof, float(f))), x, rtol=1e-14,
                                   err_msg=name)
        np.testing.assert_allclose(pb.apply(prob, mu, x), np.full(prob.n_dof, float(f)), rtol=1e-13,
                                   err_msg=name)
        n_cases += 1
    assert n_cases == 4


def test_block_map_sizes():
    # floor(i nb / m): near-equal blocks, larger ones first
    assert np.bincount(pb.block_index(64, 2)).tolist() == [32, 32]
    assert np.bincount(pb.block_index(512, 3)).tolist() == [171, 171, 170]
    assert np.bincount(pb.block_index(256, 3)).tolist() == [86, 85, 85]
    assert np.bincount(pb.block_index(128, 2)).tolist() == [64, 64]


def test_loads_at_nodes():
    prob = _prob((9, 7), (1, 1), bumps=True)
    mu = np.array([2.0, 0.3, 0.7])
    f = pb.load(prob, mu).reshape(7, 9)
    # node (ix=4, iy=2): coordinates (5/10, 3/8)
    x, y = 5 / 10, 3 / 8
    expect = 1.0
    for r, w in ((1, 0.3), (2, 0.7)):
        c, s = prob.loads[r].center, prob.loads[r].sigma
        expect += w * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2) / (2 * s * s))
    assert abs(f[2, 4] - expect) < 1e-15 * 4


@pytest.mark.parametrize("dims", [(5, 4), (3, 4, 5)])
def test_colouring_is_a_two_colouring(dims):
    prob = _prob(dims, (1,) * len(dims))
    A = pb.assemble_csr(prob, np.ones(1)).toarray()
    col = pb.colour(prob)
    i, j = np.nonzero(A - np.diag(np.diag(A)))
    assert np.all(col[i] != col[j])
    assert col[0] == 0
