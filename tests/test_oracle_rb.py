"""Pins of the oracle's greedy basis, RBI and RBCG (Sections 2-4, Lemmas 1-3)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as wl
from oracle import direct, greedy, rb, smoothers
from oracle import problem as pb
from tests import pins


@pytest.fixture(scope="module")
def small_case():
    w = wl.small((24, 20), (2, 2), n_basis=8, n_train=40, bumps=True)
    basis = greedy.greedy(w.problem, w.train_mu(), w.n_basis)
    return w, basis


def test_basis_orthonormal_and_affine_blocks(small_case):
    w, B = small_case
    prob = w.problem
    assert np.abs(B.W.T @ B.W - np.eye(B.N)).max() < 1e-13
    # eq. 12c recomputed from dense affine terms built by the incidence route
    for q in range(prob.P):
        e = np.zeros(prob.n_mu); e[q] = 1.0
        Aq = pins.incidence_operator(prob.dims, prob.blocks, e)
        ref = B.W.T @ Aq @ B.W
        assert np.abs(B.ANq[q] - ref).max() <= 1e-12 * np.abs(ref).max()
    for r in range(len(prob.loads)):
        np.testing.assert_allclose(B.fNr[r], B.W.T @ pb.load_term(prob, r), rtol=1e-12, atol=1e-14)
    assert len(set(B.selected)) == B.N and B.selected[0] == 0


def test_snapshot_factor_and_scores(small_case):
    w, B = small_case
    prob, train = w.problem, w.train_mu()
    X = np.stack([direct.sparse_direct(prob, train[j]) for j in B.selected], axis=1)
    assert np.allclose(np.triu(B.R), B.R)
    assert np.linalg.norm(B.W @ B.R - X) <= 1e-11 * np.linalg.norm(X)
    s = greedy.scores(B, train)
    # a selected parameter is reproduced by its own snapshot: coefficient vector e_j
    np.testing.assert_allclose(s[B.selected], 1.0, rtol=1e-8)
    # the score by a different route: least-squares coefficients of x_hat in the snapshots
    for i in (3, 17, 31):
        xh = rb.rb_approximation(B, train[i])
        c = np.linalg.lstsq(X, xh, rcond=None)[0]
        assert abs(np.abs(c).sum() - s[i]) <= 1e-7 * s[i]


def test_greedy_choice_is_argmax_of_previous_scores():
    w = wl.small((20, 16), (2, 2), n_basis=5, n_train=30)
    B = greedy.greedy(w.problem, w.train_mu(), 5)
    train = w.train_mu()
    for N in range(1, 5):
        s = greedy.scores(B.truncated(N), train)
        s[B.selected[:N]] = -np.inf
        assert int(np.argmax(s)) == B.selected[N]


def test_lemma1_snapshot_parameter_converges_in_one_iteration(small_case):
    w, B = small_case
    mu = w.train_mu()[B.selected[3]]
    xs = direct.sparse_direct(w.problem, mu)
    np.testing.assert_allclose(rb.rb_approximation(B, mu), xs, rtol=0, atol=1e-11 * np.abs(xs).max())
    res = rb.rbi(B, mu, tol=1e-10)
    assert res.iters == 1 and res.converged
    res = rb.rbcg(B, mu, tol=1e-10)
    assert res.iters == 1 and res.converged


def test_lemma2_no_smoother_stagnates(small_case):
    w, B = small_case
    mu = w.test_mu(1)[0]
    xh = rb.rb_approximation(B, mu)
    f = pb.load(w.problem, mu)
    factor = rb.reduced_factor(B, mu)
    x1, _ = rb.rbi_step(B, mu, factor, np.zeros_like(f), f, smoother="none")
    x2, _ = rb.rbi_step(B, mu, factor, x1, f, smoother="none")
    scale = np.abs(xh).max()
    assert np.abs(x1 - xh).max() < 1e-12 * scale
    assert np.abs(x2 - x1).max() < 1e-12 * scale
    # any start in span W gives the same iterate after step 6 (x_hat)
    x0 = B.W @ np.random.default_rng(0).standard_normal(B.N)
    x1b, _ = rb.rbi_step(B, mu, factor, x0, f, smoother="none")
    assert np.abs(x1b - xh).max() < 1e-10 * scale


def test_lemma3_galerkin_orthogonality_and_energy_optimality(small_case):
    w, B = small_case
    prob = w.problem
    mu = w.test_mu(2)[1]
    f = pb.load(prob, mu)
    a = rb.rb_coefficients(B, mu)
    xh = B.W @ a
    assert np.linalg.norm(B.W.T @ (f - pb.apply(prob, mu, xh))) <= 1e-12 * np.linalg.norm(B.W.T @ f)
    xs = direct.sparse_direct(prob, mu)
    A_N, _ = rb.reduced_system(B, mu)
    en = lambda e: e @ pb.apply(prob, mu, e)
    rng = np.random.default_rng(1)
    base = en(xs - xh)
    for _ in range(20):
        d = rng.standard_normal(B.N) * 1e-3
        diff = en(xs - B.W @ (a + d)) - base
        assert diff >= 0
        assert abs(diff - d @ A_N @ d) <= 1e-7 * abs(d @ A_N @ d) + 1e-12 * base


def test_rbi_energy_error_decreases_and_reaches_truth(small_case):
    w, B = small_case
    prob = w.problem
    mu = w.test_mu(3)[2]
    xs = direct.sparse_direct(prob, mu)
    f = pb.load(prob, mu)
    factor = rb.reduced_factor(B, mu)
    en = lambda e: np.sqrt(max(e @ pb.apply(prob, mu, e), 0.0))
    x = np.zeros(prob.n_dof)
    prev = en(xs)
    for _ in range(15):
        x, _ = rb.rbi_step(B, mu, factor, x, f)
        cur = en(xs - x)
        assert cur <= prev * (1 + 1e-12)
        prev = cur
    res = rb.rbi(B, mu, tol=1e-10)
    assert res.converged and res.rel_res < 1e-10
    assert np.linalg.norm(res.x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_rbi_without_basis_is_gauss_seidel():
    w = wl.small((6, 5), (2, 2), n_basis=1)
    prob = w.problem
    mu = w.test_mu(1)[0]
    empty = rb.Basis(prob, np.zeros((prob.n_dof, 0)), np.zeros((prob.P, 0, 0)), np.zeros((1, 0)))
    res = rb.rbi(empty, mu, tol=0.0, max_iter=7)
    A = pins.incidence_operator(prob.dims, prob.blocks, mu)
    f = pb.load(prob, mu)
    ref = pins.textbook_gs(A, f, np.zeros(prob.n_dof), 7, pins.red_black_permutation(prob.dims))
    np.testing.assert_allclose(res.x, ref, rtol=1e-12, atol=1e-14)


def test_rbcg_exact_preconditioner_one_iteration():
    w = wl.small((5, 4), (2, 2), n_basis=1, bumps=True)
    prob = w.problem
    W = np.eye(prob.n_dof)
    ANq, fNr = rb.affine_blocks(prob, W)
    full = rb.Basis(prob, W, ANq, fNr)
    res = rb.rbcg(full, w.test_mu(1)[0], tol=1e-12)
    assert res.iters == 1 and res.converged


def test_rbcg_no_basis_jacobi_is_textbook_jacobi_pcg():
    """With W empty and one unweighted Jacobi sweep from 0, M^{-1} r = D^{-1} r."""
    w = wl.small((20, 18), (3, 3), n_basis=1, bumps=True)
    prob = w.problem
    mu = w.test_mu(1)[0]
    empty = rb.Basis(prob, np.zeros((prob.n_dof, 0)), np.zeros((prob.P, 0, 0)), np.zeros((3, 0)))
    calls = [0]
    res = rb.rbcg(empty, mu, tol=1e-9, smoother="jacobi", omega=1.0, apply_counter=calls)
    A = pb.assemble_csr(prob, mu)
    D = A.diagonal()
    f = pb.load(prob, mu)
    lib_it = [0]
    xl, info = spla.cg(A, f, rtol=1e-9, atol=0.0, maxiter=10000,
                       M=spla.LinearOperator(A.shape, matvec=lambda r: r / D),
                       callback=lambda xk: lib_it.__setitem__(0, lib_it[0] + 1))
    assert info == 0 and abs(res.iters - lib_it[0]) <= 1
    assert np.linalg.norm(res.x - xl) <= 1e-7 * np.linalg.norm(xl)
    # one matrix-vector product per iteration (Section 4.1)
    assert calls[0] == res.iters
    # symmetric preconditioner: the two beta forms agree
    res_pr = rb.rbcg(empty, mu, tol=1e-9, smoother="jacobi", omega=1.0, beta="pr")
    assert abs(res_pr.iters - res.iters) <= 1


@pytest.mark.parametrize("beta", ["fr", "pr"])
def test_rbcg_converges_to_truth_faster_than_cg(small_case, beta):
    w, B = small_case
    prob = w.problem
    for mu in w.test_mu(3):
        xs = direct.sparse_direct(prob, mu)
        calls = [0]
        res = rb.rbcg(B, mu, tol=1e-10, beta=beta, apply_counter=calls)
        assert res.converged and res.rel_res < 1e-10
        assert calls[0] == res.iters
        assert np.linalg.norm(res.x - xs) <= 1e-8 * np.linalg.norm(xs)
        _, it_cg, _ = direct.cg(prob, mu, tol=1e-10)
        assert res.iters < it_cg


def test_adaptive_greedy_matches_plain_greedy():
    """Alg. 4 (snapshots by RBCG with W_{N-1}) selects the same parameters as Alg. 1."""
    w = wl.small((20, 16), (2, 2), n_basis=5, n_train=30)
    B1 = greedy.greedy(w.problem, w.train_mu(), 5, truth="direct")
    B4 = greedy.greedy(w.problem, w.train_mu(), 5, truth="rbcg", truth_tol=1e-13)
    assert B1.selected == B4.selected
    signs = np.sign(np.sum(B1.W * B4.W, axis=0))
    assert np.abs(B1.W - B4.W * signs).max() < 1e-8


def test_nested_reduced_factor(small_case):
    """W_N is nested in W_{N+1} (Section 4.1, end): the reduced matrix of the first k basis
    vectors is the leading k x k block of A_N(mu), and its Cholesky factor is the leading block
    of the full factor, so growing N adds one row to the factor."""
    w, B = small_case
    for mu in w.test_mu(2):
        L = np.tril(rb.reduced_factor(B, mu)[0])
        for k in range(1, B.N + 1):
            Lk = np.tril(rb.leading_factor(B, mu, k)[0])
            assert np.abs(Lk - L[:k, :k]).max() <= 1e-13 * np.abs(L).max()
            assert np.array_equal(Lk, np.tril(rb.reduced_factor(B.truncated(k), mu)[0]))
            # and by a third route: the factor reproduces W_k^T A(mu) W_k built from the operator
            Wk = B.W[:, :k]
            AW = np.stack([pb.apply(w.problem, mu, Wk[:, j]) for j in range(k)], axis=1)
            assert np.abs(Lk @ Lk.T - Wk.T @ AW).max() <= 1e-11 * np.abs(Wk.T @ AW).max()


def test_adaptive_n_limits_reduce_to_fixed_bases(small_case):
    """Adaptive N (Section 4.1, end) in its two limits: a ratio test that never holds keeps W_k
    (the same iteration as RBCG on the truncated basis), one that always holds adds a vector
    after every iteration; starting at the full basis leaves nothing to grow (plain RBCG)."""
    w, B = small_case
    for mu in w.test_mu(2):
        ref = rb.rbcg(B, mu, tol=1e-10, beta="pr")
        full = rb.rbcg(B, mu, tol=1e-10, beta="pr", adaptive_n=B.N)
        assert full.iters == ref.iters and np.array_equal(full.x, ref.x)
        assert set(full.n_history) == {B.N}
        for k in (1, 3):
            never = rb.rbcg(B, mu, tol=1e-10, beta="pr", adaptive_n=k, gamma=0.0)
            trunc = rb.rbcg(B.truncated(k), mu, tol=1e-10, beta="pr")
            assert never.iters == trunc.iters and np.array_equal(never.x, trunc.x)
            assert set(never.n_history) == {k}
            always = rb.rbcg(B, mu, tol=1e-10, beta="pr", adaptive_n=k, gamma=np.inf)
            h = always.n_history
            m = min(len(h), B.N - k + 1)
            assert h[:m] == list(range(k, k + m))
            assert all(v == B.N for v in h[m:])
            assert always.converged


def test_adaptive_n_follows_the_ratio_rule_and_reaches_truth(small_case):
    """With gamma = 10 the recorded N grows exactly after the iterations whose residual fell by
    less than gamma, and the iteration still converges to the truth of eq. 1."""
    w, B = small_case
    prob = w.problem
    for mu in w.test_mu(3):
        res = rb.rbcg(B, mu, tol=1e-10, beta="pr", adaptive_n=2, gamma=10.0)
        assert res.converged and res.restarts == 0
        h, n = res.history, res.n_history
        assert n[0] == 2 and len(n) == res.iters     # one application per iteration except the last
        for i in range(1, len(n)):
            grow = h[i - 1] / h[i] < 10.0 and n[i - 1] < B.N
            assert n[i] == n[i - 1] + (1 if grow else 0), (i, h[i - 1] / h[i], n[i - 1], n[i])
        xs = direct.sparse_direct(prob, mu)
        assert np.linalg.norm(res.x - xs) <= 1e-8 * np.linalg.norm(xs)


def test_restart_factor_only_acts_after_a_failed_true_residual_check(small_case):
    """The stopping test of Alg. 3 step 8 is the plain one: with no restart the target factor of
    restarted cycles changes nothing."""
    w, B = small_case
    for mu in w.test_mu(2):
        a = rb.rbcg(B, mu, tol=1e-10, beta="pr")
        b = rb.rbcg(B, mu, tol=1e-10, beta="pr", restart_factor=0.5)
        assert a.restarts == b.restarts == 0
        assert a.iters == b.iters and np.array_equal(a.x, b.x)


def test_stored_oracle_solves_and_the_restart_policy():
    """The stored oracle solves of the 512 x 512 workload: every one converged to a true relative
    residual below 1e-10 under the plain stopping rule of Alg. 3 step 8 (restarted cycles aim at
    tol) and under the library's policy (they aim at tol / 2).  The target of a restarted cycle is
    the only difference between the two, so a solve that never restarted has the same count
    under both, and a restart can only add iterations."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rbcg_2d_512_oracle.json")))
    for sfx in ("", "_nu6"):
        plain, half = g["iters" + sfx], g["iters" + sfx + "_half"]
        rs_plain, rs_half = g["restarts" + sfx], g["restarts" + sfx + "_half"]
        assert len(plain) == len(half) == 16
        for a, b, ra, rb_ in zip(plain, half, rs_plain, rs_half):
            if ra == 0:
                assert rb_ == 0 and a == b
            assert b >= a or rb_ > 0
    assert all(r < 1e-10 for r in g["rel_res"] + g["rel_res_nu6"] + g["rel_res_nu9"]) and all(g["converged"])
    # more sweeps per preconditioner application, fewer iterations (the smoother's error reduction)
    mean = lambda v: sum(v) / len(v)
    assert mean(g["iters"]) > mean(g["iters_nu6"]) > mean(g["iters_nu9"])


def test_multi_fidelity_sample_from_the_coarse_grid():
    """Section 4.2, last paragraph: the parameter sample comes from the greedy on the coarse grid
    and the fine basis holds the fine snapshots of that sample.  With the coarse grid equal to the
    fine one the construction is the plain greedy of Alg. 1."""
    fine = wl.small((24, 20), (2, 2), n_basis=5, n_train=30, bumps=True)
    coarse = wl.small((12, 10), (2, 2), n_basis=5, n_train=30, bumps=True)
    train = fine.train_mu()
    assert np.array_equal(train, coarse.train_mu())
    B = greedy.multi_fidelity(fine.problem, coarse.problem, train, 5)
    Bc = greedy.greedy(coarse.problem, train, 5)
    assert B.selected == Bc.selected
    X = np.stack([direct.sparse_direct(fine.problem, train[j]) for j in B.selected], axis=1)
    assert np.abs(B.W.T @ B.W - np.eye(B.N)).max() < 1e-13
    assert np.linalg.norm(B.W @ B.R - X) <= 1e-11 * np.linalg.norm(X)
    for q in range(fine.problem.P):
        e = np.zeros(fine.problem.n_mu); e[q] = 1.0
        Aq = pins.incidence_operator(fine.problem.dims, fine.problem.blocks, e)
        assert np.abs(B.ANq[q] - B.W.T @ Aq @ B.W).max() <= 1e-12 * np.abs(B.ANq[q]).max()
    same = greedy.multi_fidelity(fine.problem, fine.problem, train, 5)
    plain = greedy.greedy(fine.problem, train, 5)
    assert same.selected == plain.selected
    np.testing.assert_array_equal(same.W, plain.W)
