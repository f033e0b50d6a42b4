"""GPU parity of the learned warm start and of the starting vectors.

* the network kernels (standardisation, forward pass, back-propagation, Adam)
  against the FP64 oracle of oracle/mlp.py on the same BF16-rounded weights;
* rb_warm_start without a network against the oracle's Galerkin approximation
  (eqs. 2-3), rb_coefficients against W^T x;
* a trained network's start against the cold start of RBCG (Alg. 3): every
  start reaches the same solution (relative L2 1e-9 of the oracle's truth at
  relative residual 1e-10), and the test reports what the network gains.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import direct, greedy, mlp
from oracle import rb as orb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_06363_gb300 import rb  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _net_case(n_in, P, hidden, n_out, S, seed):
    """Initial parameters (Glorot weights, small random biases), parameter vectors of a
    workload-like distribution and random targets with offsets and unequal scales."""
    sizes = (n_in, hidden, hidden, n_out)
    rng = np.random.default_rng(seed)
    layers = [(W, 0.1 * rng.standard_normal(W.shape[0])) for W, _ in wl.mlp_init(sizes, seed)]
    u = wl.uniform01(100 + seed, S * n_in).reshape(S, n_in)
    mu = u.copy()
    mu[:, :P] = np.exp(np.log(0.1) + u[:, :P] * np.log(100.0))
    Y = rng.standard_normal((S, n_out)) * rng.uniform(0.1, 3.0, n_out) + rng.uniform(-2, 2, n_out)
    return sizes, layers, mu, Y


@pytest.mark.parametrize("n_in,P,hidden,n_out,S", [(11, 9, 128, 40, 100), (3, 2, 48, 7, 37), (8, 8, 128, 60, 64)])
def test_gradient_and_standardisation_match_oracle(n_in, P, hidden, n_out, S):
    sizes, layers, mu, Y = _net_case(n_in, P, hidden, n_out, S, seed=7)
    net = rb.Mlp(n_in, P, hidden, n_out, rb.flatten_params(layers), max_samples=S)
    loss, g = net.gradient(mu, Y)
    _, scale, t = net.get()
    assert t == 0
    onet = mlp.from_init(layers, mlp.features(mu, P), Y)
    np.testing.assert_allclose(scale, np.concatenate([onet.in_mean, onet.in_scale, onet.out_mean, onet.out_scale]),
                               rtol=1e-12, atol=1e-14)
    X = (mlp.features(mu, P) - onet.in_mean) / onet.in_scale
    Ts = (Y - onet.out_mean) / onet.out_scale
    oloss, gW, gb = mlp.loss_and_grads(onet, X, Ts, rounding=True)
    assert abs(loss - oloss) <= 1e-5 * oloss, (loss, oloss)
    got = rb.unflatten_params(g, sizes)
    for l in range(3):
        assert _rel(got[l][0], gW[l]) < 1e-4, ("W", l, _rel(got[l][0], gW[l]))
        assert _rel(got[l][1], gb[l]) < 1e-4, ("b", l, _rel(got[l][1], gb[l]))
    net.close()


def test_adam_training_and_inference_match_oracle():
    n_in, P, hidden, n_out, S = 11, 9, 128, 40, 200
    sizes, layers, mu, Y = _net_case(n_in, P, hidden, n_out, S, seed=11)
    net = rb.Mlp(n_in, P, hidden, n_out, rb.flatten_params(layers), max_samples=S)
    steps = 40                         # two replays of the captured 16-step graph and 8 direct steps
    hist = net.fit(mu, Y, steps, lr=3e-3)
    onet = mlp.from_init(layers, mlp.features(mu, P), Y)
    ohist = mlp.train(onet, mlp.features(mu, P), Y, steps, lr=3e-3)
    np.testing.assert_allclose(hist, ohist, rtol=2e-3)
    assert hist[-1] < 0.8 * hist[0]     # random targets: the loss falls, slowly
    # inference on new parameters with the trained masters: the oracle rounds the
    # same FP32 masters to the same BF16 weights
    flat, scale, t = net.get()
    assert t == steps
    trained = rb.unflatten_params(flat, sizes)
    onet2 = mlp.Net([W for W, _ in trained], [b for _, b in trained], scale[:n_in], scale[n_in:2 * n_in],
                    scale[2 * n_in:2 * n_in + n_out], scale[2 * n_in + n_out:])
    _, _, mu_new, _ = _net_case(n_in, P, hidden, n_out, 77, seed=12)
    pred = net.predict(mu_new)
    ref = mlp.predict(onet2, mu_new, P)
    assert np.max(np.abs(pred - ref) / onet2.out_scale) < 2e-5
    # device output buffer, same values
    out = torch.zeros((77, n_out), dtype=torch.float64, device="cuda")
    net.predict(mu_new, out=out)
    np.testing.assert_allclose(out.cpu().numpy(), pred, rtol=0, atol=0)
    net.close()


@pytest.fixture(scope="module")
def case2d():
    w = wl.small((40, 36), (3, 3), n_basis=8, n_train=40, bumps=True)
    basis = greedy.greedy(w.problem, w.train_mu(), w.n_basis)
    ctx = rb.Context.from_arrays(w.problem, basis.W, basis.ANq, basis.fNr, max_batch=5)
    yield w, basis, ctx
    ctx.close()


def test_galerkin_start_matches_oracle(case2d):
    w, basis, ctx = case2d
    mu = w.test_mu(7)                                  # two chunks of the 5-query workspace
    ref_c = np.stack([orb.rb_coefficients(basis, m) for m in mu])
    for on_device in (False, True):
        if on_device:
            x = torch.zeros((7, w.problem.n_dof), dtype=torch.float64, device="cuda")
            c = torch.zeros((7, basis.N), dtype=torch.float64, device="cuda")
        else:
            x, c = np.zeros((7, w.problem.n_dof)), np.zeros((7, basis.N))
        assert ctx.warm_start(mu, x, coef=c) == rb.RB_OK
        xs = x.cpu().numpy() if on_device else x
        cs = c.cpu().numpy() if on_device else c
        for b in range(7):
            assert _rel(cs[b], ref_c[b]) < 1e-11
            assert _rel(xs[b], basis.W @ ref_c[b]) < 1e-6       # FP32 lift
    bad = mu[:1].copy()
    bad[0, 0] = -1.0                                     # A(mu) would not be SPD: rejected before any launch
    with pytest.raises(rb.RbError):
        ctx.warm_start(bad, np.zeros((1, w.problem.n_dof)))


def test_coefficients_match_projection(case2d):
    w, basis, ctx = case2d
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, w.problem.n_dof))
    c = ctx.coefficients(x)
    cd = ctx.coefficients(torch.as_tensor(x, device="cuda"))
    ref = x @ basis.W
    for b in range(6):
        assert _rel(c[b], ref[b]) < 1e-6
    np.testing.assert_array_equal(c, cd)


def test_learned_warm_start_reaches_truth_and_reports_gain():
    """3D 24^3, P = 8, n = 12: network trained on 512 truth solves, 48 test queries."""
    w = wl.small((24, 24, 24), (2, 2, 2), n_basis=12, n_train=96)
    prob = w.problem
    S, T = 512, 48
    ctx = rb.Context.build(prob, w.n_basis, w.train_mu(), max_batch=S)
    n = ctx.n
    mu_tr = wl.mlp_train_mu(w, S)
    x_tr = torch.zeros((S, prob.n_dof), dtype=torch.float64, device="cuda")
    status, st = ctx.pcg(mu_tr, x_tr, precision="mixed")
    assert status == rb.RB_OK
    Y = ctx.coefficients(x_tr)
    sizes = wl.mlp_layer_sizes(prob.n_mu, n)
    net = rb.Mlp(prob.n_mu, prob.P, sizes[1], n, rb.flatten_params(wl.mlp_init(sizes)), max_samples=S)
    hist = net.fit(mu_tr, Y, 1500, lr=3e-3)
    assert hist[-1] < 0.02 * hist[0], (hist[0], hist[-1])

    mu = w.test_mu(T)
    truth = np.stack([direct.sparse_direct(prob, m) for m in mu[:4]])
    runs = {}
    for name in ("cold", "galerkin", "learned"):
        x = torch.zeros((T, prob.n_dof), dtype=torch.float64, device="cuda")
        if name != "cold":
            ctx.warm_start(mu, x, net=net if name == "learned" else None)
        x0 = x.cpu().numpy()
        status, st = ctx.pcg(mu, x, precision="mixed", x0=name != "cold")
        assert status == rb.RB_OK and np.all(st["rel_res"] < 1e-10), name
        xs = x.cpu().numpy()
        for b in range(4):
            assert _rel(xs[b], truth[b]) < 1e-9, (name, b)
        runs[name] = (x0, xs, st)
    ref = runs["cold"][1]
    err0 = {k: float(np.mean([_rel(v[0][b], ref[b]) for b in range(T)])) for k, v in runs.items()}
    its = {k: float(v[2]["iters"].mean()) for k, v in runs.items()}
    print("\nwarm start, 24^3 P=8 n=%d: mean initial error %s; mean inner iterations %s" % (n, err0, its))
    assert err0["cold"] == 1.0
    # Bars from what fixes them.  Any start in span(W) is at least as far from the solution as the
    # orthogonal projection W W^T x (mean 0.2-0.3 here: n = 12 vectors for 8 block parameters); the
    # Galerkin start is the oracle's RB approximation of eq. 3 computed with the same basis; the
    # network's start lies within the projection error plus its fitting error.
    W, ANq, fNr, _, _ = ctx.basis()
    obasis = orb.Basis(prob, W, ANq, fNr)
    proj = np.array([_rel(W @ (W.T @ ref[b]), ref[b]) for b in range(T)])
    gal = np.array([_rel(runs["galerkin"][0][b], ref[b]) for b in range(T)])
    learned = np.array([_rel(runs["learned"][0][b], ref[b]) for b in range(T)])
    ogal = np.array([_rel(orb.rb_approximation(obasis, mu[b]), ref[b]) for b in range(T)])
    assert np.all(np.abs(gal - ogal) < 1e-5)                        # FP32 lift of the same x_hat
    assert np.all(gal >= proj - 1e-5) and np.all(learned >= proj - 1e-5)
    assert err0["learned"] < 0.5 and err0["galerkin"] < 0.6
    # any start in span(W) reaches the Galerkin point with the first RB correction (Section 3.1),
    # so the Galerkin start and the cold start take about the same number of iterations
    assert abs(its["galerkin"] - its["cold"]) <= 2.0
    assert its["learned"] <= its["cold"] + 1.0
    net.close()
    ctx.close()


def test_error_basis_matches_oracle():
    """rb_error_basis (method of snapshots on the device) against the oracle's POD: the same
    singular values, the same targets Z = V^T E up to the sign of each mode; rb_error_coefficients
    reproduces Z; with as many modes as snapshots x_hat + V z_s is the training solution itself."""
    from oracle import errbasis
    w = wl.small((40, 36), (3, 3), n_basis=6, n_train=30, bumps=True)
    prob = w.problem
    basis = greedy.greedy(prob, w.train_mu(), w.n_basis)
    S = 24
    mus = wl.mlp_train_mu(w, S)
    X = np.stack([direct.sparse_direct(prob, m) for m in mus])
    ctx = rb.Context.from_arrays(prob, basis.W, basis.ANq, basis.fNr, max_batch=S)
    m = 5
    Zg, sg = ctx.error_basis(mus, X, m)
    Vo, Zo, so = errbasis.error_basis(basis, mus, X, m)
    np.testing.assert_allclose(sg, so, rtol=1e-8)
    signs = np.sign(np.sum(Zg.T * Zo, axis=1))
    np.testing.assert_allclose(Zg * signs[None, :], Zo.T, rtol=0, atol=1e-7 * np.abs(Zo).max())
    Xd = torch.as_tensor(X, device="cuda")
    Zc = ctx.error_coefficients(mus, Xd, m)
    np.testing.assert_allclose(Zc, Zg, rtol=0, atol=1e-5 * np.abs(Zg).max())
    # the start from given coefficients equals the oracle's x_hat + V z
    x0 = np.zeros((S, prob.n_dof))
    ctx.warm_start_error(mus, x0, z=Zg)
    for s in (0, 7, 23):
        ref = errbasis.warm_start(basis, Vo * signs[None, :], mus[s], Zg[s])
        assert _rel(x0[s], ref) < 1e-6, s
    # full rank: the training solutions come back
    Zf, _ = ctx.error_basis(mus, Xd, S)
    xf = torch.zeros((S, prob.n_dof), dtype=torch.float64, device="cuda")
    ctx.warm_start_error(mus, xf, z=Zf)
    for s in range(S):
        assert _rel(xf[s].cpu().numpy(), X[s]) < 1e-6, s
    ctx.close()


def test_error_basis_warm_start_reaches_truth_and_reports_gain():
    """3D 24^3, P = 8, n = 12: an error basis of 128 truth solves (m = 16) and a network for its
    coefficients trained on 512 pairs; the start x_hat + V z(mu) leaves span(W).  Every start reaches
    the truth; the test reports the initial error and the iterations of each start."""
    w = wl.small((24, 24, 24), (2, 2, 2), n_basis=12, n_train=96)
    prob = w.problem
    S, T, m, Sp = 512, 48, 16, 128
    ctx = rb.Context.build(prob, w.n_basis, w.train_mu(), max_batch=S)
    mu_tr = wl.mlp_train_mu(w, S)
    x_tr = torch.zeros((S, prob.n_dof), dtype=torch.float64, device="cuda")
    status, _ = ctx.pcg(mu_tr, x_tr, precision="mixed")
    assert status == rb.RB_OK
    Z0, sig = ctx.error_basis(mu_tr[:Sp], x_tr[:Sp], m)
    assert sig[0] > 0 and np.all(np.diff(sig) <= 1e-12 * sig[0])
    Z = ctx.error_coefficients(mu_tr, x_tr, m)
    np.testing.assert_allclose(Z[:Sp], Z0, rtol=0, atol=1e-5 * np.abs(Z0).max())
    sizes = wl.mlp_layer_sizes(prob.n_mu, m)
    net = rb.Mlp(prob.n_mu, prob.P, sizes[1], m, rb.flatten_params(wl.mlp_init(sizes)), max_samples=S)
    hist = net.fit(mu_tr, Z, 1500, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0], (hist[0], hist[-1])
    mu = w.test_mu(T)
    truth = np.stack([direct.sparse_direct(prob, mm) for mm in mu[:4]])
    runs = {}
    for name in ("cold", "galerkin", "error_basis"):
        x = torch.zeros((T, prob.n_dof), dtype=torch.float64, device="cuda")
        if name == "galerkin":
            ctx.warm_start(mu, x)
        elif name == "error_basis":
            ctx.warm_start_error(mu, x, net=net)
        x0 = x.cpu().numpy()
        status, st = ctx.pcg(mu, x, precision="mixed", x0=name != "cold")
        assert status == rb.RB_OK and np.all(st["rel_res"] < 1e-10), name
        xs = x.cpu().numpy()
        for b in range(4):
            assert _rel(xs[b], truth[b]) < 1e-9, (name, b)
        runs[name] = (x0, xs, st)
    ref = runs["cold"][1]
    err0 = {k: float(np.mean([_rel(v[0][b], ref[b]) for b in range(T)])) for k, v in runs.items()}
    its = {k: float(v[2]["iters"].mean()) for k, v in runs.items()}
    print("\nerror-basis warm start, 24^3 P=8 n=12 m=16: mean initial error %s; mean inner iterations %s"
          % (err0, its))
    # the error basis removes most of the Galerkin error
    assert err0["error_basis"] < 0.5 * err0["galerkin"]
    net.close()
    ctx.close()
