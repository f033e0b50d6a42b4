"""rb_residual_noalloc: the residual check for callers that cannot allocate device memory.

Such callers run under a framework whose caching allocator already holds the
device's memory, or cannot accept the device-wide synchronisation an allocation
may trigger.  They cannot create a context (that allocates a workspace), so
they check their solutions with this entry point, whose only scratch is a
static device array.  Here it is called twice in a row through the C interface
and must reproduce the true relative residuals that rb_pcg reports for the
same solutions, and the residuals the FP64 oracle computes for the same
vectors (f - A x from its own operator).  Tolerance: 1e-13 absolute on the
relative residual, one
thousandth of the 1e-10 residual bar of the parity tests.  At a converged
solution every entry of f - A x is a cancellation of terms about 1e6 times
larger, so two FP64 evaluations agree to about 1e-15 in these units and no
tighter relative agreement is meaningful.
"""
import numpy as np
import pytest

import ctypes

import workloads as wl
from oracle import greedy
from oracle import problem as pb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_06363_gb300 import rb  # noqa: E402


def _oracle_rel_res(prob, mu, x):
    xs = x.cpu().numpy()
    out = []
    for b in range(len(mu)):
        f = pb.load(prob, mu[b])
        out.append(np.linalg.norm(f - pb.apply(prob, mu[b], xs[b])) / np.linalg.norm(f))
    return np.array(out)


@pytest.mark.parametrize("dims,blocks,precision", [((40, 36), (3, 3), "fp64"), ((14, 12, 10), (2, 2, 2), "mixed")])
def test_noalloc_residual_matches_pcg(dims, blocks, precision):
    w = wl.small(dims, blocks, n_basis=6, n_train=24, bumps=True)
    prob = w.problem
    basis = greedy.greedy(prob, w.train_mu(), w.n_basis)
    mu = w.test_mu(4)
    ctx = rb.Context.from_arrays(prob, basis.W, basis.ANq, basis.fNr, max_batch=4)
    x = torch.zeros((4, prob.n_dof), dtype=torch.float64, device="cuda")
    status, st = ctx.pcg(mu, x, precision=precision)
    assert status == rb.RB_OK
    first = rb.residual_noalloc(prob, mu, x)
    second = rb.residual_noalloc(prob, mu, x)
    np.testing.assert_allclose(first, st["rel_res"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(second, st["rel_res"], rtol=0, atol=1e-13)
    np.testing.assert_array_equal(first, second)
    # the oracle's residual of the same vectors, from its own operator and load
    np.testing.assert_allclose(first, _oracle_rel_res(prob, mu, x), rtol=0, atol=1e-13)
    # a perturbed vector: the scratch keeps nothing from the previous call that matters
    xp = x * (1.0 + 1e-3)
    pert = rb.residual_noalloc(prob, mu, xp)
    assert np.all(pert > 1e-6) and np.all(pert < 1e-2)
    # away from convergence the two agree in relative terms as well: one rb_pcg iteration from
    # the perturbed start, then compare its reported residual with the one of its output vector
    xq = xp.clone()
    _, st_q = ctx.pcg(mu, xq, precision="fp64", x0=True, max_iter=1, max_outer=1)
    assert np.all(st_q["rel_res"] > 1e-8)
    np.testing.assert_allclose(rb.residual_noalloc(prob, mu, xq), st_q["rel_res"], rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(rb.residual_noalloc(prob, mu, xq), _oracle_rel_res(prob, mu, xq), rtol=1e-9,
                               atol=1e-13)
    np.testing.assert_allclose(pert, _oracle_rel_res(prob, mu, xp), rtol=1e-9, atol=1e-13)
    again = rb.residual_noalloc(prob, mu, x)
    np.testing.assert_array_equal(again, first)
    ctx.close()


def test_noalloc_rejects_oversized_batches_and_host_memory():
    prob = wl.rbcg_2d_512().problem
    mu = wl.rbcg_2d_512().test_mu(300)          # 300 queries x 256 tiles of partials > 1 MiB
    x = torch.zeros((1, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbError) as e:
        rb.residual_noalloc(prob, mu, x)
    assert e.value.status == rb.RB_EINVAL and "1 MiB" in str(e.value)
    with pytest.raises(rb.RbError) as e:
        rb.residual_noalloc(prob, mu[:1], np.zeros((1, prob.n_dof)))
    assert e.value.status == rb.RB_EINVAL
    # a Gaussian load with sigma = 0 is rejected before any device work (it would give 0 / 0)
    w = wl.small((16, 12), (2, 2), n_basis=1, bumps=True)
    p, keep = rb.make_problem(w.problem)
    p.loads[1].sigma = 0.0
    mu1 = np.ascontiguousarray(w.test_mu(1))
    xd = torch.zeros((1, w.problem.n_dof), dtype=torch.float64, device="cuda")
    out = np.zeros(1)
    st = rb.lib().rb_residual_noalloc(ctypes.byref(p), 1, mu1.ctypes.data, xd.data_ptr(), out.ctypes.data, None)
    assert st == rb.RB_EINVAL and b"sigma" in rb.lib().rb_last_error(None)
