"""The failure path of the bounded device waits, exercised without faulting the GPU.

Every kernel that waits on an asynchronous copy bounds the wait; on expiry it
raises a device error flag, keeps its barriers matched, lets its copies land
and returns, and the solve returns RB_ETIMEOUT.  rb_debug_wait shortens the
limit to 5 ms and makes the first CTA of the staged CG kernel leave one stage
unissued: nothing is in flight for that stage, so the wait simply runs out.
The same context then solves normally.
"""
import time

import numpy as np
import pytest

import workloads as wl
from oracle import direct, greedy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_06363_gb300 import rb  # noqa: E402


def test_expired_wait_returns_timeout_and_the_context_recovers():
    w = wl.small((128, 40), (2, 2), n_basis=4, n_train=12)
    prob = w.problem
    basis = greedy.greedy(prob, w.train_mu(), w.n_basis)
    mu = w.test_mu(2)
    ctx = rb.Context.from_arrays(prob, basis.W, basis.ANq, basis.fNr, max_batch=2)
    x = torch.zeros((2, prob.n_dof), dtype=torch.float64, device="cuda")
    status, _ = ctx.pcg(mu, x, precision="fp64")          # warm-up: modules loaded, graph path exercised
    assert status == rb.RB_OK
    ctx.debug_wait(0.005, 3)
    x.zero_()
    t0 = time.perf_counter()
    with pytest.raises(rb.RbError) as e:
        ctx.pcg(mu, x, precision="fp64")
    elapsed = time.perf_counter() - t0
    assert e.value.status == rb.RB_ETIMEOUT
    assert "timeout" in str(e.value)
    assert elapsed < 1.5, elapsed                          # the 5 ms limit ran out, not the default 2 s
    ctx.debug_wait(2.0, -1)
    x.zero_()
    status, st = ctx.pcg(mu, x, precision="fp64")
    assert status == rb.RB_OK
    for b in range(2):
        truth = direct.sparse_direct(prob, mu[b])
        assert np.linalg.norm(x[b].cpu().numpy() - truth) / np.linalg.norm(truth) < 1e-9
    with pytest.raises(rb.RbError):
        ctx.debug_wait(0.0, -1)
    ctx.close()
