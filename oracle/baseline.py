"""CPU-baseline timing of the oracle (used only by bench.py's CPU legs).

The oracle is timed as it stands: `rb.rbcg` (Alg. 3) on the host cores, one
process per core (spawn), each single-threaded.  Complete solves give the
CPU baseline and, with the oracle's sparse-direct truth of the same queries,
the error of the GPU's solutions (parity stated per result).  The basis is the oracle's
own: the greedy selection stored by tests/golden/make_golden.py (oracle-only)
is turned back into W by solving those snapshots with the oracle's sparse
direct solver (in parallel, they are independent once selected), modified
Gram-Schmidt twice and eq. 12c.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _init(env_root):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    if env_root not in sys.path:
        sys.path.insert(0, env_root)


def _snapshot(args):
    name, mu = args
    import workloads as wl
    from oracle import direct
    w = wl.WORKLOADS[name]()
    return direct.sparse_direct(w.problem, mu)


def _basis(name, paths):
    import workloads as wl
    from oracle import rb
    w = wl.WORKLOADS[name]()
    W = np.load(paths["W"], mmap_mode="r")
    return rb.Basis(w.problem, np.asarray(W), np.load(paths["ANq"]), np.load(paths["fNr"]))


def _iterate(args):
    name, paths, mu, max_iter, nu = args
    from oracle import rb
    basis = _basis(name, paths)
    t0 = time.perf_counter()
    res = rb.rbcg(basis, mu, tol=1e-10, beta="pr", nu=nu, max_iter=max_iter)
    return res.iters, time.perf_counter() - t0


def _solve(args):
    """One complete Alg. 3 solve (timed); returns (iterations, seconds, restarts, rel_res, x)."""
    name, paths, mu, nu = args
    from oracle import rb
    basis = _basis(name, paths)
    t0 = time.perf_counter()
    res = rb.rbcg(basis, mu, tol=1e-10, beta="pr", nu=nu)
    return res.iters, time.perf_counter() - t0, res.restarts, res.rel_res, res.x


def _errors(args):
    """Relative L2 errors against the sparse-direct truth of eq. 1 and the oracle's relative
    residual of each given vector: [(err, rel_res) for each vector]."""
    name, mu, vectors = args
    import workloads as wl
    from oracle import direct
    from oracle import problem as pb
    prob = wl.WORKLOADS[name]().problem
    truth = direct.sparse_direct(prob, mu)
    f = pb.load(prob, mu)
    tn, fn = np.linalg.norm(truth), np.linalg.norm(f)
    return [(float(np.linalg.norm(v - truth) / tn), float(np.linalg.norm(f - pb.apply(prob, mu, v)) / fn))
            for v in vectors]


def pool(processes: int):
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    return mp.get_context("spawn").Pool(processes, initializer=_init, initargs=(ROOT,))


def basis_from_selection(name: str, selected, p) -> "object":
    """The oracle basis of workload `name` for a stored greedy selection."""
    import workloads as wl
    from oracle import greedy, rb
    w = wl.WORKLOADS[name]()
    train = w.train_mu()
    snaps = p.map(_snapshot, [(name, train[i]) for i in selected])
    W = np.zeros((w.problem.n_dof, 0))
    for x in snaps:
        v, _, nrm = greedy.mgs_twice(W, x)
        W = np.concatenate([W, (v / nrm)[:, None]], axis=1)
    ANq, fNr = rb.affine_blocks(w.problem, W)
    return rb.Basis(w.problem, W, ANq, fNr, None, list(selected))


class OracleRunner:
    """Holds the oracle basis on disk and a spawn pool; times bounded RBCG samples."""

    def __init__(self, name: str, selected, processes: int):
        self.name = name
        self.processes = processes
        self.pool = pool(processes)
        t0 = time.perf_counter()
        basis = basis_from_selection(name, selected, self.pool)
        self.setup_s = time.perf_counter() - t0
        self.tmp = tempfile.TemporaryDirectory()
        self.paths = {}
        for k, a in (("W", basis.W), ("ANq", basis.ANq), ("fNr", basis.fNr)):
            self.paths[k] = os.path.join(self.tmp.name, k + ".npy")
            np.save(self.paths[k], a)

    def sample(self, mus, max_iter: int, nu: int = 1):
        """Run Alg. 3 on each mu (one per process) for at most max_iter iterations.

        Returns (total iterations, wall seconds)."""
        t0 = time.perf_counter()
        out = self.pool.map(_iterate, [(self.name, self.paths, mu, max_iter, nu) for mu in mus])
        wall = time.perf_counter() - t0
        return sum(o[0] for o in out), wall

    def solve(self, mus, nu: int):
        """Complete Alg. 3 solves of every mu (one per process).

        Returns (wall seconds, [(iterations, seconds, restarts, rel_res, x)])."""
        t0 = time.perf_counter()
        out = self.pool.map(_solve, [(self.name, self.paths, mu, nu) for mu in mus])
        return time.perf_counter() - t0, out

    def errors(self, mus, vectors):
        """Per query, [(relative error vs the truth, oracle relative residual)] of each of its vectors."""
        return self.pool.map(_errors, [(self.name, mu, vs) for mu, vs in zip(mus, vectors)])

    def close(self):
        self.pool.close()
        self.pool.join()
        self.tmp.cleanup()
