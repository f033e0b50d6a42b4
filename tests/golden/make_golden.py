"""Write tests/golden/rbcg_2d_512_oracle.json from the FP64 oracle alone.

Contents, for the 512 x 512, 3 x 3-block, two-bump workload with n = 40:
  * `selected`: the training indices chosen by the oracle's greedy (Alg. 1,
    sparse-direct snapshots, snapshot-basis L1 score);
  * `iters`: the oracle's Alg. 3 iteration counts (PR beta, one red-black
    Gauss-Seidel sweep, tol 1e-10) for the first 16 test parameters, solved
    with the basis rebuilt from `selected`.
It calls only `oracle/` and `workloads`.  Run: python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "rbcg_2d_512_oracle.json")
N_TEST = 16


def _worker_init():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _solve(args):
    import workloads as wl
    from oracle import rb
    W, ANq, fNr, mu, beta = args
    w = wl.rbcg_2d_512()
    basis = rb.Basis(w.problem, W, ANq, fNr)
    res = rb.rbcg(basis, mu, tol=1e-10, beta=beta)
    return res.iters, res.rel_res, res.converged


def main():
    _worker_init()
    import numpy as np
    import workloads as wl
    from oracle import greedy
    w = wl.rbcg_2d_512()
    t0 = time.time()
    basis = greedy.greedy(w.problem, w.train_mu(), w.n_basis)
    t_greedy = time.time() - t0
    mu = w.test_mu(N_TEST)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(N_TEST, os.cpu_count() or 1), initializer=_worker_init) as pool:
        res = pool.map(_solve, [(basis.W, basis.ANq, basis.fNr, mu[i], "pr") for i in range(N_TEST)])
    out = {
        "workload": w.name,
        "source": "oracle greedy (Alg. 1) and oracle RBCG (Alg. 3, PR beta, rbgs nu=1, tol 1e-10)",
        "selected": [int(s) for s in basis.selected],
        "test_indices": list(range(N_TEST)),
        "iters": [int(r[0]) for r in res],
        "rel_res": [float(r[1]) for r in res],
        "converged": [bool(r[2]) for r in res],
        "greedy_seconds": round(t_greedy, 1),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
