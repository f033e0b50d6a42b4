"""Write tests/golden/rbcg_2d_512_oracle.json from the FP64 oracle alone.

Contents, for the 512 x 512, 3 x 3-block, two-bump workload with n = 40:
  * `selected`: the training indices chosen by the oracle's greedy (Alg. 1,
    sparse-direct snapshots, snapshot-basis L1 score);
  * `iters`, `rel_res`, `restarts`: the oracle's Alg. 3 (PR beta, one
    red-black Gauss-Seidel sweep, tol 1e-10, the plain stopping rule: no
    restart aims below tol) for the first 16 test parameters, solved with the
    basis rebuilt from `selected`;
  * `iters_nu6`, `restarts_nu6`: the same with six red-black sweeps per
    preconditioner application (the sweep count the GPU benchmark's
    autotuner picks on this workload);
  * `*_half`: the same solves when a restarted cycle aims at half the
    tolerance (restart_factor 0.5), the CUDA library's FP64 restart policy,
    for comparing its iteration counts.
  * `iters_nu9`, `rel_res_nu9`, `restarts_nu9`: the plain-rule solves with nine sweeps (the
    autotuner's choice once the smoother runs three sweeps per pass), added to an existing file by
    `--add-nu 9` with the basis rebuilt from `selected` (the reference arm of bench.py scales its
    iteration rate by these counts).
It calls only `oracle/` and `workloads`.  Run: python tests/golden/make_golden.py [--add-nu NU]
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
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def _solve(args):
    import workloads as wl
    from oracle import rb
    W, ANq, fNr, mu, beta, nu, rf = args
    w = wl.rbcg_2d_512()
    basis = rb.Basis(w.problem, W, ANq, fNr)
    res = rb.rbcg(basis, mu, tol=1e-10, beta=beta, nu=nu, restart_factor=rf)
    return res.iters, res.rel_res, res.converged, res.restarts


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
        runs = {}
        for nu in (1, 6):
            for rf in (1.0, 0.5):
                runs[nu, rf] = pool.map(_solve, [(basis.W, basis.ANq, basis.fNr, mu[i], "pr", nu, rf)
                                                 for i in range(N_TEST)])
        res, res6 = runs[1, 1.0], runs[6, 1.0]
    out = {
        "workload": w.name,
        "source": "oracle greedy (Alg. 1) and oracle RBCG (Alg. 3, PR beta, rbgs nu=1 and nu=6, tol 1e-10, plain stopping rule)",
        "selected": [int(s) for s in basis.selected],
        "test_indices": list(range(N_TEST)),
        "iters": [int(r[0]) for r in res],
        "rel_res": [float(r[1]) for r in res],
        "converged": [bool(r[2]) for r in res],
        "restarts": [int(r[3]) for r in res],
        "iters_nu6": [int(r[0]) for r in res6],
        "rel_res_nu6": [float(r[1]) for r in res6],
        "restarts_nu6": [int(r[3]) for r in res6],
        "iters_half": [int(r[0]) for r in runs[1, 0.5]],
        "restarts_half": [int(r[3]) for r in runs[1, 0.5]],
        "iters_nu6_half": [int(r[0]) for r in runs[6, 0.5]],
        "restarts_nu6_half": [int(r[3]) for r in runs[6, 0.5]],
        "greedy_seconds": round(t_greedy, 1),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


def add_nu(nu: int):
    """Add the plain-rule solves with `nu` sweeps to the stored file (basis from its selection)."""
    _worker_init()
    import workloads as wl
    from oracle import baseline
    with open(OUT) as f:
        out = json.load(f)
    w = wl.rbcg_2d_512()
    assert out["workload"] == w.name
    mu = w.test_mu(N_TEST)
    pool = baseline.pool(min(N_TEST, os.cpu_count() or 1))
    basis = baseline.basis_from_selection("rbcg_2d_512", out["selected"], pool)
    res = pool.map(_solve, [(basis.W, basis.ANq, basis.fNr, mu[i], "pr", nu, 1.0) for i in range(N_TEST)])
    pool.close()
    out[f"iters_nu{nu}"] = [int(r[0]) for r in res]
    out[f"rel_res_nu{nu}"] = [float(r[1]) for r in res]
    out[f"restarts_nu{nu}"] = [int(r[3]) for r in res]
    out["source"] += f"; nu={nu} added from the stored selection"
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in (f"iters_nu{nu}", f"restarts_nu{nu}")}))


if __name__ == "__main__":
    if len(sys.argv) == 3 and sys.argv[1] == "--add-nu":
        add_nu(int(sys.argv[2]))
    else:
        main()
