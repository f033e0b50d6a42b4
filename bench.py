#!/usr/bin/env python
"""Benchmark: RB-preconditioned CG (Alg. 3) solves per second on one or more GB300s.

One step = one batch of test queries solved to true relative residual 1e-10
(the whole online hot path: reduced set-up, FP64 residual refinement, FP32
inner RBCG with RBI preconditioner, tensor-core projections), inputs resident
in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

After the timed region the default run also compares three starts of the same
solves on rank 0 (cold, Galerkin, learned network; "warm_start" in the JSON).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RB-PCG solves/sec to rel. residual 1e-10 (mixed+batched vs FP64 plain), % HBM roofline"
GOLDEN = os.path.join(ROOT, "tests", "golden", "rbcg_2d_512_oracle.json")
TUNE_SAMPLE = 256          # parameters the autotuner times (own seeded stream: not training, not test)
PARITY_SEED = 7

# Algorithmic bytes per grid point per launch unit (one query, one application), by kernel and
# inner precision: every operand read or written once (eqs. 5-8 and the steps of Alg. 3).  The
# smoother's unit is one preconditioner application, whatever the sweep count: it reads its
# source y and r, reads the direction p for the Polak-Ribiere term and writes y.
BYTES_PER_POINT = {
    "f32": {"cg_a": 12, "cg_b": 20, "smooth": 16, "project": 4, "tc_project": 4, "prolong": 4, "tc_prolong": 4,
            "outer_residual": 12, "outer_update": 24},
    "f64": {"cg_a": 24, "cg_b": 40, "smooth": 32, "project": 8, "prolong": 8, "outer_residual": 16},
}
# Bytes per point of one streaming pass over memory before the last (source, r, output): the
# smoother moves this much more per extra pass.  kernels 0 and 2 make one pass per sweep, 1 one
# pass for all sweeps, 3 and 4 one pass per three and per two sweeps.
SWEEP_PASS_BYTES = {"f32": 12, "f64": 24}


def outer_flops(dim, n_loads):
    """FP64 operations per point of the outer residual f - A x with its two squared norms: the load
    sum (one FMA per term), the 5- or 7-point stencil (one FMA per coefficient), the difference and
    two FMAs for the squares."""
    return 2 * n_loads + 2 * (2 * dim + 1) + 1 + 4


def smoother_passes(kernels, nu):
    """Passes over memory of one 2D smoother application."""
    if kernels == 1:
        return 1
    if kernels in (3, 4):
        nf = 3 if kernels == 3 else 2
        return (nu + nf - 1) // nf
    return nu
# With BF16 storage of the preconditioner's intermediate vectors: the prolongation writes 2 B;
# a pass before the last reads source (2) and r (4) and writes 2; the last reads source (2), r (4),
# p (4) and writes y (4).
BF16_SMOOTH_LAST, BF16_SMOOTH_SWEEP, BF16_PROLONG = 14, 8, 2

# DRAM bytes per point and query of the dominant kernel from an ncu capture, valid only while the
# kernel's source files hash to what they were when the counters were taken (otherwise the line
# reports traffic null).  Key: (inner precision, storage, kernel family, kernel, nu).  Filled from a
# capture of the current kernels.
NCU_TRAFFIC = {
    ("f32", "f32", 3, "smooth", 9): {
        "bytes_per_point": 37.56, "sources": ["rb_smooth_multi.cu", "rb_stage.cuh", "rb_common.cuh"],
        "sha": "4d6d87647bc00ade",
        "capture": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one application (two passes of "
                   "k2_smooth_multi<3, 0, 512> and one of <3, 1, 512>), 512x512, 64 queries, nu = 9"},
}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rbcg_2d_512")
    ap.add_argument("--batch", type=int, default=0, help="queries per step and GPU (default: the workload's)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--nu", type=int, default=1)
    ap.add_argument("--gemm", default="auto")
    ap.add_argument("--kernels", type=int, default=0, help="stencil kernel family (rb_opts.kernels)")
    ap.add_argument("--fp64-queries", type=int, default=0,
                    help="queries of the FP64 plain comparator (default: the timed batch; -1: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-nu", type=int, default=9,
                    help="reference arm: smoother sweeps of the oracle (the GPU arm's tuned value on the default "
                         "workload; stored oracle counts exist for 1, 6 and 9); the GPU arm's own CPU baseline "
                         "uses its tuned value")
    ap.add_argument("--cpu-iters", type=int, default=60,
                    help="reference arm: Alg. 3 iterations per core and step (about 10 s of oracle work)")
    ap.add_argument("--basis", default="", help="basis file: loaded if it exists, else built and saved there")
    ap.add_argument("--mf-coarse", type=int, default=0,
                    help="build the basis by the multi-fidelity greedy: sample selected on this many nodes per "
                         "direction, snapshots on the workload's grid (0: plain greedy on the workload's grid)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (use --nu, --gemm as given)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only (no per-kernel pass, e2e, FP64 comparator or CPU baseline); for profilers")
    ap.add_argument("--warm", action="store_true",
                    help="run the learned warm-start comparison (cold / Galerkin / network start) also with --quick")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start comparison")
    ap.add_argument("--warm-pairs", type=int, default=4096, help="training pairs (truth solves) of the network")
    ap.add_argument("--warm-steps", type=int, default=2000, help="Adam steps of the network")
    ap.add_argument("--warm-test", type=int, default=0, help="test queries of the comparison (default: the step's)")
    ap.add_argument("--warm-modes", type=int, default=24, help="modes of the error basis of the warm start")
    ap.add_argument("--no-leg3d", action="store_true",
                    help="skip the 3D leg (128^3, 256 queries per step, timed after the 2D results)")
    ap.add_argument("--leg3d-steps", type=int, default=2)
    ap.add_argument("--n-sweep", default="",
                    help="comma-separated basis sizes: steps of RBI and RBCG versus N on the workload's test "
                         "parameters (the paper's steps-versus-RB-dimension study) instead of the timed bench")
    ap.add_argument("--rank-check", action="store_true",
                    help="CPU only: start the ranks, shard the queries and agree on the max time over gloo")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def launch_ranks(n: int, argv) -> int:
    """Run this script as n ranks (one process per GPU) under torch.distributed.run on 127.0.0.1
    and return the exit code of the launcher.  Used when --gpus N > 1 is given outside a launcher."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]
    return subprocess.run(cmd).returncode


def rank_check(args):
    """--rank-check: the multi-rank path without a GPU (gloo): each rank takes its shard of the
    timed batch, the step time is the max over ranks, rank 0 prints one JSON line."""
    import torch.distributed as dist

    import workloads as wl
    from paper_1804_06363_gb300.shard import max_over_ranks, shard_range
    rank, world, _ = dist_env()
    if world > 1:
        dist.init_process_group("gloo")
    w = wl.WORKLOADS[args.workload]()
    B = args.batch or w.batch
    lo, hi = shard_range(B * world, rank, world)
    t = max_over_ranks(1.0 + rank, dist, "cpu")
    shards = [None] * world
    if world > 1:
        dist.all_gather_object(shards, (rank, lo, hi))
    else:
        shards = [(0, lo, hi)]
    if rank == 0:
        print(json.dumps({"rank_check": True, "n_ranks": world, "queries": B * world, "shards": shards,
                          "t_max": t}))
    if world > 1:
        dist.destroy_process_group()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q, "--format=csv",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [ln.strip() for ln in open(self.f.name) if ln.strip() and not ln.startswith("index")]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            c = [t.strip() for t in r.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1].split()[0]))
                smax.append(float(c[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


def load_golden():
    if os.path.exists(GOLDEN):
        return json.load(open(GOLDEN))
    return None


def base_options(precision: str, stream) -> dict:
    """Options of the timed solves before tuning: PR beta, red-black GS."""
    return dict(precision=precision, beta="pr", nu=1, gemm="auto", kernels=0, stream=stream)


def tune(ctx, w, x, opts, n_sample: int = TUNE_SAMPLE):
    """The autotuner on n_sample parameters of its own seeded stream (neither the greedy's training
    set nor the timed test queries); updates opts with its choice and returns the summary."""
    import workloads as wl
    tB = min(x.shape[0], n_sample)
    tuned = ctx.autotune(wl.tune_mu(w, tB), x[:tB], **opts)
    opts.update(nu=tuned["nu"], inner_tol=tuned["inner_tol"], gemm=tuned["gemm"], kernels=tuned["kernels"],
                store=tuned["store"], x0=tuned["x0"])
    tuned["sample"] = f"{tB} tuning parameters (seeded stream {wl.TUNE_SEED})"
    return tuned


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: implementer and part codes)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    fields = {}
    for line in info:
        if ":" in line:
            k, v = (t.strip() for t in line.split(":", 1))
            fields.setdefault(k, v)
    if "model name" in fields:
        return fields["model name"]
    parts = [f"{k} {fields[k]}" for k in ("CPU implementer", "CPU part") if k in fields]
    return " ".join([platform.machine()] + parts) if parts else platform.machine()


def parity_sample(B: int, k: int):
    """Seeded sample of k query indices of a batch of B (sorted)."""
    import numpy as np
    return sorted(int(i) for i in np.random.default_rng(PARITY_SEED).choice(B, min(k, B), replace=False))


def source_hash(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1804_06363_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def oracle_runner(workload_name, cores):
    """The oracle's basis for the workload (from the stored greedy selection) behind a spawn pool."""
    import workloads as wl
    from oracle import baseline
    g = load_golden()
    if g is None or g.get("workload") != wl.WORKLOADS[workload_name]().name:
        return None, "no stored oracle greedy selection for this workload"
    return baseline.OracleRunner(workload_name, g["selected"], cores), None


def run_reference(args):
    """--impl reference: the FP64 oracle (Alg. 3) timed on the host cores, each step a bounded sample."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads as wl
    w = wl.WORKLOADS[args.workload]()
    cores = min(16, os.cpu_count() or 1)
    g = load_golden()
    key = "iters" if args.cpu_nu == 1 else f"iters_nu{args.cpu_nu}"
    if g is None or g.get("workload") != w.name or key not in g:
        print(json.dumps({"impl": "reference", "unavailable": "no stored oracle iteration counts for this "
                                                              "workload and sweep count"}))
        return
    runner, why = oracle_runner(args.workload, cores)
    if runner is None:
        print(json.dumps({"impl": "reference", "unavailable": why}))
        return
    mean_iters = float(sum(g[key])) / len(g[key])
    mu = w.test_mu(cores * (args.warmup + args.steps))
    samples = [runner.sample(mu[s * cores:(s + 1) * cores], args.cpu_iters, args.cpu_nu)
               for s in range(args.warmup + args.steps)]
    runner.close()
    timed = samples[args.warmup:]
    its = sum(t[0] for t in timed)
    wall = sum(t[1] for t in timed)
    value = its / wall / mean_iters
    sample = (f"{cores} test parameters per step, one per core, {args.cpu_iters} Alg. 3 iterations each with "
              f"{args.cpu_nu} red-black sweeps; solves/s = iteration rate / the oracle's mean {mean_iters:.1f} "
              f"iterations per solve at that sweep count (stored oracle counts of 16 complete solves)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(1, len(timed)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "solver": "oracle FP64 Alg. 3 (numpy)",
                                            "smoother": f"red-black GS nu={args.cpu_nu}", "beta": "pr",
                                            "tol": 1e-10, "cores": cores},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def progress(msg: str) -> None:
    """One line of progress on stderr (the JSON result goes to stdout)."""
    sys.stderr.write("[bench %.1fs] %s\n" % (time.perf_counter() - T_START, msg))
    sys.stderr.flush()


T_START = time.perf_counter()


def warm_start_experiment(ctx, w, args, opts, dev, stream):
    """Learned warm starts: networks trained on truth solves supply x_0 = W c(mu) (coefficients in
    span(W)) or x_0 = x_hat(mu) + V z(mu) (an error basis V, the POD of x - x_hat over training
    solutions, which leaves span(W)).  Each start is timed as a whole (starting vector + RBCG) on
    the same test queries; the set-up (truth solves, POD, training) is reported beside it with the
    number of solves after which it pays off."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_1804_06363_gb300 import rb
    prob = w.problem
    N, n = prob.n_dof, ctx.n
    S = args.warm_pairs
    chunk = args.batch or w.batch
    m_err = args.warm_modes
    s_pod = min(256, chunk, S)
    mu_tr = wl.mlp_train_mu(w, S)
    Y = np.zeros((S, n))
    Z = np.zeros((S, m_err))
    xb = torch.zeros((chunk, N), dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    pod_s = 0.0
    for c0 in range(0, S, chunk):
        m = np.ascontiguousarray(mu_tr[c0:c0 + chunk])
        ctx.pcg(m, xb[:len(m)], **opts)
        Y[c0:c0 + len(m)] = ctx.coefficients(xb[:len(m)], stream=stream.cuda_stream)
        if c0 == 0:
            tp = time.perf_counter()
            _, sig = ctx.error_basis(m[:s_pod], xb[:s_pod], m_err, stream=stream.cuda_stream)
            pod_s = time.perf_counter() - tp
        Z[c0:c0 + len(m)] = ctx.error_coefficients(m, xb[:len(m)], m_err, stream=stream.cuda_stream)
    pairs_s = time.perf_counter() - t0 - pod_s
    progress(f"warm start: {S} truth solves and their coefficients in {pairs_s:.1f} s, error basis "
             f"({s_pod} snapshots, {m_err} modes) in {pod_s:.2f} s")
    del xb
    sizes = wl.mlp_layer_sizes(prob.n_mu, n)
    sizes_e = wl.mlp_layer_sizes(prob.n_mu, m_err)
    net = rb.Mlp(prob.n_mu, prob.P, sizes[1], n, rb.flatten_params(wl.mlp_init(sizes)), max_samples=S)
    net_e = rb.Mlp(prob.n_mu, prob.P, sizes_e[1], m_err, rb.flatten_params(wl.mlp_init(sizes_e)), max_samples=S)
    torch.cuda.synchronize()
    train = {}
    for name, nt, targets in (("learned", net, Y), ("error_basis", net_e, Z)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        hist = nt.fit(mu_tr, targets, args.warm_steps, lr=3e-3, stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        train[name] = (a.elapsed_time(b), hist)
        progress(f"warm start: {name} network, {args.warm_steps} Adam steps in {train[name][0]:.0f} ms, "
                 f"loss {hist[0]:.3g} -> {hist[-1]:.3g}")

    T = args.warm_test or (args.batch or w.batch)
    mu = np.ascontiguousarray(w.draw_mu(w.test_seed, T))
    x = torch.zeros((T, N), dtype=torch.float64, device=dev)
    out = {"workload": w.name, "pairs": S, "pairs_solve_s": round(pairs_s, 2), "network": "x".join(map(str, sizes)),
           "error_basis": {"snapshots": s_pod, "modes": m_err, "pod_s": round(pod_s, 3),
                           "singular_values_first_last": [float(sig[0]), float(sig[-1])],
                           "network": "x".join(map(str, sizes_e))},
           "adam_steps": args.warm_steps,
           "train_ms": {k: round(v[0], 1) for k, v in train.items()},
           "loss_first_last": {k: [float(v[1][0]), float(v[1][-1])] for k, v in train.items()},
           "test_queries": T}
    ref = None

    def start(name):
        if name == "cold":
            x.zero_()   # rb_pcg zeroes x itself for a cold start; this keeps x0 visible below
        elif name == "galerkin":
            ctx.warm_start(mu, x, stream=stream.cuda_stream)
        elif name == "learned":
            ctx.warm_start(mu, x, net=net, stream=stream.cuda_stream)
        else:
            ctx.warm_start_error(mu, x, net=net_e, stream=stream.cuda_stream)

    for name in ("cold", "galerkin", "learned", "error_basis"):
        kw = {**opts, "x0": name != "cold"}

        def run():
            start(name)
            return ctx.pcg(mu, x, **kw)

        run()                                    # warm-up
        start(name)
        x0 = x.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status, st = run()
        e1.record(stream)
        torch.cuda.synchronize()
        s_ = e0.elapsed_time(e1) / 1000.0
        if ref is None:
            ref = x.clone()
        err0 = ((x0 - ref).norm(dim=1) / ref.norm(dim=1)).mean().item()
        dev_sol = ((x - ref).norm(dim=1) / ref.norm(dim=1)).max().item()
        out[name] = {"solves_per_s": round(T / s_, 1), "mean_iters": float(st["iters"].mean()),
                     "mean_outer": float(st["outer"].mean()), "all_converged": bool(np.all(st["status"] == 0)),
                     "max_rel_res": float(st["rel_res"].max()), "mean_initial_rel_error": err0,
                     "max_rel_diff_to_cold_solution": dev_sol}
        progress(f"warm start: {name}: {out[name]}")
    # set-up cost of each learned start and the number of solves after which it pays off
    v_cold = out["cold"]["solves_per_s"]
    for name, extra in (("learned", train["learned"][0] / 1000.0),
                        ("error_basis", train["error_basis"][0] / 1000.0 + pod_s)):
        setup = pairs_s + extra
        v = out[name]["solves_per_s"]
        gain = 1.0 / v_cold - 1.0 / v
        out[name]["setup_s"] = round(setup, 2)
        out[name]["break_even_solves"] = round(setup / gain) if gain > 0 else None
    net.close()
    net_e.close()
    return out


def n_sweep(args, w, ctx, dev, stream):
    """Steps to relative residual 1e-10 of RBI (Alg. 2) and RBCG (Alg. 3, FP64, PR beta) versus the
    basis size N, on the workload's test parameters, with the leading N vectors of one greedy basis
    (the greedy's bases are nested).  Per N: mean, best and worst step counts and their mid-range
    (the paper's Fig. 5 plots the average of the best and the worst case), and the throughput of
    the mixed-precision RBCG on the same queries."""
    import numpy as np
    import torch
    from paper_1804_06363_gb300 import rb
    prob = w.problem
    sizes = [int(t) for t in args.n_sweep.split(",") if t.strip()]
    W, ANq, fNr, _, _ = ctx.basis()
    mu = w.test_mu()
    B = len(mu)
    x = torch.zeros((B, prob.n_dof), dtype=torch.float64, device=dev)
    rows = []

    def summary(st):
        it = st["iters"].astype(np.int64)
        return {"mean": float(it.mean()), "best": int(it.min()), "worst": int(it.max()),
                "mid_range": 0.5 * float(it.min() + it.max()),
                "converged": int(np.sum(st["status"] == rb.RB_OK))}

    for n in sizes:
        c = rb.Context.from_arrays(prob, W[:, :n], ANq[:, :n, :n], fNr[:, :n], max_batch=B)
        x.zero_()
        _, st_rbi = c.solve(mu, x, max_iter=20000, stream=stream.cuda_stream)
        x.zero_()
        _, st_cg = c.pcg(mu, x, precision="fp64", beta="pr", max_iter=5000, stream=stream.cuda_stream)
        row = {"N": n, "rbi_steps": summary(st_rbi), "rbcg_steps": summary(st_cg)}
        # mixed precision with each engine of the projections, TF32 tensor cores (auto) and FP32
        # (zero start), and the FP32 engine from the RB approximation
        for key, gemm, x0 in (("rbcg_mixed_tf32", "auto", "zero"), ("rbcg_mixed_fp32", "cuda_cores", "zero"),
                              ("rbcg_mixed_fp32_rb_start", "cuda_cores", "rb")):
            x.zero_()
            c.pcg(mu, x, precision="mixed", gemm=gemm, x0=x0, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record(stream)
            _, st_mx = c.pcg(mu, x, precision="mixed", gemm=gemm, x0=x0, stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            row[key] = {"solves_per_s": round(B / (e0.elapsed_time(e1) / 1000.0), 1),
                        "mean_inner_iters": float(st_mx["iters"].mean()),
                        "mean_outer": float(st_mx["outer"].mean()),
                        "converged": int(np.sum(st_mx["status"] == rb.RB_OK))}
        rows.append(row)
        progress(f"N = {n}: RBI {rows[-1]['rbi_steps']['mid_range']}, RBCG {rows[-1]['rbcg_steps']['mid_range']} "
                 f"(mid-range of best and worst steps)")
        c.close()
    return {"metric": "steps to rel. residual 1e-10 versus RB dimension N", "workload": w.name,
            "grid": "x".join(map(str, prob.dims)), "queries": B, "smoother": "red-black GS nu=1",
            "data": "synthetic", "n_sweep": rows}


def leg_3d(args, dev, stream, peak, peak_kind):
    """The 3D workload (128^3, P = 8, n = 60, 256 queries per step) on the same GPU after the 2D
    results: basis built by the GPU greedy (snapshots by mixed-precision RBCG to 1e-11), the
    autotuner on 64 tuning parameters, warm-up, timed steps with their own clock record, then a
    per-kernel pass for the roofline of its dominant kernel."""
    import numpy as np
    import torch

    import workloads as wl
    from paper_1804_06363_gb300 import rb
    w = wl.batched_3d_128()
    prob = w.problem
    B, N = w.batch, prob.n_dof
    t0 = time.perf_counter()
    ctx = rb.Context.build(prob, w.n_basis, w.train_mu(), max_batch=B, precision="mixed", stream=stream.cuda_stream)
    build_s = time.perf_counter() - t0
    progress(f"3D leg: basis of {w.name} ready in {build_s:.1f} s")
    mu = np.ascontiguousarray(w.test_mu(B))
    x = torch.zeros((B, N), dtype=torch.float64, device=dev)
    opts = base_options("mixed", stream.cuda_stream)
    tuned = tune(ctx, w, x, opts, n_sample=64)
    progress(f"3D leg: autotuned {tuned}")
    ctx.pcg(mu, x, **opts)
    torch.cuda.synchronize()
    clk = Clocks(dev.index or 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.leg3d_steps):
        status, st = ctx.pcg(mu, x, **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    secs = e0.elapsed_time(e1) / 1000.0
    value = B * args.leg3d_steps / secs
    progress(f"3D leg: {value:.1f} solves/s, mean iterations {float(st['iters'].mean()):.1f}")
    ctx.profile(True)
    _, stp = ctx.pcg(mu, x, **opts)
    ctx.profile(False)
    prof = ctx.profile_read()
    kernels, units = kernel_table(prof, "f32", opts, N, int(stp["iters"].sum()), int(stp["outer"].sum()))
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    achieved = kernels[dom].get("gbs")
    n_launch = max(1, kernels[dom]["launches"])
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4) if achieved else None, "traffic": None, "peak_source": peak_kind,
                "alg_bytes_per_unit": kernels[dom].get("alg_bytes_per_point"),
                "alg_bytes_per_launch": round((kernels[dom].get("alg_bytes") or 0) / n_launch)}
    if "pass_gbs" in kernels[dom]:
        roofline["per_pass"] = {"bytes_per_point": kernels[dom]["pass_bytes_per_point"],
                                "achieved": kernels[dom]["pass_gbs"], "frac": round(kernels[dom]["pass_gbs"] / peak, 4)}
    out = {"workload": w.name, "metric": "RB-PCG solves/sec to rel. residual 1e-10", "value": value,
           "unit": "solves/s", "steps": args.leg3d_steps, "warmup": 1, "ms_per_step": 1000.0 * secs / args.leg3d_steps,
           "queries_per_step": B, "grid": "x".join(map(str, prob.dims)), "P": prob.P, "n_basis": w.n_basis,
           "all_converged": bool(np.all(st["status"] == rb.RB_OK)), "mean_iters": float(st["iters"].mean()),
           "max_rel_res": float(st["rel_res"].max()), "autotuned": tuned, "offline_build_s": round(build_s, 1),
           "roofline": roofline, "kernels": kernels, "clocks": clocks,
           "l2": "inputs larger than L2 (FP64 solutions %.1f GB per step)" % (B * N * 8 / 1e9)}
    ctx.close()
    return out


def kernel_table(prof, prec, opts, N, iters, outers, alu=None):
    """Per-kernel device time and algorithmic bytes from the rb_profile counters.  alu =
    (FP64 flops per point of the outer residual, measured FP64 FMA rate in flop/s) adds that
    kernel's arithmetic roofline."""
    nu = max(1, opts["nu"])
    units = {"cg_a": iters, "cg_b": iters, "smooth": iters, "project": iters, "tc_project": iters,
             "prolong": iters, "tc_prolong": iters, "outer_residual": outers, "outer_update": outers}
    bf16 = prec == "f32" and opts.get("store", "f32") == "bf16"
    kernels = {}
    for k, (n_launch, ms) in prof.items():
        bpp = BYTES_PER_POINT[prec].get(k)
        if bf16 and k in ("prolong", "tc_prolong"):
            bpp = BF16_PROLONG
        entry = {"launches": n_launch, "ms": round(ms, 3)}
        if bpp is not None and ms > 0:
            alg = bpp * N * units[k]
            entry["alg_bytes"] = alg
            entry["alg_bytes_per_point"] = bpp
            entry["gbs"] = round(alg / (ms / 1000.0) / 1e9, 1)
            if k == "smooth":
                # the streaming passes over memory of one application
                if bf16:
                    pas = BF16_SMOOTH_LAST + BF16_SMOOTH_SWEEP * (nu - 1)
                else:
                    passes = smoother_passes(opts.get("kernels", 0), nu) if prec == "f32" else nu
                    pas = bpp + SWEEP_PASS_BYTES[prec] * (passes - 1)
                entry["pass_bytes_per_point"] = pas
                entry["pass_gbs"] = round(pas * N * units[k] / (ms / 1000.0) / 1e9, 1)
        if k == "outer_residual" and alu is not None and ms > 0:
            fpp, rate = alu
            tf = fpp * N * units[k] / (ms / 1000.0) / 1e12
            entry["fp64_flops_per_point"] = fpp
            entry["fp64_tflops"] = round(tf, 3)
            entry["fp64_frac"] = round(tf / (rate / 1e12), 4)
        kernels[k] = entry
    return kernels, units


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus, sys.argv[1:]))
    if args.rank_check:
        rank_check(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import workloads as wl
    from paper_1804_06363_gb300 import rb

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = wl.WORKLOADS[args.workload]()
    prob = w.problem
    B = args.batch or w.batch
    N = prob.n_dof

    # ---- CPU baseline (rank 0, one GPU only): a spawn pool of oracle processes rebuilds the
    #      oracle's basis in the background while the GPU works
    cores = min(16, os.cpu_count() or 1)
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick
    cpu_setup = {}

    def start_oracle():
        try:
            cpu_setup["runner"], cpu_setup["why"] = oracle_runner(args.workload, cores)
        except Exception as e:  # the baseline must not sink the GPU number
            cpu_setup["runner"], cpu_setup["why"] = None, f"oracle set-up failed: {type(e).__name__}: {e}"

    oracle_thread = None
    if want_cpu:
        import threading
        oracle_thread = threading.Thread(target=start_oracle, daemon=True)
        oracle_thread.start()

    # ---- offline (not timed): greedy basis on the GPU
    t0 = time.perf_counter()
    if args.basis and os.path.exists(args.basis):
        ctx = rb.Context.load(args.basis, max_batch=B)
    else:
        if args.mf_coarse > 0:
            import dataclasses
            coarse = dataclasses.replace(prob, dims=(args.mf_coarse,) * prob.dim)
            ctx = rb.Context.build_multi_fidelity(prob, coarse, w.n_basis, w.train_mu(), max_batch=B,
                                                  precision="mixed")
        else:
            n_build = max([w.n_basis] + [int(t) for t in args.n_sweep.split(",") if t.strip()])
            ctx = rb.Context.build(prob, n_build, w.train_mu(), max_batch=B, precision="mixed",
                                   stream=torch.cuda.current_stream(dev).cuda_stream)
        if args.basis:
            ctx.save(args.basis)
    offline_s = time.perf_counter() - t0
    progress(f"basis of {w.name} ready in {offline_s:.1f} s")
    _, _, _, _, sel = ctx.basis()
    if args.n_sweep:
        if rank == 0:
            print(json.dumps(n_sweep(args, w, ctx, dev, torch.cuda.current_stream(dev))))
        ctx.close()
        return 0

    # weak scaling: every rank solves its own B test parameters (replicas, no data-path collective)
    from paper_1804_06363_gb300.shard import max_over_ranks, shard_range
    mu_all = w.test_mu(B * world) if B * world <= w.n_test else w.draw_mu(w.test_seed, B * world)
    lo, hi = shard_range(B * world, rank, world)
    mu = np.ascontiguousarray(mu_all[lo:hi])
    x = torch.zeros((B, N), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    opts = base_options(args.precision, stream.cuda_stream)
    opts.update(nu=args.nu, gemm=args.gemm, kernels=args.kernels)

    # ---- autotuner (setup, not timed): on its own parameter stream, never on the timed test queries
    tuned = None
    if not args.no_tune:
        tuned = tune(ctx, w, x, opts)
        progress(f"autotuned: {tuned}")

    def step(xbuf, **kw):
        status, st = ctx.pcg(mu, xbuf, **{**opts, **kw})
        return status, st

    for _ in range(args.warmup):
        status, st = step(x)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = Clocks(local)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        status, st = step(x)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_local = e0.elapsed_time(e1) / 1000.0
    t_max = max_over_ranks(t_local, dist, dev)
    if world > 1:
        dist.barrier()
    value = world * B * args.steps / t_max
    last = stats[-1]
    progress(f"timed steps: {value:.1f} solves/s, mean iterations {float(last['iters'].mean()):.1f}")
    ok = bool(np.all(last["status"] == rb.RB_OK))

    # learned warm start (after the timed region; rank 0): on by default, off under --quick unless --warm
    warm = None
    if (args.warm or not args.quick) and not args.no_warm and rank == 0:
        try:
            warm = warm_start_experiment(ctx, w, args, opts, dev, stream)
        except Exception as e:  # the comparison must not sink the headline number
            warm = {"error": f"{type(e).__name__}: {e}"}

    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps,
                              "quick": True, "all_converged": ok, "mean_iters": float(last["iters"].mean()),
                              "config": {"workload": w.name, "queries_per_step_per_gpu": B, "autotuned": tuned},
                              "clocks": clocks, "warm_start": warm}))
        ctx.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- per-kernel device time (CUDA events around every launch; separate pass)
    ctx.profile(True)
    _, st_prof = step(x)
    ctx.profile(False)
    prof = ctx.profile_read()
    torch.cuda.synchronize()
    launches_per_step = sum(v[0] for v in prof.values())
    prec = "f32" if args.precision == "mixed" else "f64"
    iters = int(st_prof["iters"].sum())
    outers = int(st_prof["outer"].sum())
    fma64 = rb.fma_rate(True, stream.cuda_stream)   # measured FP64 rate (outside every timed region)
    fma32 = rb.fma_rate(False, stream.cuda_stream)
    kernels, units = kernel_table(prof, prec, opts, N, iters, outers,
                                  alu=(outer_flops(prob.dim, len(prob.loads)), fma64))
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    peak, peak_kind = measured_peaks()
    achieved = kernels[dom].get("gbs")
    n_launch = max(1, kernels[dom]["launches"])
    traffic, traffic_src = None, None
    nt = NCU_TRAFFIC.get((prec, opts.get("store", "f32"), opts.get("kernels", 0), dom, opts["nu"]))
    if nt is not None and source_hash(nt["sources"]) == nt["sha"]:
        traffic = round(nt["bytes_per_point"] * N * units[dom] / n_launch)
        traffic_src = nt["capture"]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4) if achieved else None, "traffic": traffic,
                "traffic_capture": traffic_src, "peak_source": peak_kind,
                "alg_bytes_per_unit": kernels[dom].get("alg_bytes_per_point"),
                "alg_bytes_per_launch": round((kernels[dom].get("alg_bytes") or 0) / n_launch),
                "unit_def": "one query x one grid point x one application of the kernel (each operand touched once)"}
    if "pass_gbs" in kernels[dom]:
        roofline["per_pass"] = {"bytes_per_point": kernels[dom]["pass_bytes_per_point"],
                                "achieved": kernels[dom]["pass_gbs"],
                                "frac": round(kernels[dom]["pass_gbs"] / peak, 4),
                                "what": "%d streaming passes over memory per application (nu = %d, kernels = %d)"
                                        % (smoother_passes(opts.get("kernels", 0), opts["nu"]) if prec == "f32"
                                           else opts["nu"], opts["nu"], opts.get("kernels", 0))}

    # ---- end to end through the C interface with host buffers (pinned)
    xh = torch.zeros((B, N), dtype=torch.float64, pin_memory=True).numpy()
    ctx.pcg(mu, xh, **{**opts, "stream": stream.cuda_stream})
    torch.cuda.synchronize()
    e2e_steps = min(args.steps, 10)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.pcg(mu, xh, **opts)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * B * e2e_steps / max_over_ranks(e2e_s, dist, dev), "unit": "solves/s",
           "steps": e2e_steps, "h2d_bytes_per_step": int(mu.nbytes), "d2h_bytes_per_step": int(B * N * 8 + B * 24)}

    # ---- FP64 plain comparator: the paper's method in FP64 on the same GPU, the same queries,
    #      its sweep count tuned on the same training sample as the mixed arm
    fp64 = None
    if args.fp64_queries >= 0 and args.precision == "mixed":
        q64 = B if args.fp64_queries == 0 else min(B, args.fp64_queries)
        x64 = x[:q64]
        opts64 = base_options("fp64", stream.cuda_stream)
        tuned64 = None
        if not args.no_tune:
            tuned64 = tune(ctx, w, x64, opts64)
        ctx.pcg(mu[:min(q64, 64)], x64[:min(q64, 64)], **opts64)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, st64 = ctx.pcg(mu[:q64], x64, **opts64)
        b.record(stream)
        torch.cuda.synchronize()
        s64 = a.elapsed_time(b) / 1000.0
        fp64 = {"value": q64 / s64, "unit": "solves/s", "queries": q64, "nu": opts64["nu"], "tuned": tuned64,
                "mean_iters": float(st64["iters"].mean()), "all_converged": bool(np.all(st64["status"] == 0)),
                "max_rel_res": float(st64["rel_res"].max()), "mixed_over_fp64": round(value / (q64 / s64), 2)}
        progress(f"FP64 comparator: {fp64['value']:.1f} solves/s on {q64} queries (nu {opts64['nu']})")
        # the timed solutions again (x was overwritten by the comparator), for the parity check
        step(x)
        torch.cuda.synchronize()

    # ---- CPU baseline and parity (rank 0, one GPU): complete oracle solves of a seeded sample of
    #      the timed queries at the GPU arm's sweep count; the oracle's sparse-direct truth of the
    #      same queries gives the error of the GPU's solutions per result
    cpu, parity = None, None
    runner, cpu_why = None, None
    if oracle_thread is not None:
        oracle_thread.join()
        runner, cpu_why = cpu_setup.get("runner"), cpu_setup.get("why")
    if want_cpu and runner is not None:
        try:
            idx = parity_sample(B, cores)
            wall, out = runner.solve([mu[i] for i in idx], opts["nu"])
            its = [o[0] for o in out]
            cpu = {"value": len(idx) / wall, "unit": "solves/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                   "sample": (f"{len(idx)} complete solves of seeded test queries of the timed batch, one per core, "
                              f"oracle FP64 Alg. 3 with the GPU arm's {opts['nu']} red-black sweeps, PR beta, "
                              f"tol 1e-10 ({wall:.1f} s wall, {np.mean(its):.1f} iterations per solve)"),
                   "mean_iters": float(np.mean(its)), "all_converged": all(o[3] < 1e-10 for o in out)}
            xs = x.cpu().numpy()
            errs = runner.errors([mu[i] for i in idx], [[xs[i], out[k][4]] for k, i in enumerate(idx)])
            e_gpu = [e[0][0] for e in errs]
            r_gpu = [e[0][1] for e in errs]
            e_orc = [e[1][0] for e in errs]
            parity = {"queries": idx, "truth": "oracle sparse-direct solve of eq. 1 (FP64)",
                      "gpu_rel_err": e_gpu, "max_rel_err": max(e_gpu), "median_rel_err": float(np.median(e_gpu)),
                      "max_oracle_rel_res_of_gpu": max(r_gpu), "oracle_rbcg_max_rel_err": max(e_orc),
                      "bar": 1e-9, "pass": max(e_gpu) <= 1e-9 and max(r_gpu) < 1e-10}
            progress(f"parity: max rel. error {parity['max_rel_err']:.3g} over {len(idx)} queries; "
                     f"CPU baseline {cpu['value']:.3f} solves/s")
        except Exception as e:  # the baseline must not sink the GPU number
            cpu = {"value": None, "unit": "solves/s", "cores": cores, "kind": "oracle",
                   "sample": f"oracle run failed: {type(e).__name__}: {e}"}
        runner.close()
    elif want_cpu:
        cpu = {"value": None, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": cpu_why}

    leg3d = None
    if rank == 0 and world == 1 and not args.no_leg3d and args.workload == "rbcg_2d_512":
        try:
            leg3d = leg_3d(args, dev, stream, peak, peak_kind)
        except Exception as e:  # the 3D leg must not sink the headline number
            leg3d = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": w.name, "grid": "x".join(map(str, prob.dims)), "P": prob.P, "n_basis": w.n_basis,
                       "queries_per_step_per_gpu": B, "precision": args.precision, "beta": "pr",
                       "smoother": f"red-black GS nu={opts['nu']}", "tol": 1e-10, "gemm": opts["gemm"],
                       "kernels": opts.get("kernels", 0), "store": opts.get("store", "f32"),
                       "inner_tol": opts.get("inner_tol"), "autotuned": tuned,
                       "l2": "inputs larger than L2 (FP64 solutions %.1f GB + FP32 work vectors per step)"
                             % (B * N * 8 / 1e9),
                       "offline_build_s": round(offline_s, 1), "greedy_selected_first": [int(s) for s in sel[:8]]},
            "all_converged": ok, "mean_iters": float(last["iters"].mean()), "max_iters": int(last["iters"].max()),
            "mean_outer": float(last["outer"].mean()), "max_rel_res": float(last["rel_res"].max()),
            "roofline": roofline, "kernels": kernels, "gpu_launches": int(launches_per_step * args.steps),
            "e2e": e2e, "fp64_plain": fp64, "cpu_baseline": cpu, "parity": parity, "clocks": clocks,
            "fma_rate": {"fp64_tflops": round(fma64 / 1e12, 3), "fp32_tflops": round(fma32 / 1e12, 2),
                         "what": "measured by rb_fma_rate on this GPU; denominator of the outer residual's "
                                 "fp64_frac"},
        }
        if warm is not None:
            line["warm_start"] = warm
        if leg3d is not None:
            line["leg_3d"] = leg3d
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
