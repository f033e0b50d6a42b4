"""Multi-process (gloo, CPU) checks of the query sharding and the max-over-ranks timing."""
import os
import socket

import pytest

from paper_1804_06363_gb300.shard import max_over_ranks, shard_range

torch = pytest.importorskip("torch")


def test_shard_ranges_cover_and_balance():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            parts = [shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, stop = shard_range(1001, rank, world)
    # every rank reports a different "step time"; all must see the maximum
    t = max_over_ranks(1.5 + rank, dist, "cpu")
    counts = torch.tensor([stop - start], dtype=torch.int64)
    dist.all_reduce(counts)
    out.put((rank, start, stop, t, int(counts.item())))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_agree_on_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, b0, t0, c0), (r1, a1, b1, t1, c1) = res
    assert (a0, b0, a1, b1) == (0, 501, 501, 1001)
    assert t0 == t1 == 2.5
    assert c0 == c1 == 1001


def test_bench_launches_its_own_ranks():
    """bench.py --gpus 2 outside a launcher starts two ranks itself (torch.distributed.run on
    127.0.0.1); --rank-check runs the rank logic on gloo without a GPU: the shards cover the
    whole batch and every rank reports the maximum step time."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--rank-check",
                        "--batch", "1000"], cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["n_ranks"] == 2 and d["queries"] == 2000
    shards = sorted(tuple(s) for s in d["shards"])
    assert shards == [(0, 0, 1000), (1, 1000, 2000)]
    assert d["t_max"] == 2.0
