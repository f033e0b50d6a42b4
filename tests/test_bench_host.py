"""Host-side arithmetic of bench.py (CPU only): passes over memory per smoother application,
FP64 flops of the outer residual, and the per-kernel byte table that the roofline reads."""
import bench


def test_smoother_passes():
    assert bench.smoother_passes(0, 6) == 6          # one pass per sweep
    assert bench.smoother_passes(2, 4) == 4
    assert bench.smoother_passes(1, 5) == 1          # all sweeps fused
    assert bench.smoother_passes(3, 9) == 3          # three sweeps per pass
    assert bench.smoother_passes(3, 7) == 3
    assert bench.smoother_passes(4, 5) == 3          # two sweeps per pass


def test_outer_flops():
    # loads (one FMA per term) + (2 d + 1)-point stencil (one FMA per coefficient) + difference + two squares
    assert bench.outer_flops(2, 3) == 6 + 10 + 5
    assert bench.outer_flops(3, 1) == 2 + 14 + 5


def test_kernel_table_bytes_and_rates():
    N, iters, outers = 1000, 10, 2
    prof = {"smooth": (10, 2.0), "cg_b": (10, 1.0), "outer_residual": (2, 0.5)}
    opts = {"nu": 9, "kernels": 3}
    k, units = bench.kernel_table(prof, "f32", opts, N, iters, outers, alu=(21, 1.0e12))
    s = k["smooth"]
    assert s["alg_bytes"] == 16 * N * iters
    assert abs(s["gbs"] - 16 * N * iters / 2.0e-3 / 1e9) < 0.1
    assert s["pass_bytes_per_point"] == 16 + 12 * 2          # three passes
    assert k["cg_b"]["alg_bytes"] == 20 * N * iters
    o = k["outer_residual"]
    assert o["alg_bytes"] == 12 * N * outers
    assert abs(o["fp64_tflops"] - 21 * N * outers / 0.5e-3 / 1e12) < 1e-3
    # one pass per sweep
    k0, _ = bench.kernel_table(prof, "f32", {"nu": 6, "kernels": 0}, N, iters, outers)
    assert k0["smooth"]["pass_bytes_per_point"] == 16 + 12 * 5
