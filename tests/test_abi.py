"""The C-ABI library builds, loads and exports every symbol include/rb.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rb.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(rb_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1804_06363_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rb_offline_load", "rb_offline_load_arrays", "rb_solve", "rb_pcg", "rb_apply",
                     "rb_last_error", "rb_free"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in _declared_functions():
        assert name in exported, name


def test_binding_covers_the_header(libpath):
    from paper_1804_06363_gb300 import rb
    assert set(rb.SIGNATURES) == set(_declared_functions())
    lib = rb.lib()
    o = rb.make_opts()
    assert o.tol == 1e-10 and o.nu == 1 and o.beta_form == rb.BETAS["pr"]
    assert o.adaptive_n == 0 and o.gamma == 10.0
    assert lib.rb_status_string(rb.RB_ENOCONV) == b"not converged"


def test_struct_layouts_match_header(libpath):
    """Field order / sizes of the ctypes mirrors agree with the C structs."""
    from paper_1804_06363_gb300 import rb
    assert ctypes.sizeof(rb.RbLoad) == 4 + 4 + 24 + 8 + 4 + 4 + 8    # field, padding, values
    assert ctypes.sizeof(rb.RbStats) == 4 * 4 + 8 + 8       # n_used and the tail padding
    assert rb.RbStats.n_used.offset == 24
    assert rb.RbOpts.adaptive_n.offset == rb.RbOpts.store.offset + 4 and rb.RbOpts.gamma.offset % 8 == 0
    assert rb.RbOpts.stream.offset == ctypes.sizeof(rb.RbOpts) - 8


def test_invalid_problem_is_rejected_without_gpu(libpath):
    """Argument validation runs before any CUDA call."""
    import workloads as wl
    from paper_1804_06363_gb300 import rb
    prob = wl.small((8, 8), (2, 2), n_basis=1).problem
    p, keep = rb.make_problem(prob)
    p.dim = 4
    h = ctypes.c_void_p()
    st = rb.lib().rb_offline_load_arrays(ctypes.byref(h), ctypes.byref(p), 0, None, None, None, 1)
    assert st == rb.RB_EINVAL and not h.value
    assert b"dim" in rb.lib().rb_last_error(None)


def test_field_problems_are_validated_without_gpu(libpath):
    """Coefficient fields and array / boundary loads: the checks of rb_problem run before any CUDA call."""
    import workloads as wl
    from paper_1804_06363_gb300 import rb
    lib = rb.lib()
    prob = wl.case_problem("case2", (6, 5, 4))
    h = ctypes.c_void_p()

    def rejected(edit, word):
        p, keep = rb.make_problem(prob)
        edit(p)
        st = lib.rb_offline_load_arrays(ctypes.byref(h), ctypes.byref(p), 0, None, None, None, 1)
        assert st == rb.RB_EINVAL and not h.value
        assert word in lib.rb_last_error(None), lib.rb_last_error(None)

    def blocks(p):
        p.nb[0] = 2
    rejected(blocks, b"one block")

    def field_index(p):
        p.loads[1].field = 2
    rejected(field_index, b"field index")

    def no_values(p):
        p.loads[0].values = None
    rejected(no_values, b"values")

    def no_fields(p):
        p.fields = None
    rejected(no_fields, b"n_fields")

    def few_mu(p):
        p.n_mu = 1
    rejected(few_mu, b"n_mu")
    # the no-allocation residual needs a context for such problems
    p, keep = rb.make_problem(prob)
    mu = (ctypes.c_double * 6)(1.0, 0.5, 0.5, 0.25, 0.5, 0.25)
    out = (ctypes.c_double * 1)()
    assert lib.rb_residual_noalloc(ctypes.byref(p), 1, mu, ctypes.c_void_p(16), out, None) == rb.RB_EINVAL
    assert b"context" in lib.rb_last_error(None)


def test_network_and_warm_start_arguments_are_validated_without_gpu(libpath):
    """rb_mlp_create checks its sizes, rb_warm_start / rb_coefficients their context, before any CUDA call."""
    from paper_1804_06363_gb300 import rb
    lib = rb.lib()
    h = ctypes.c_void_p()
    params = (ctypes.c_double * 8)()
    for args in ((0, 0, 8, 4), (33, 0, 8, 4), (4, 5, 8, 4), (4, 2, 129, 4), (4, 2, 8, 129), (4, 2, 0, 4)):
        st = lib.rb_mlp_create(ctypes.byref(h), *args, params, 16)
        assert st == rb.RB_EINVAL and not h.value, args
    assert b"sizes" in lib.rb_last_error(None)
    bad = (ctypes.c_double * (8 * 4 + 8 + 8 * 8 + 8 + 3 * 8 + 3))()
    bad[5] = float("nan")
    assert lib.rb_mlp_create(ctypes.byref(h), 4, 2, 8, 3, bad, 16) == rb.RB_EINVAL and not h.value
    assert b"finite" in lib.rb_last_error(None)
    assert lib.rb_mlp_num_params(None) == -1
    assert lib.rb_warm_start(None, None, 1, None, None, None, None) == rb.RB_EINVAL
    assert lib.rb_coefficients(None, 1, None, None, None) == rb.RB_EINVAL
    lib.rb_mlp_free(None)


def test_network_parameter_layout_round_trip():
    """flatten_params follows the header's order (W1, b1, W2, b2, W3, b3) and unflatten_params inverts it."""
    import numpy as np

    import workloads as wl
    from paper_1804_06363_gb300 import rb
    sizes = (5, 7, 7, 3)
    layers = [(W, np.arange(W.shape[0], dtype=float) + 100 * l) for l, (W, _) in enumerate(wl.mlp_init(sizes))]
    flat = rb.flatten_params(layers)
    assert flat.size == 5 * 7 + 7 + 7 * 7 + 7 + 7 * 3 + 3
    np.testing.assert_array_equal(flat[:35], layers[0][0].ravel())
    np.testing.assert_array_equal(flat[35:42], layers[0][1])
    back = rb.unflatten_params(flat, sizes)
    for (W, b), (W2, b2) in zip(layers, back):
        np.testing.assert_array_equal(W, W2)
        np.testing.assert_array_equal(b, b2)


def test_struct_layouts_match_compiled_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal what a C compiler makes of include/rb.h."""
    import shutil
    from paper_1804_06363_gb300 import rb
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = {"rb_opts": (rb.RbOpts, ["tol", "nu", "omega", "inner_tol", "store", "adaptive_n", "gamma", "stream"]),
              "rb_stats": (rb.RbStats, ["iters", "status", "rel_res", "n_used"]),
              "rb_problem": (rb.RbProblem, ["dim", "m", "nb", "n_loads", "loads", "n_mu", "n_fields", "fields"]),
              "rb_load": (rb.RbLoad, ["kind", "param", "center", "sigma", "field", "values"]),
              "rb_tune_result": (rb.RbTuneResult, ["nu", "inner_tol", "ms_per_solve", "store", "x0_mode"]),
              "rb_kernel_time": (rb.RbKernelTime, ["name", "launches", "ms"])}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rb.h"', "int main(void) {"]
    for cname, (_, fields) in checks.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for cname, (cls, fields) in checks.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f in fields:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)
