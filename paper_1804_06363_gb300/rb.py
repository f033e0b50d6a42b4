"""ctypes binding of librb (include/rb.h): argument marshalling only.

Every computation runs in the CUDA library.  Arrays may be numpy arrays (host
memory) or any object exposing ``__cuda_array_interface__`` (device memory,
e.g. a CUDA tensor); plain integers are taken as raw device pointers.  If the
library is missing this module raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librb.so")

RB_OK, RB_EINVAL, RB_ENOMEM, RB_EFORMAT, RB_ECUDA, RB_EBREAKDOWN, RB_ENOCONV, RB_ETIMEOUT, RB_EIO = range(9)
STATUS_NAMES = ["ok", "einval", "enomem", "eformat", "ecuda", "ebreakdown", "enoconv", "etimeout", "eio"]
SMOOTHERS = {"none": 0, "rbgs": 1, "jacobi": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
BETAS = {"fr": 0, "pr": 1}
GEMMS = {"auto": 0, "cuda_cores": 1, "tensor": 2}
STORES = {"f32": 0, "bf16": 1}
STARTS = {"zero": 0, "given": 1, "rb": 2}


LOAD_KINDS = {"const": 0, "gauss": 1, "array": 2, "boundary": 3}


class RbLoad(C.Structure):
    _fields_ = [("kind", C.c_int), ("param", C.c_int), ("center", C.c_double * 3), ("sigma", C.c_double),
                ("field", C.c_int), ("values", C.c_void_p)]


class RbProblem(C.Structure):
    _fields_ = [("dim", C.c_int), ("m", C.c_int * 3), ("nb", C.c_int * 3), ("n_loads", C.c_int),
                ("loads", C.POINTER(RbLoad)), ("n_mu", C.c_int), ("n_fields", C.c_int), ("fields", C.c_void_p)]


class RbOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("smoother", C.c_int), ("nu", C.c_int),
                ("omega", C.c_double), ("precision", C.c_int), ("beta_form", C.c_int), ("x0_mode", C.c_int),
                ("inner_tol", C.c_double), ("max_outer", C.c_int), ("gemm", C.c_int), ("graph", C.c_int),
                ("kernels", C.c_int), ("store", C.c_int), ("adaptive_n", C.c_int), ("gamma", C.c_double),
                ("stream", C.c_void_p)]


class RbStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("rel_res", C.c_double), ("n_used", C.c_int)]


class RbBuildOpts(C.Structure):
    _fields_ = [("truth_tol", C.c_double), ("truth_max_iter", C.c_int), ("score", C.c_int),
                ("drop_tol", C.c_double)]


class RbTuneResult(C.Structure):
    _fields_ = [("nu", C.c_int), ("inner_tol", C.c_double), ("gemm", C.c_int), ("ms_per_solve", C.c_double),
                ("trials", C.c_int), ("kernels", C.c_int), ("store", C.c_int), ("x0_mode", C.c_int)]


class RbKernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_longlong), ("ms", C.c_double)]


_lib = None

# every function declared in include/rb.h, with its ctypes signature
SIGNATURES = {
    "rb_default_opts": (None, [C.POINTER(RbOpts)]),
    "rb_default_build_opts": (None, [C.POINTER(RbBuildOpts)]),
    "rb_offline_load_arrays": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(RbProblem), C.c_int, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_int]),
    "rb_offline_build": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(RbProblem), C.c_int, C.c_int, C.c_void_p,
                                   C.POINTER(RbBuildOpts), C.POINTER(RbOpts), C.c_int]),
    "rb_offline_build_mf": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(RbProblem), C.POINTER(RbProblem), C.c_int,
                                      C.c_int, C.c_void_p, C.POINTER(RbBuildOpts), C.POINTER(RbOpts), C.c_int]),
    "rb_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "rb_offline_load": (C.c_int, [C.POINTER(C.c_void_p), C.c_char_p, C.c_int]),
    "rb_debug_wait": (C.c_int, [C.c_void_p, C.c_double, C.c_longlong]),
    "rb_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int),
                          C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "rb_get_basis": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rb_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(RbOpts), C.c_void_p]),
    "rb_pcg": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(RbOpts), C.c_void_p]),
    "rb_pcg_ragged": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(RbOpts),
                                C.c_void_p]),
    "rb_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rb_products": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "rb_precondition": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(RbOpts)]),
    "rb_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(RbOpts),
                              C.POINTER(RbTuneResult)]),
    "rb_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "rb_profile_read": (C.c_int, [C.c_void_p, C.POINTER(RbKernelTime), C.c_int, C.POINTER(C.c_int)]),
    "rb_fma_rate": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_void_p]),
    "rb_residual_noalloc": (C.c_int, [C.POINTER(RbProblem), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "rb_warm_start": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rb_error_basis": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "rb_error_coefficients": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rb_warm_start_error": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "rb_coefficients": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rb_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "rb_mlp_num_params": (C.c_int, [C.c_void_p]),
    "rb_mlp_fit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                             C.c_void_p]),
    "rb_mlp_gradient": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "rb_mlp_predict": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "rb_mlp_get": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "rb_mlp_free": (None, [C.c_void_p]),
    "rb_last_error": (C.c_char_p, [C.c_void_p]),
    "rb_status_string": (C.c_char_p, [C.c_int]),
    "rb_free": (None, [C.c_void_p]),
}


def lib() -> C.CDLL:
    """Load librb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1804_06363_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class RbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def _ptr(a) -> int:
    """Raw address of a host (numpy) or device (__cuda_array_interface__) array, or an int."""
    if a is None:
        return 0
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    cai = getattr(a, "__cuda_array_interface__", None)
    if cai is not None:
        if cai.get("strides") is not None:
            raise ValueError("device arrays must be contiguous")
        return int(cai["data"][0])
    raise TypeError(f"cannot take the address of {type(a)}")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_problem(prob):
    """rb_problem from a problem description with dims, blocks, loads and n_mu (and, for problems
    with coefficient fields or array / boundary loads, field_values() and load_values(r)).
    Returns the structure and the objects that must stay alive while it is used."""
    dims = list(prob.dims) + [1] * (3 - len(prob.dims))
    blocks = list(prob.blocks) + [1] * (3 - len(prob.blocks))
    loads = (RbLoad * len(prob.loads))()
    keep = [loads]
    for i, ld in enumerate(prob.loads):
        loads[i].kind = LOAD_KINDS[ld.kind]
        loads[i].param = ld.param
        for j in range(3):
            loads[i].center[j] = ld.center[j]
        loads[i].sigma = ld.sigma
        loads[i].field = getattr(ld, "field", 0)
        if loads[i].kind >= 2:
            vals = _f64(prob.load_values(i))
            keep.append(vals)
            loads[i].values = vals.ctypes.data
    p = RbProblem()
    p.dim = len(prob.dims)
    for j in range(3):
        p.m[j] = dims[j]
        p.nb[j] = blocks[j]
    p.n_loads = len(prob.loads)
    p.loads = C.cast(loads, C.POINTER(RbLoad))
    p.n_mu = prob.n_mu
    fields = prob.field_values() if hasattr(prob, "field_values") else None
    if fields is not None:
        fields = _f64(fields)
        keep.append(fields)
        p.n_fields = fields.shape[0]
        p.fields = fields.ctypes.data
    return p, keep


def make_opts(**kw) -> RbOpts:
    o = RbOpts()
    lib().rb_default_opts(C.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "smoother":
            v = SMOOTHERS[v] if isinstance(v, str) else v
        elif k == "precision":
            v = PRECISIONS[v] if isinstance(v, str) else v
        elif k == "beta":
            k, v = "beta_form", BETAS[v] if isinstance(v, str) else v
        elif k == "gemm":
            v = GEMMS[v] if isinstance(v, str) else v
        elif k == "store":
            v = STORES[v] if isinstance(v, str) else v
        elif k == "x0":   # "zero", "given", "rb", or a bool (True: given)
            k, v = "x0_mode", STARTS[v] if isinstance(v, str) else (1 if v else 0)
        elif k == "stream":
            v = C.c_void_p(int(v) if v else 0)
        elif k == "graph":
            v = int(bool(v))
        setattr(o, k, v)
    return o


def stats_array(st) -> np.ndarray:
    n = len(st)
    out = np.zeros(n, dtype=[("iters", "i4"), ("outer", "i4"), ("restarts", "i4"), ("status", "i4"),
                             ("rel_res", "f8"), ("n_used", "i4")])
    for i in range(n):
        out[i] = (st[i].iters, st[i].outer, st[i].restarts, st[i].status, st[i].rel_res, st[i].n_used)
    return out


def fma_rate(fp64: bool = True, stream: Optional[int] = None) -> float:
    """rb_fma_rate: measured FMA throughput of the current device in flop/s."""
    out = C.c_double()
    st = lib().rb_fma_rate(1 if fp64 else 0, C.byref(out), stream)
    if st != RB_OK:
        raise RbError(st, "rb_fma_rate failed")
    return out.value


def residual_noalloc(prob, mu, x, stream: Optional[int] = None) -> np.ndarray:
    """rb_residual_noalloc: relative residuals of device vectors x [B][N_dof], no device allocation."""
    p, keep = make_problem(prob)
    mu = _f64(mu).reshape(-1, prob.n_mu)
    out = np.zeros(mu.shape[0])
    st = lib().rb_residual_noalloc(C.byref(p), mu.shape[0], _ptr(mu), _ptr(x), _ptr(out),
                                   C.c_void_p(int(stream) if stream else 0))
    if st != RB_OK:
        raise RbError(st, lib().rb_last_error(None).decode())
    return out


def flatten_params(layers) -> np.ndarray:
    """The flat parameter vector of rb_mlp_create from [(W_1, b_1), (W_2, b_2), (W_3, b_3)],
    W_l [out][in] (concatenation in the header's order)."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64).ravel()])
                           for W, b in layers])


def unflatten_params(flat, sizes):
    """Inverse of flatten_params for layer widths sizes = (n_in, hidden, hidden, n_out)."""
    out, o = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + fi * fo].reshape(fo, fi)
        o += fi * fo
        b = flat[o:o + fo]
        o += fo
        out.append((W.copy(), b.copy()))
    return out


class Mlp:
    """The warm-start network (rb_mlp*): n_in -> hidden -> hidden -> n_out, BF16 weights."""

    def __init__(self, n_in: int, n_log: int, hidden: int, n_out: int, params, max_samples: int):
        flat = _f64(params)
        self.sizes = (n_in, hidden, hidden, n_out)
        self._h = C.c_void_p()
        st = lib().rb_mlp_create(C.byref(self._h), n_in, n_log, hidden, n_out, _ptr(flat), max_samples)
        if st != RB_OK:
            raise RbError(st, lib().rb_last_error(None).decode())
        self.num_params = lib().rb_mlp_num_params(self._h)
        if self.num_params != flat.size:
            expected = self.num_params
            self.close()
            raise ValueError(f"expected {expected} parameters, got {flat.size}")

    @property
    def handle(self):
        return self._h

    def _check(self, st):
        if st != RB_OK:
            raise RbError(st, lib().rb_last_error(None).decode())

    def fit(self, mu, Y, steps: int, lr: float = 3e-3, stream: Optional[int] = None) -> np.ndarray:
        """rb_mlp_fit: Adam steps on the pairs (mu host [S][n_in], Y host or device [S][n_out]);
        returns the loss before each step."""
        mu = _f64(mu)
        Y = _f64(Y) if isinstance(Y, np.ndarray) else Y
        loss = np.zeros(max(steps, 1))
        self._check(lib().rb_mlp_fit(self._h, mu.shape[0], _ptr(mu), _ptr(Y), steps, lr, _ptr(loss),
                                     C.c_void_p(int(stream) if stream else 0)))
        return loss[:steps]

    def gradient(self, mu, Y, stream: Optional[int] = None):
        """rb_mlp_gradient: (loss, flat gradient) of the current parameters."""
        mu = _f64(mu)
        Y = _f64(Y) if isinstance(Y, np.ndarray) else Y
        loss = np.zeros(1)
        grad = np.zeros(self.num_params)
        self._check(lib().rb_mlp_gradient(self._h, mu.shape[0], _ptr(mu), _ptr(Y), _ptr(loss), _ptr(grad),
                                          C.c_void_p(int(stream) if stream else 0)))
        return float(loss[0]), grad

    def predict(self, mu, out=None, stream: Optional[int] = None):
        """rb_mlp_predict: coefficients [B][n_out] (host array unless a device out is given)."""
        mu = _f64(mu).reshape(-1, self.sizes[0])
        if out is None:
            out = np.zeros((mu.shape[0], self.sizes[-1]))
        self._check(lib().rb_mlp_predict(self._h, mu.shape[0], _ptr(mu), _ptr(out),
                                         C.c_void_p(int(stream) if stream else 0)))
        return out

    def get(self):
        """rb_mlp_get: (flat FP32 master parameters, standardisation, Adam steps)."""
        p = np.zeros(self.num_params)
        sc = np.zeros(2 * self.sizes[0] + 2 * self.sizes[-1])
        t = C.c_int()
        self._check(lib().rb_mlp_get(self._h, _ptr(p), _ptr(sc), C.byref(t)))
        return p, sc, t.value

    def close(self) -> None:
        if self._h:
            lib().rb_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcg_ragged(contexts, mus, xs, **kw):
    """rb_pcg_ragged: RBCG on several contexts (one batch each, device x) in one launch
    sequence; returns (status, [stats of each context])."""
    n = len(contexts)
    ctxs = (C.c_void_p * n)(*[c.handle for c in contexts])
    mus = [_f64(m).reshape(-1, c.n_mu) for m, c in zip(mus, contexts)]
    B = (C.c_int * n)(*[m.shape[0] for m in mus])
    mu_p = (C.c_void_p * n)(*[_ptr(m) for m in mus])
    x_p = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    sts = [(RbStats * max(m.shape[0], 1))() for m in mus]
    st_p = (C.c_void_p * n)(*[C.cast(st, C.c_void_p) for st in sts])
    o = make_opts(**kw)
    status = lib().rb_pcg_ragged(C.cast(ctxs, C.c_void_p), n, C.cast(B, C.c_void_p), C.cast(mu_p, C.c_void_p),
                                 C.cast(x_p, C.c_void_p), C.byref(o), C.cast(st_p, C.c_void_p))
    if status not in (RB_OK, RB_ENOCONV, RB_EBREAKDOWN):
        msgs = "; ".join(lib().rb_last_error(c.handle).decode() for c in contexts)
        raise RbError(status, msgs or lib().rb_last_error(None).decode())
    return status, [stats_array(st)[:m.shape[0]] for st, m in zip(sts, mus)]


class Context:
    """An online RB context (rb_ctx*)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle
        n_dof, n, Q, R, n_mu = C.c_longlong(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        lib().rb_info(self._h, C.byref(n_dof), C.byref(n), C.byref(Q), C.byref(R), C.byref(n_mu))
        self.n_dof, self.n, self.Q, self.R, self.n_mu = n_dof.value, n.value, Q.value, R.value, n_mu.value

    # -- creation
    @classmethod
    def _check_create(cls, st, h):
        if st != RB_OK:
            raise RbError(st, lib().rb_last_error(None).decode())
        return cls(h)

    @classmethod
    def from_arrays(cls, prob, W, ANq, fNr, max_batch: int = 1) -> "Context":
        """rb_offline_load_arrays: W [N_dof][n], ANq [Q][n][n], fNr [R][n] (host)."""
        p, keep = make_problem(prob)
        W, ANq, fNr = _f64(W), _f64(ANq), _f64(fNr)
        n = W.shape[1] if W.ndim == 2 else 0
        h = C.c_void_p()
        st = lib().rb_offline_load_arrays(C.byref(h), C.byref(p), n, _ptr(W), _ptr(ANq), _ptr(fNr), max_batch)
        return cls._check_create(st, h)

    @classmethod
    def build(cls, prob, n_max: int, train_mu, max_batch: int = 1, truth_tol: float = 1e-11,
              literal_score: bool = False, **solve_kw) -> "Context":
        """rb_offline_build: greedy basis of size n_max from the training parameters (host)."""
        p, keep = make_problem(prob)
        mu = _f64(train_mu)
        b = RbBuildOpts()
        lib().rb_default_build_opts(C.byref(b))
        b.truth_tol = truth_tol
        b.score = 1 if literal_score else 0
        o = make_opts(**solve_kw)
        h = C.c_void_p()
        st = lib().rb_offline_build(C.byref(h), C.byref(p), n_max, mu.shape[0], _ptr(mu), C.byref(b), C.byref(o),
                                    max_batch)
        return cls._check_create(st, h)

    @classmethod
    def build_multi_fidelity(cls, prob, coarse, n_max: int, train_mu, max_batch: int = 1, truth_tol: float = 1e-11,
                             **solve_kw) -> "Context":
        """rb_offline_build_mf: parameter sample by the greedy on the coarse problem, snapshots on prob."""
        p, keep = make_problem(prob)
        pc, keepc = make_problem(coarse)
        mu = _f64(train_mu)
        b = RbBuildOpts()
        lib().rb_default_build_opts(C.byref(b))
        b.truth_tol = truth_tol
        o = make_opts(**solve_kw)
        h = C.c_void_p()
        st = lib().rb_offline_build_mf(C.byref(h), C.byref(p), C.byref(pc), n_max, mu.shape[0], _ptr(mu), C.byref(b),
                                       C.byref(o), max_batch)
        return cls._check_create(st, h)

    @classmethod
    def load(cls, path: str, max_batch: int = 1) -> "Context":
        h = C.c_void_p()
        st = lib().rb_offline_load(C.byref(h), path.encode(), max_batch)
        return cls._check_create(st, h)

    # -- use
    def _check(self, st):
        if st not in (RB_OK, RB_ENOCONV, RB_EBREAKDOWN):
            raise RbError(st, lib().rb_last_error(self._h).decode())
        return st

    @property
    def handle(self):
        return self._h

    def save(self, path: str) -> None:
        self._check(lib().rb_save(self._h, path.encode()))

    def basis(self):
        n, N = self.n, self.n_dof
        W = np.zeros((N, n))
        ANq = np.zeros((self.Q, n, n))
        fNr = np.zeros((self.R, n))
        Rs = np.zeros((n, n))
        sel = np.zeros(n, dtype=np.int32)
        self._check(lib().rb_get_basis(self._h, _ptr(W), _ptr(ANq), _ptr(fNr), _ptr(Rs), _ptr(sel)))
        return W, ANq, fNr, Rs, sel

    def _run(self, fn, mu, x, kw):
        mu = _f64(mu).reshape(-1, self.n_mu)
        B = mu.shape[0]
        st = (RbStats * max(B, 1))()
        o = make_opts(**kw)
        status = fn(self._h, B, _ptr(mu), _ptr(x), C.byref(o), C.cast(st, C.c_void_p))
        self._check(status)
        return status, stats_array(st)[:B]

    def solve(self, mu, x, **kw):
        """rb_solve (RBI, Alg. 2).  x: [B][N_dof] host or device; returns (status, stats)."""
        return self._run(lib().rb_solve, mu, x, kw)

    def pcg(self, mu, x, **kw):
        """rb_pcg (RBCG, Alg. 3).  x: [B][N_dof] host or device; returns (status, stats)."""
        return self._run(lib().rb_pcg, mu, x, kw)

    def apply(self, mu, x, y, stream: Optional[int] = None) -> None:
        mu = _f64(mu).reshape(-1, self.n_mu)
        self._check(lib().rb_apply(self._h, mu.shape[0], _ptr(mu), _ptr(x), _ptr(y),
                                   C.c_void_p(int(stream) if stream else 0)))

    def products(self, R=None, E=None, engine="auto"):
        """rb_products: (W^T R, W E) for FP32 batches R [B][N_dof] and E [B][n] (host arrays)."""
        R = None if R is None else np.ascontiguousarray(R, dtype=np.float32)
        E = None if E is None else np.ascontiguousarray(E, dtype=np.float32)
        B = (R if R is not None else E).shape[0]
        WtR = None if R is None else np.zeros((B, self.n))
        WE = None if E is None else np.zeros((B, self.n_dof), dtype=np.float32)
        eng = GEMMS[engine] if isinstance(engine, str) else engine
        self._check(lib().rb_products(self._h, B, _ptr(R), _ptr(WtR), _ptr(E), _ptr(WE), eng))
        return WtR, WE

    def precondition(self, mu, r, **kw) -> np.ndarray:
        """rb_precondition: y = RBI(A(mu), r, W, 1) for host arrays r [B][N_dof]
        (float64, or float32 with precision="mixed")."""
        mu = _f64(mu).reshape(-1, self.n_mu)
        mixed = kw.get("precision", "fp64") == "mixed"
        r = np.ascontiguousarray(r, dtype=np.float32 if mixed else np.float64)
        y = np.zeros_like(r)
        o = make_opts(**kw)
        self._check(lib().rb_precondition(self._h, mu.shape[0], _ptr(mu), _ptr(r), _ptr(y), C.byref(o)))
        return y

    def autotune(self, mu, x, **kw) -> dict:
        """rb_autotune: fastest (nu, inner_tol, gemm) on the sample queries; returns the chosen options."""
        mu = _f64(mu).reshape(-1, self.n_mu)
        o = make_opts(**kw)
        r = RbTuneResult()
        self._check(lib().rb_autotune(self._h, mu.shape[0], _ptr(mu), _ptr(x), C.byref(o), C.byref(r)))
        inv = {v: k for k, v in GEMMS.items()}
        return {"nu": r.nu, "inner_tol": r.inner_tol, "gemm": inv.get(r.gemm, r.gemm),
                "ms_per_solve": r.ms_per_solve, "trials": r.trials, "kernels": r.kernels,
                "store": {v: k for k, v in STORES.items()}.get(r.store, r.store),
                "x0": {v: k for k, v in STARTS.items()}.get(r.x0_mode, r.x0_mode)}

    def warm_start(self, mu, x, net: Optional[Mlp] = None, coef=None, stream: Optional[int] = None) -> int:
        """rb_warm_start: x [B][N_dof] (host or device) = W c(mu), c = Galerkin coefficients (net None)
        or the network's prediction; coef [B][n] receives c when given."""
        mu = _f64(mu).reshape(-1, self.n_mu)
        return self._check(lib().rb_warm_start(self._h, net.handle if net is not None else None, mu.shape[0],
                                               _ptr(mu), _ptr(x), _ptr(coef),
                                               C.c_void_p(int(stream) if stream else 0)))

    def error_basis(self, mu, X, m: int, stream: Optional[int] = None):
        """rb_error_basis: POD of the errors x_s - x_hat(mu_s) of S solutions X [S][N_dof] (host or
        device); returns (Z = V^T E [S][m], singular values [m]) and keeps V in the context."""
        mu = _f64(mu).reshape(-1, self.n_mu)
        S = mu.shape[0]
        Z = np.zeros((S, m))
        sig = np.zeros(m)
        self._check(lib().rb_error_basis(self._h, S, _ptr(mu), _ptr(X), m, _ptr(Z), _ptr(sig),
                                         C.c_void_p(int(stream) if stream else 0)))
        return Z, sig

    def error_coefficients(self, mu, X, m: int, Z=None, stream: Optional[int] = None):
        """rb_error_coefficients: V^T (x_b - x_hat(mu_b)) for solutions X [B][N_dof]."""
        mu = _f64(mu).reshape(-1, self.n_mu)
        if Z is None:
            Z = np.zeros((mu.shape[0], m))
        self._check(lib().rb_error_coefficients(self._h, mu.shape[0], _ptr(mu), _ptr(X), _ptr(Z),
                                                C.c_void_p(int(stream) if stream else 0)))
        return Z

    def warm_start_error(self, mu, x, net: Optional[Mlp] = None, z=None, stream: Optional[int] = None) -> int:
        """rb_warm_start_error: x [B][N_dof] = x_hat(mu) + V z, z from the network or given."""
        mu = _f64(mu).reshape(-1, self.n_mu)
        zz = None if z is None else (_f64(z) if isinstance(z, np.ndarray) else z)
        return self._check(lib().rb_warm_start_error(self._h, net.handle if net is not None else None, mu.shape[0],
                                                     _ptr(mu), _ptr(x), _ptr(zz),
                                                     C.c_void_p(int(stream) if stream else 0)))

    def coefficients(self, x, coef=None, stream: Optional[int] = None):
        """rb_coefficients: W^T x_b for x [B][N_dof] (host or device); returns coef (host unless given)."""
        B = x.shape[0]
        if coef is None:
            coef = np.zeros((B, self.n))
        self._check(lib().rb_coefficients(self._h, B, _ptr(x), _ptr(coef), C.c_void_p(int(stream) if stream else 0)))
        return coef

    def debug_wait(self, limit_s: float = 2.0, skip_stage: int = -1) -> None:
        """rb_debug_wait: limit of the kernels' bounded waits and the stage the test hook leaves out."""
        self._check(lib().rb_debug_wait(self._h, limit_s, skip_stage))

    def profile(self, enable: bool) -> None:
        """rb_profile: time every kernel launch with CUDA events (graphs off) while enabled."""
        self._check(lib().rb_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """rb_profile_read: {kernel name: (launches, device ms)}."""
        buf = (RbKernelTime * 32)()
        cnt = C.c_int()
        self._check(lib().rb_profile_read(self._h, buf, 32, C.byref(cnt)))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(min(cnt.value, 32))}

    def close(self) -> None:
        if self._h:
            lib().rb_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
