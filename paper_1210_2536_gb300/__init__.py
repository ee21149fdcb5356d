"""Input-adaptive SpMV for GB300 after SMAT (arXiv 1210.2536): Python binding.

The functions below carry the names of the C ABI in ``include/smat.h`` and do
argument marshalling only; every step of the product runs in libsmat's CUDA
kernels.  PyTorch supplies device memory and streams.  ``SpMatrix`` wraps a
handle for convenience.

The library is built by ``__graft_entry__.build()`` (or
``python -m paper_1210_2536_gb300._build``); importing this package without it
raises, so nothing can silently fall back to another implementation.
"""
from __future__ import annotations

import ctypes
import os
import struct

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsmat.so")

SMAT_OK, SMAT_ERR_INVALID_ARG, SMAT_ERR_INVALID_CSR, SMAT_ERR_ALLOC, SMAT_ERR_CUDA, \
    SMAT_ERR_UNSUPPORTED, SMAT_ERR_MODEL, SMAT_ERR_NOT_CONVERGED = range(8)
SMAT_F64, SMAT_F32, SMAT_BF16 = range(3)
(SMAT_FMT_CSR, SMAT_FMT_ELL, SMAT_FMT_DIA, SMAT_FMT_COO, SMAT_FMT_HYB, SMAT_FMT_SELL, SMAT_FMT_BCSR,
 SMAT_FMT_SPLIT) = range(8)
(SMAT_V_CSR_SCALAR, SMAT_V_CSR_VEC4, SMAT_V_CSR_VEC8, SMAT_V_CSR_VEC32, SMAT_V_CSR_MERGE, SMAT_V_ELL,
 SMAT_V_DIA, SMAT_V_COO) = range(8)
SMAT_NUM_VARIANTS = 8
SMAT_V_CSR_SCALAR_EXACT = 8
SMAT_V_HYB, SMAT_V_SELL, SMAT_V_BCSR, SMAT_V_SPLIT = 9, 10, 11, 12
SMAT_NUM_ALL_VARIANTS = 13
VARIANT_NAMES = ["csr_scalar", "csr_vec4", "csr_vec8", "csr_vec32", "csr_merge", "ell", "dia", "coo",
                 "csr_scalar_exact", "hyb", "sell", "bcsr", "split"]
SMAT_TUNE_LEARNED, SMAT_TUNE_EXHAUSTIVE, SMAT_TUNE_RULES, SMAT_TUNE_FIXED = range(4)
SMAT_BATCH_AUTO, SMAT_BATCH_GRAPH, SMAT_BATCH_PER_MATRIX = range(3)
SMAT_MLP_PARAMS = 5512
DTYPES = {"f64": SMAT_F64, "f32": SMAT_F32, "bf16": SMAT_BF16}


class SmatError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {smat_status_string(status)} (status {status})")


class smat_features_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("m", "n", "nnz", "max_rd", "min_rd", "empty_rows", "ndiags",
                                              "ntdiags")] + \
               [("s2", ctypes.c_uint64)] + \
               [(n, ctypes.c_double) for n in ("aver_rd", "var_rd", "er_dia", "er_ell", "ntdiags_ratio", "r")] + \
               [("r_valid", ctypes.c_int32), ("admissible", ctypes.c_uint32)]


class smat_tune_opts_t(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("fixed_variant", ctypes.c_int32), ("conf_threshold", ctypes.c_float),
                ("fallback_topk", ctypes.c_int32), ("tau_num", ctypes.c_int32), ("tau_den", ctypes.c_int32),
                ("fill_ratio_max", ctypes.c_int32), ("bytes_cap", ctypes.c_double), ("trial_reps", ctypes.c_int32),
                ("trial_warmup", ctypes.c_int32), ("trial_budget_ms", ctypes.c_double),
                ("allowed", ctypes.c_uint32), ("keep_formats", ctypes.c_int32), ("sell_sigma", ctypes.c_int32),
                ("trial_extended", ctypes.c_int32), ("plan_cache", ctypes.c_int32), ("trial_race", ctypes.c_float),
                ("trial_tie", ctypes.c_float)]


class smat_cg_opts_t(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
                ("inner_rtol", ctypes.c_float), ("max_total_inner", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("use_graph", ctypes.c_int32)]


class smat_cg_info_t(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int32), ("inner_total", ctypes.c_int32), ("relres", ctypes.c_double),
                ("seconds", ctypes.c_double), ("converged", ctypes.c_int32)]


class smat_batch_opts_t(ctypes.Structure):
    _fields_ = [("tile_scale", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("trial_reps", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("own_launches", ctypes.c_int32)]


class smat_batch_info_t(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int32), ("tiles", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("tile_scale", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("tuned_ms", ctypes.c_double),
                ("per_matrix", ctypes.c_int32), ("graph_ms", ctypes.c_double), ("per_matrix_ms", ctypes.c_double),
                ("own_launches", ctypes.c_int32)]


_VP, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_SIGS = {
    "smat_tune_opts_default": (None, [ctypes.POINTER(smat_tune_opts_t)]),
    "smat_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "smat_test_fail_alloc_after": (None, [_I32]),
    "smat_test_stall_pipelines": (None, [_I32, _I64]),
    "smat_release_cached_memory": (ctypes.c_int, []),
    "smat_create": (ctypes.c_int, [ctypes.POINTER(_VP), _I64, _I64, _I64, _VP, _VP, _VP, ctypes.c_int]),
    "smat_destroy": (ctypes.c_int, [_VP]),
    "smat_tune": (ctypes.c_int, [_VP, ctypes.POINTER(smat_tune_opts_t), _VP]),
    "smat_spmv": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smat_spmv_variant": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP, _VP, _VP, _VP]),
    "smat_spmv_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smat_spmv_many": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP, _VP]),
    "smat_set_kernel": (ctypes.c_int, [_VP, ctypes.c_int, _I32]),
    "smat_get_kernel": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "smat_spmv_host_async": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smat_spmv_host_pipelined": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smat_variant_bytes": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "smat_spmv_launches": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "smat_get_features": (ctypes.c_int, [_VP, ctypes.POINTER(smat_features_t)]),
    "smat_get_feature_vector": (ctypes.c_int, [_VP, _VP]),
    "smat_get_plan": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "smat_get_plan_source": (ctypes.c_int, [_VP, _VP]),
    "smat_plan_key": (ctypes.c_int, [_VP, _VP, _VP]),
    "smat_plan_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "smat_plan_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "smat_plan_cache_clear": (None, []),
    "smat_plan_cache_size": (_I64, []),
    "smat_get_timings": (ctypes.c_int, [_VP, _VP]),
    "smat_measure_gather_rate": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int32, _VP]),
    "smat_measure_fp64_rate": (ctypes.c_int, [ctypes.c_int32, _VP]),
    "smat_get_wait_timeouts": (ctypes.c_int, [_VP]),
    "smat_convert": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "smat_format_dims": (ctypes.c_int, [_VP, ctypes.c_int, _VP]),
    "smat_export_format": (ctypes.c_int, [_VP, ctypes.c_int, _VP, _VP]),
    "smat_set_model": (ctypes.c_int, [_VP, _VP, _VP]),
    "smat_load_model": (ctypes.c_int, [ctypes.c_char_p]),
    "smat_mlp_forward": (ctypes.c_int, [_VP, _VP, _I32, _VP, _VP]),
    "smat_mlp_work_floats": (_I64, [_I32]),
    "smat_mlp_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, _I32, _VP, _VP, _VP, _VP]),
    "smat_mlp_adam": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I64, _I32, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, _VP]),
    "smat_spmv_csr_merge_noalloc": (ctypes.c_int, [_I64, _I64, _I64, _VP, _VP, _VP, ctypes.c_int, _VP, _VP, _VP,
                                                   _VP, _VP]),
    "smat_batch_opts_default": (None, [ctypes.POINTER(smat_batch_opts_t)]),
    "smat_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), _VP, _I32]),
    "smat_batch_tune": (ctypes.c_int, [_VP, ctypes.POINTER(smat_batch_opts_t), _VP]),
    "smat_batch_spmv": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smat_batch_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(smat_batch_info_t)]),
    "smat_batch_destroy": (ctypes.c_int, [_VP]),
    "smat_segments_create": (ctypes.c_int, [ctypes.POINTER(_VP), _VP, _I32, ctypes.POINTER(smat_tune_opts_t),
                                            _VP]),
    "smat_segments_spmv": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "smat_segments_info": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "smat_segments_destroy": (ctypes.c_int, [_VP]),
    "smat_cg_opts_default": (None, [ctypes.POINTER(smat_cg_opts_t)]),
    "smat_cg_mixed": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.POINTER(smat_cg_opts_t),
                                     ctypes.POINTER(smat_cg_info_t), _VP]),
    "smat_cast_f64_to_f32": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "smat_cast_f64_to_bf16": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
}

_lib = None


def lib():
    """The loaded libsmat (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, where):
    if status != SMAT_OK:
        raise SmatError(status, where)
    return status


def smat_status_string(s: int) -> str:
    try:
        return lib().smat_status_string(int(s)).decode()
    except RuntimeError:
        return f"status {s}"


def smat_tune_opts_default() -> smat_tune_opts_t:
    o = smat_tune_opts_t()
    lib().smat_tune_opts_default(ctypes.byref(o))
    return o


# -- raw entry points: integers are pointers (tensor.data_ptr() / ndarray.ctypes.data) --

def smat_create(m, n, nnz, rowptr_ptr, colidx_ptr, vals_ptr, dtype):
    h = _VP()
    st = lib().smat_create(ctypes.byref(h), m, n, nnz, rowptr_ptr, colidx_ptr, vals_ptr, dtype)
    return st, h.value


def smat_destroy(h):
    return lib().smat_destroy(h)


def smat_tune(h, opts: smat_tune_opts_t | None, stream=0):
    return lib().smat_tune(h, ctypes.byref(opts) if opts is not None else None, stream)


def smat_spmv(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream=0):
    return lib().smat_spmv(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream)


def smat_spmv_variant(h, v, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream=0):
    return lib().smat_spmv_variant(h, v, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream)


def smat_spmv_host(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream=0):
    return lib().smat_spmv_host(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream)


def smat_spmv_host_async(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream=0):
    return lib().smat_spmv_host_async(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream)


def smat_spmv_host_pipelined(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream=0):
    return lib().smat_spmv_host_pipelined(h, alpha_ptr, x_ptr, beta_ptr, y_ptr, stream)


def smat_spmv_launches(h, v) -> int:
    n = ctypes.c_int32()
    _check(lib().smat_spmv_launches(h, v, ctypes.byref(n)), "smat_spmv_launches")
    return n.value


def smat_get_features(h) -> smat_features_t:
    f = smat_features_t()
    _check(lib().smat_get_features(h, ctypes.byref(f)), "smat_get_features")
    return f


def smat_get_feature_vector(h) -> np.ndarray:
    out = np.zeros(12, dtype=np.float32)
    _check(lib().smat_get_feature_vector(h, out.ctypes.data), "smat_get_feature_vector")
    return out


def smat_get_plan(h):
    v, ms, conf, tr = ctypes.c_int32(), ctypes.c_double(), ctypes.c_float(), ctypes.c_int32()
    _check(lib().smat_get_plan(h, ctypes.byref(v), ctypes.byref(ms), ctypes.byref(conf), ctypes.byref(tr)),
           "smat_get_plan")
    return v.value, ms.value, conf.value, tr.value


def smat_get_plan_source(h) -> int:
    c = ctypes.c_int32()
    _check(lib().smat_get_plan_source(h, ctypes.byref(c)), "smat_get_plan_source")
    return c.value


def smat_plan_key(h, stream=0) -> int:
    k = ctypes.c_uint64()
    _check(lib().smat_plan_key(h, ctypes.byref(k), stream), "smat_plan_key")
    return k.value


def plan_cache_save(path):
    """Write the process-wide plan cache to a text file (see smat.h)."""
    _check(lib().smat_plan_cache_save(os.fsencode(path)), "smat_plan_cache_save")


def plan_cache_load(path):
    """Merge a plan-cache file into the process-wide cache."""
    _check(lib().smat_plan_cache_load(os.fsencode(path)), "smat_plan_cache_load")


def plan_cache_clear():
    lib().smat_plan_cache_clear()


def plan_cache_size() -> int:
    return int(lib().smat_plan_cache_size())


def smat_get_timings(h) -> np.ndarray:
    out = np.zeros(SMAT_NUM_ALL_VARIANTS, dtype=np.float32)
    _check(lib().smat_get_timings(h, out.ctypes.data), "smat_get_timings")
    return out


def smat_convert(h, fmt, stream=0):
    return lib().smat_convert(h, fmt, stream)


def smat_measure_gather_rate(n: int, nidx: int, dtype: str = "f64", reps: int = 20) -> float:
    """Random gathers per second this GPU serves from an x of n elements (see smat.h)."""
    r = ctypes.c_double(0.0)
    _check(lib().smat_measure_gather_rate(n, nidx, DTYPES[dtype], reps, ctypes.byref(r)), "smat_measure_gather_rate")
    return float(r.value)


def spmv_many(mats, xs, ys, alphas=None, betas=None, stream=None):
    """Independent products ys[i] = alphas[i]*mats[i]*xs[i] + betas[i]*ys[i],
    each through its plan, side by side on library streams ordered after and
    before `stream` (see smat_spmv_many).  Returns ys."""
    n = len(mats)
    if n == 0:
        return ys
    alphas = [1.0] * n if alphas is None else alphas
    betas = [0.0] * n if betas is None else betas
    scal = [M._scalars(a, b) for M, a, b in zip(mats, alphas, betas)]
    hs = (_VP * n)(*[M.h for M in mats])
    ap = (_VP * n)(*[ctypes.addressof(a) for a, _ in scal])
    bp = (_VP * n)(*[ctypes.addressof(b) for _, b in scal])
    xp = (_VP * n)(*[x.data_ptr() for x in xs])
    yp = (_VP * n)(*[y.data_ptr() for y in ys])
    _check(lib().smat_spmv_many(hs, n, ap, xp, bp, yp, _stream_ptr(stream)), "smat_spmv_many")
    return ys


def smat_measure_fp64_rate(reps: int = 10) -> float:
    """FP64 fused multiply-adds per second this GPU sustains (see smat.h)."""
    r = ctypes.c_double(0.0)
    _check(lib().smat_measure_fp64_rate(reps, ctypes.byref(r)), "smat_measure_fp64_rate")
    return float(r.value)


def smat_get_wait_timeouts() -> int:
    """Bounded waits in the pipelined kernels that ran out so far (0 when all is well)."""
    c = ctypes.c_uint64(0)
    _check(lib().smat_get_wait_timeouts(ctypes.byref(c)), "smat_get_wait_timeouts")
    return int(c.value)


def smat_format_dims(h, fmt):
    d = np.zeros(2, dtype=np.int64)
    st = lib().smat_format_dims(h, fmt, d.ctypes.data)
    return st, int(d[0]), int(d[1])


def smat_export_format(h, fmt, idx_ptr, val_ptr):
    return lib().smat_export_format(h, fmt, idx_ptr, val_ptr)


def smat_set_model(params, mean, std):
    if params is None:
        return lib().smat_set_model(None, None, None)
    p = np.ascontiguousarray(params, dtype=np.float32)
    mu = np.ascontiguousarray(mean, dtype=np.float32)
    sd = np.ascontiguousarray(std, dtype=np.float32)
    assert p.size == SMAT_MLP_PARAMS and mu.size == 12 and sd.size == 12
    return lib().smat_set_model(p.ctypes.data, mu.ctypes.data, sd.ctypes.data)


def smat_load_model(path=None):
    """Load a selector model file; None loads the file SMAT_MODEL_PATH names."""
    return lib().smat_load_model(None if path is None else os.fsencode(path))


def smat_mlp_forward(params_ptr, x_ptr, B, logits_ptr, stream=0):
    return lib().smat_mlp_forward(params_ptr, x_ptr, B, logits_ptr, stream)


def smat_mlp_work_floats(B) -> int:
    return int(lib().smat_mlp_work_floats(B))


def smat_mlp_loss_grad(params_ptr, x_ptr, t_ptr, B, grad_ptr, loss_ptr, work_ptr, stream=0):
    return lib().smat_mlp_loss_grad(params_ptr, x_ptr, t_ptr, B, grad_ptr, loss_ptr, work_ptr, stream)


def smat_mlp_adam(p_ptr, g_ptr, m_ptr, v_ptr, n, t, lr, b1, b2, eps, stream=0):
    return lib().smat_mlp_adam(p_ptr, g_ptr, m_ptr, v_ptr, n, t, lr, b1, b2, eps, stream)


def smat_spmv_csr_merge_noalloc(m, n, nnz, rowptr_ptr, colidx_ptr, vals_ptr, dtype, alpha_ptr, x_ptr, beta_ptr,
                                y_ptr, stream=0):
    """Merge-path CSR product with no allocation (see include/smat.h)."""
    return lib().smat_spmv_csr_merge_noalloc(m, n, nnz, rowptr_ptr, colidx_ptr, vals_ptr, dtype, alpha_ptr, x_ptr,
                                             beta_ptr, y_ptr, stream)


def smat_batch_opts_default() -> smat_batch_opts_t:
    o = smat_batch_opts_t()
    lib().smat_batch_opts_default(ctypes.byref(o))
    return o


class Batch:
    """Several SpMatrix handles multiplied in one persistent launch (graph)."""

    def __init__(self, mats):
        self.mats = list(mats)
        arr = (_VP * len(self.mats))(*[m.h for m in self.mats])
        b = _VP()
        _check(lib().smat_batch_create(ctypes.byref(b), arr, len(self.mats)), "smat_batch_create")
        self.b = b.value
        self.dtype = self.mats[0].dtype

    def tune(self, stream=None, **opts):
        o = smat_batch_opts_default()
        for k, v in opts.items():
            setattr(o, k, v)
        _check(lib().smat_batch_tune(self.b, ctypes.byref(o), _stream_ptr(stream)), "smat_batch_tune")
        return self

    def spmv(self, xs, ys, alphas=None, betas=None, stream=None):
        n = len(self.mats)
        ct = ctypes.c_double if self.dtype == "f64" else ctypes.c_float
        a = (ct * n)(*(alphas if alphas is not None else [1.0] * n))
        b = (ct * n)(*(betas if betas is not None else [0.0] * n))
        xp = (_VP * n)(*[x.data_ptr() for x in xs])
        yp = (_VP * n)(*[y.data_ptr() for y in ys])
        _check(lib().smat_batch_spmv(self.b, a, xp, b, yp, _stream_ptr(stream)), "smat_batch_spmv")
        return ys

    def info(self) -> dict:
        i = smat_batch_info_t()
        _check(lib().smat_batch_get_info(self.b, ctypes.byref(i)), "smat_batch_get_info")
        return {n: getattr(i, n) for n, _ in smat_batch_info_t._fields_}

    def close(self):
        if getattr(self, "b", None):
            lib().smat_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Segments:
    """Per-segment plans of one SpMatrix (Sec. 6): nonzero-balanced row segments,
    each tuned to its own format, run as one batched launch."""

    def __init__(self, M: "SpMatrix", nseg: int, mode="exhaustive", stream=None, **kw):
        o = smat_tune_opts_default()
        o.mode = {"learned": SMAT_TUNE_LEARNED, "exhaustive": SMAT_TUNE_EXHAUSTIVE, "rules": SMAT_TUNE_RULES}[mode]
        for k, v in kw.items():
            setattr(o, k, v)
        s = _VP()
        _check(lib().smat_segments_create(ctypes.byref(s), M.h, int(nseg), ctypes.byref(o), _stream_ptr(stream)),
               "smat_segments_create")
        self.s, self.M = s.value, M

    def info(self):
        n = ctypes.c_int32()
        lib().smat_segments_info(self.s, ctypes.byref(n), None, None)
        v = np.zeros(n.value, np.int32)
        r = np.zeros(n.value + 1, np.int64)
        _check(lib().smat_segments_info(self.s, ctypes.byref(n), v.ctypes.data, r.ctypes.data), "smat_segments_info")
        return {"variants": [VARIANT_NAMES[i] for i in v], "row_starts": r.tolist()}

    def spmv(self, x, y=None, alpha=1.0, beta=0.0, stream=None):
        import torch
        if y is None:
            y = torch.empty(self.M.m, dtype=self.M.compute_dtype, device=x.device)
        a, b = self.M._scalars(alpha, beta)
        _check(lib().smat_segments_spmv(self.s, ctypes.addressof(a), x.data_ptr(), ctypes.addressof(b), y.data_ptr(),
                                        _stream_ptr(stream)), "smat_segments_spmv")
        return y

    def close(self):
        if getattr(self, "s", None):
            lib().smat_segments_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def smat_cg_opts_default() -> smat_cg_opts_t:
    o = smat_cg_opts_t()
    lib().smat_cg_opts_default(ctypes.byref(o))
    return o


def smat_cg_mixed(a64, a32, b_ptr, x_ptr, opts: smat_cg_opts_t | None = None, stream=0):
    """Returns (status, smat_cg_info_t)."""
    info = smat_cg_info_t()
    st = lib().smat_cg_mixed(a64, a32, b_ptr, x_ptr, ctypes.byref(opts) if opts is not None else None,
                             ctypes.byref(info), stream)
    return st, info


def cg_mixed(A64: "SpMatrix", A32: "SpMatrix", b, x, stream=None, **opts):
    """Mixed-precision CG on device FP64 tensors b and x (x: initial guess, overwritten)."""
    o = smat_cg_opts_default()
    for k, v in opts.items():
        setattr(o, k, v)
    st, info = smat_cg_mixed(A64.h, A32.h, b.data_ptr(), x.data_ptr(), o, _stream_ptr(stream))
    if st not in (SMAT_OK, SMAT_ERR_NOT_CONVERGED):
        _check(st, "smat_cg_mixed")
    return {"status": st, "outer": info.outer, "inner_total": info.inner_total, "relres": info.relres,
            "seconds": info.seconds, "converged": bool(info.converged)}


def smat_cast_f64_to_f32(in_ptr, out_ptr, n, stream=0):
    return lib().smat_cast_f64_to_f32(in_ptr, out_ptr, n, stream)


def smat_cast_f64_to_bf16(in_ptr, out_ptr, n, stream=0):
    return lib().smat_cast_f64_to_bf16(in_ptr, out_ptr, n, stream)


def write_model(path, params, mean, std):
    """Model file read by smat_load_model: b"SMATMLP1", int32 1, mean[12], std[12], params[5512] (FP32 LE)."""
    with open(path, "wb") as f:
        f.write(b"SMATMLP1")
        f.write(struct.pack("<i", 1))
        for a in (mean, std, params):
            f.write(np.ascontiguousarray(a, dtype="<f4").tobytes())


def read_model(path):
    """(params[5512], mean[12], std[12]) from a model file (see write_model)."""
    with open(path, "rb") as f:
        assert f.read(8) == b"SMATMLP1" and struct.unpack("<i", f.read(4))[0] == 1
        a = np.frombuffer(f.read(), dtype="<f4")
    assert a.size == 24 + SMAT_MLP_PARAMS
    return a[24:].copy(), a[:12].copy(), a[12:24].copy()


MODEL_PATH = os.path.join(_PKG, "selector_mlp.bin")
DATASET_PATH = os.path.join(_PKG, "selector_dataset.jsonl")


# ---------------------------------------------------------------------------
# Convenience wrapper over torch tensors (marshalling only)
# ---------------------------------------------------------------------------

def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class SpMatrix:
    """A CSR matrix handed to libsmat (Sec. 3: the unified CSR interface).

    ``rowptr``/``colidx``/``vals`` may be torch tensors (CPU or CUDA) or numpy
    arrays; they are copied into library-owned device memory.  ``dtype`` is the
    value storage: "f64", "f32" or "bf16" (bf16 values are passed as 16-bit
    patterns in a uint16/int16 array or as a torch.bfloat16 tensor)."""

    def __init__(self, m, n, rowptr, colidx, vals, dtype="f64"):
        self.m, self.n = int(m), int(n)
        self.dtype = dtype
        self._keep = [rowptr, colidx, vals]
        rp, ci, vv = (_ptr(a) for a in (rowptr, colidx, vals))
        self.nnz = int(_len(colidx))
        st, h = smat_create(self.m, self.n, self.nnz, rp, ci, vv, DTYPES[dtype])
        self._keep = None
        _check(st, "smat_create")
        self.h = h

    @property
    def compute_dtype(self):
        import torch
        return torch.float64 if self.dtype == "f64" else torch.float32

    def close(self):
        if getattr(self, "h", None):
            smat_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, mode="exhaustive", variant=None, stream=None, **kw):
        o = smat_tune_opts_default()
        o.mode = {"learned": SMAT_TUNE_LEARNED, "exhaustive": SMAT_TUNE_EXHAUSTIVE, "rules": SMAT_TUNE_RULES,
                  "fixed": SMAT_TUNE_FIXED}[mode]
        if variant is not None:
            o.fixed_variant = int(variant)
        for k, v in kw.items():
            setattr(o, k, v)
        _check(smat_tune(self.h, o, _stream_ptr(stream)), "smat_tune")
        return self

    def _scalars(self, alpha, beta):
        if self.dtype == "f64":
            a, b = ctypes.c_double(alpha), ctypes.c_double(beta)
        else:
            a, b = ctypes.c_float(alpha), ctypes.c_float(beta)
        return a, b

    def spmv(self, x, y=None, alpha=1.0, beta=0.0, variant=None, stream=None):
        """y = alpha*A*x + beta*y on the device; returns y (a CUDA tensor)."""
        import torch
        if y is None:
            y = torch.empty(self.m, dtype=self.compute_dtype, device=x.device)
        assert x.dtype == self.compute_dtype and y.dtype == self.compute_dtype and x.is_cuda and y.is_cuda
        assert x.is_contiguous() and y.is_contiguous()
        a, b = self._scalars(alpha, beta)
        s = _stream_ptr(stream)
        if variant is None:
            st = smat_spmv(self.h, ctypes.addressof(a), x.data_ptr(), ctypes.addressof(b), y.data_ptr(), s)
        else:
            st = smat_spmv_variant(self.h, int(variant), ctypes.addressof(a), x.data_ptr(), ctypes.addressof(b),
                                   y.data_ptr(), s)
        _check(st, "smat_spmv")
        return y

    def spmv_host(self, x, y, alpha=1.0, beta=0.0, stream=None):
        """Same product with host (CPU tensor / ndarray) x and y; y holds the result on return."""
        a, b = self._scalars(alpha, beta)
        _check(smat_spmv_host(self.h, ctypes.addressof(a), _ptr(x), ctypes.addressof(b), _ptr(y),
                              _stream_ptr(stream)), "smat_spmv_host")
        return y

    def spmv_host_async(self, x, y, alpha=1.0, beta=0.0, stream=None):
        """Enqueue the host-buffer product on `stream` without waiting (pinned x, y)."""
        a, b = self._scalars(alpha, beta)
        _check(smat_spmv_host_async(self.h, ctypes.addressof(a), _ptr(x), ctypes.addressof(b), _ptr(y),
                                    _stream_ptr(stream)), "smat_spmv_host_async")
        return y

    def variant_bytes(self, variant) -> float:
        """Matrix bytes one product through `variant` reads (smat_variant_bytes)."""
        b = ctypes.c_double()
        _check(lib().smat_variant_bytes(self.h, int(variant), ctypes.byref(b)), "smat_variant_bytes")
        return b.value

    def spmv_host_pipelined(self, x, y, alpha=1.0, beta=0.0, stream=None):
        """The host-buffer product on the handle's own streams and alternating
        staging sets (smat_spmv_host_pipelined); y is valid once `stream` has
        finished.  x (and y when beta != 0) must hold their values now."""
        a, b = self._scalars(alpha, beta)
        _check(smat_spmv_host_pipelined(self.h, ctypes.addressof(a), _ptr(x), ctypes.addressof(b), _ptr(y),
                                        _stream_ptr(stream)), "smat_spmv_host_pipelined")
        return y

    def features(self) -> dict:
        """Feature parameters, plus the sizes of the built HYB / SELL / BCSR /
        SPLIT formats (hyb_K, hyb_ncoo, sell_ns, sell_slots, bcsr_b, bcsr_nb,
        split_nc, split_ns)."""
        f = smat_get_features(self.h)
        out = {n: getattr(f, n) for n, _ in smat_features_t._fields_}
        out.update(self.layout())
        return out

    def layout(self) -> dict:
        out = {}
        for fmt, keys in ((SMAT_FMT_HYB, ("hyb_K", "hyb_ncoo")), (SMAT_FMT_SELL, ("sell_ns", "sell_slots")),
                          (SMAT_FMT_BCSR, ("bcsr_b", "bcsr_nb")), (SMAT_FMT_SPLIT, ("split_nc", "split_ns"))):
            st, d0, d1 = smat_format_dims(self.h, fmt)
            if st == SMAT_OK:
                out[keys[0]], out[keys[1]] = d0, d1
        return out

    def feature_vector(self) -> np.ndarray:
        return smat_get_feature_vector(self.h)

    def plan(self) -> dict:
        v, ms, conf, tr = smat_get_plan(self.h)
        return {"variant": v, "name": VARIANT_NAMES[v], "tune_ms": ms, "confidence": conf, "trialled": tr,
                "from_cache": smat_get_plan_source(self.h)}

    def plan_key(self, stream=None) -> int:
        """64-bit key of this matrix's structure in the plan cache."""
        return smat_plan_key(self.h, _stream_ptr(stream))

    def launches(self, variant=None) -> int:
        """Kernel launches of one product (through the plan, or `variant`)."""
        return smat_spmv_launches(self.h, self.plan()["variant"] if variant is None else int(variant))

    def timings(self) -> np.ndarray:
        return smat_get_timings(self.h)

    def kernel(self, variant) -> int:
        """The kernel behind ``variant`` (DIA: 0 direct, 1 staged; ELL: 0
        consecutive rows, 1 lane-striped); its format must be built."""
        k = ctypes.c_int32(0)
        _check(lib().smat_get_kernel(self.h, int(variant), ctypes.byref(k)), "smat_get_kernel")
        return int(k.value)

    def set_kernel(self, variant, kernel: int):
        """Pin the kernel behind ``variant`` for later products (see kernel())."""
        _check(lib().smat_set_kernel(self.h, int(variant), int(kernel)), "smat_set_kernel")

    def convert(self, fmt, stream=None):
        _check(smat_convert(self.h, fmt, _stream_ptr(stream)), "smat_convert")

    def export(self, fmt):
        """Copy a built format to host numpy arrays (see smat_format_dims)."""
        st, d0, d1 = smat_format_dims(self.h, fmt)
        _check(st, "smat_format_dims")
        vdt = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16}[self.dtype]
        P = (self.m + 31) // 32 * 32
        if fmt == SMAT_FMT_ELL:
            idx, val = np.empty(d0 * d1, np.int32), np.empty(d0 * d1, vdt)
        elif fmt == SMAT_FMT_DIA:
            idx, val = np.empty(d0, np.int32), np.empty(d0 * d1, vdt)
        elif fmt == SMAT_FMT_HYB:
            idx, val = np.empty(d0 * P + 2 * d1, np.int32), np.empty(d0 * P + d1, vdt)
        elif fmt == SMAT_FMT_SELL:
            idx, val = np.empty(33 * d0 + d1, np.int32), np.empty(d1, vdt)
        elif fmt == SMAT_FMT_BCSR:
            mb = (self.m + d0 - 1) // d0
            idx, val = np.empty(mb + 1 + d1, np.int32), np.empty(d1 * d0 * d0, vdt)
        elif fmt == SMAT_FMT_SPLIT:
            idx, val = np.empty(3 * d0 + 2 * d1, np.int32), np.empty(d1, vdt)
        else:
            idx, val = np.empty(d0, np.int32), None
        _check(smat_export_format(self.h, fmt, idx.ctypes.data, None if val is None else val.ctypes.data),
               "smat_export_format")
        return idx, val, d0, d1

    def export_parts(self, fmt) -> dict:
        """A built HYB / SELL / BCSR / SPLIT format split into its named arrays."""
        idx, val, d0, d1 = self.export(fmt)
        if fmt == SMAT_FMT_HYB:
            ne = d0 * ((self.m + 31) // 32 * 32)
            return {"K": d0, "ell_col": idx[:ne], "ell_val": val[:ne], "coo_row": idx[ne:ne + d1],
                    "coo_col": idx[ne + d1:], "coo_val": val[ne:]}
        if fmt == SMAT_FMT_SELL:
            return {"perm": idx[:32 * d0], "width": idx[32 * d0:33 * d0], "col": idx[33 * d0:], "val": val}
        if fmt == SMAT_FMT_BCSR:
            mb = (self.m + d0 - 1) // d0
            return {"b": d0, "browptr": idx[:mb + 1], "bcol": idx[mb + 1:], "val": val}
        if fmt == SMAT_FMT_SPLIT:
            return {"crow": idx[:d0], "cstart": idx[d0:2 * d0], "cend": idx[2 * d0:3 * d0],
                    "srow": idx[3 * d0:3 * d0 + d1], "scol": idx[3 * d0 + d1:], "sval": val}
        raise ValueError(fmt)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr() if a.numel() else None
    a = np.asarray(a)
    assert a.flags.c_contiguous
    return a.ctypes.data if a.size else None


def _len(a):
    return a.numel() if hasattr(a, "numel") else np.asarray(a).size
