"""ctypes binding of libtsx.so (include/tsx.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts Python
and numpy arguments into the C structs, calls the entry points of the same
names, and copies result views into numpy arrays.  If the library is
missing or cannot be loaded, the calls raise -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtsx.so")

TSX_OK, TSX_EINVAL, TSX_ENOMEM, TSX_ECUDA, TSX_ETIMEDOUT = 0, -1, -2, -3, -4
TSX_EBUSY, TSX_EUNSUPPORTED, TSX_ENOTFOUND, TSX_EAGAIN = -5, -6, -7, -8
TSX_CODE_QC, TSX_CODE_CSR = 0, 1
TSX_DEC_NMS_I16, TSX_DEC_NMS_I8, TSX_DEC_SPA_F32 = 0, 1, 2
DECODERS = {"nms16": TSX_DEC_NMS_I16, "nms8": TSX_DEC_NMS_I8, "spa": TSX_DEC_SPA_F32}

I32 = C.POINTER(C.c_int32)
I64 = C.POINTER(C.c_int64)
F32 = C.POINTER(C.c_float)


class TsxError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {strerror(status)} ({status})")
        self.status = status


class CodeDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("m_b", C.c_int32), ("n_b", C.c_int32), ("Z", C.c_int32),
                ("shifts", I32), ("n", C.c_int32), ("m", C.c_int32), ("row_ptr", I32), ("col_idx", I32)]


class CodeInfo(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32), ("m", C.c_int32), ("E", C.c_int32),
                ("Z", C.c_int32), ("n_b", C.c_int32), ("m_b", C.c_int32), ("dv_max", C.c_int32),
                ("dc_max", C.c_int32), ("girth", C.c_int32), ("n_rep", C.c_int32),
                ("ball_total", C.c_int64), ("device_bytes", C.c_int64)]


class EnumParams(C.Structure):
    _fields_ = [("decoder", C.c_int32), ("K", C.c_int32), ("base_llr", C.c_int32), ("sat", C.c_int32),
                ("alpha_num", C.c_int32), ("alpha_shift", C.c_int32), ("amp_steps", C.c_int32),
                ("spa_clip", C.c_float), ("spa_amax", C.c_float), ("max_size", C.c_int32),
                ("cycle_len", C.c_int32), ("record_candidates", C.c_int32), ("cand_begin", C.c_int64),
                ("cand_end", C.c_int64), ("warps_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("kernel", C.c_int32), ("list_mode", C.c_int32), ("kstart", C.c_int32), ("budget_wref", C.c_int32),
                ("budget_kmin", C.c_int32)]


class EnumStats(C.Structure):
    _fields_ = [("n_cand", C.c_int64), ("n_cand_total", C.c_int64), ("n_ts", C.c_int64),
                ("decodes", C.c_int64), ("iterations", C.c_int64), ("edge_updates", C.c_int64),
                ("acyclic", C.c_int64), ("ms_total", C.c_double), ("ms_candidates", C.c_double),
                ("ms_decode", C.c_double), ("ms_sieve", C.c_double), ("converged", C.c_int64),
                ("converged_iterations", C.c_int64), ("list_kstart", C.c_int64), ("list_patterns", C.c_int64),
                ("list_iterations", C.c_int64)]


class IsParams(C.Structure):
    _fields_ = [("ebn0_db", C.c_double), ("rate", C.c_double), ("mu", C.c_double), ("n_samples", C.c_int64),
                ("job_key", C.c_uint64), ("sample_begin", C.c_int64), ("K", C.c_int32), ("sat", C.c_int32),
                ("alpha_num", C.c_int32), ("alpha_shift", C.c_int32)]


class IsResult(C.Structure):
    _fields_ = [("fer", C.c_double), ("var", C.c_double), ("sum_w", C.c_double), ("sum_w2", C.c_double),
                ("n_samples", C.c_int64), ("n_fail", C.c_int64), ("decodes", C.c_int64),
                ("iterations", C.c_int64), ("edge_updates", C.c_int64), ("ms", C.c_double)]


class ServerParams(C.Structure):
    _fields_ = [("max_jobs", C.c_int32), ("serial", C.c_int32), ("device", C.c_int32), ("hbm_bytes", C.c_int64),
                ("chunk_candidates", C.c_int64), ("chunk_samples", C.c_int64), ("small_work", C.c_double),
                ("backfill_ms", C.c_double), ("max_large", C.c_int32)]


class Job(C.Structure):
    _fields_ = [("kind", C.c_int32), ("code", C.c_void_p), ("enum_params", EnumParams), ("is_params", IsParams),
                ("ts_vars", C.c_void_p), ("a", C.c_int32)]


class JobResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("high_priority", C.c_int32), ("grid_sms", C.c_int32),
                ("device_bytes", C.c_int64), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("latency_ms", C.c_double), ("enum_stats", EnumStats), ("is_result", IsResult)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("done", C.c_int64), ("failed", C.c_int64), ("running", C.c_int64),
                ("queued", C.c_int64), ("p50_ms", C.c_double), ("p90_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("mean_ms", C.c_double), ("mean_queue_ms", C.c_double),
                ("makespan_ms", C.c_double), ("edge_updates", C.c_int64), ("decodes", C.c_int64),
                ("edge_updates_per_s", C.c_double), ("hbm_peak_bytes", C.c_int64), ("max_concurrent", C.c_int32)]


class Peaks(C.Structure):
    _fields_ = [("num_sms", C.c_int32), ("int32_ops_per_clk_sm", C.c_double), ("u16x2_ops_per_clk_sm", C.c_double),
                ("smem_bytes_per_clk_sm", C.c_double), ("sfu_ops_per_clk_sm", C.c_double),
                ("fp32_fma_per_clk_sm", C.c_double), ("imad_ops_per_clk_sm", C.c_double)]


class LnmsParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("llr_bits", C.c_int32), ("c2v_bits", C.c_int32), ("v2c_bits", C.c_int32),
                ("alpha_num", C.c_int32), ("alpha_shift", C.c_int32)]


class SimParams(C.Structure):
    _fields_ = [("ebn0_db", C.c_double), ("rate", C.c_double), ("llr_scale", C.c_double), ("max_frames", C.c_int64),
                ("max_errors", C.c_int64), ("job_key", C.c_uint64), ("frame_begin", C.c_int64)]


class SimResult(C.Structure):
    _fields_ = [("frames", C.c_int64), ("frame_errors", C.c_int64), ("bit_errors", C.c_int64), ("fer", C.c_double),
                ("ber", C.c_double), ("iterations", C.c_int64), ("edge_updates", C.c_int64), ("ms", C.c_double)]


class UnionResult(C.Structure):
    _fields_ = [("fer_ub", C.c_double), ("var_ub", C.c_double), ("n_sets", C.c_int64), ("samples", C.c_int64),
                ("n_fail", C.c_int64), ("edge_updates", C.c_int64), ("ms", C.c_double)]


class EmdSpectrum(C.Structure):
    _fields_ = [("lmax", C.c_int32), ("walks", C.c_int64 * 7), ("count2l", (C.c_int64 * 128) * 7), ("ms", C.c_double)]


TSX_JOB_ENUMERATE, TSX_JOB_IS_FER = 0, 1
TSX_ENOTFOUND, TSX_EAGAIN = -7, -8


class TsView(C.Structure):
    _fields_ = [("stats", EnumStats), ("n_ts", C.c_int64), ("a", I32), ("b", I32), ("orbit", I32),
                ("count", I32), ("thr", I32), ("flags", I32), ("thr_f", F32), ("var_off", I64),
                ("vars", I32), ("n_cand", C.c_int64), ("cand_vars", I32), ("cand_thr", I32),
                ("cand_ts", I32), ("cand_flags", I32), ("cand_decodes", I32), ("cand_iters", I32),
                ("cand_thr_f", F32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libtsx.so (build it first with paper_2208_05795_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libtsx.so not built ({LIB_PATH}); run paper_2208_05795_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            vp = C.c_void_p
            L.tsx_strerror.restype = C.c_char_p
            L.tsx_strerror.argtypes = [C.c_int]
            L.load_code.argtypes = [C.POINTER(CodeDesc), vp, C.POINTER(vp)]
            L.load_code.restype = C.c_int
            L.free_code.argtypes = [vp]
            L.free_code.restype = None
            L.code_info.argtypes = [vp, C.POINTER(CodeInfo)]
            L.code_info.restype = C.c_int
            L.enum_params_default.argtypes = [C.POINTER(EnumParams)]
            L.enum_params_default.restype = None
            L.enumerate_ts.argtypes = [vp, C.POINTER(EnumParams), vp, C.POINTER(vp)]
            L.enumerate_ts.restype = C.c_int
            L.ts_list_view.argtypes = [vp, C.POINTER(TsView)]
            L.ts_list_view.restype = C.c_int
            L.ts_list_stats.argtypes = [vp, C.POINTER(EnumStats)]
            L.ts_list_stats.restype = C.c_int
            L.free_ts_list.argtypes = [vp]
            L.free_ts_list.restype = None
            L.is_params_default.argtypes = [C.POINTER(IsParams)]
            L.is_params_default.restype = None
            L.is_fer_estimate.argtypes = [vp, vp, C.c_int32, C.POINTER(IsParams), vp, C.POINTER(IsResult), vp, vp]
            L.is_fer_estimate.restype = C.c_int
            L.decode_thresholds_noalloc.argtypes = [vp, C.POINTER(EnumParams), vp, C.c_int64, vp, vp, vp, vp, vp]
            L.decode_thresholds_noalloc.restype = C.c_int
            L.tune_tile.argtypes = [vp, C.POINTER(EnumParams), vp, C.POINTER(EnumParams), C.POINTER(C.c_float)]
            L.tune_tile.restype = C.c_int
            L.batch_create.argtypes = [C.POINTER(vp), C.POINTER(EnumParams), C.c_int32, vp, C.POINTER(vp)]
            L.batch_create.restype = C.c_int
            L.batch_run.argtypes = [vp, vp]
            L.batch_run.restype = C.c_int
            L.batch_size.argtypes = [vp]
            L.batch_size.restype = C.c_int
            L.batch_multi_launch.argtypes = [vp]
            L.batch_multi_launch.restype = C.c_int
            L.batch_decode_launches.argtypes = [vp]
            L.batch_decode_launches.restype = C.c_int
            L.batch_view.argtypes = [vp, C.c_int32, C.POINTER(TsView)]
            L.batch_view.restype = C.c_int
            L.batch_stats.argtypes = [vp, C.POINTER(EnumStats)]
            L.batch_stats.restype = C.c_int
            L.batch_free.argtypes = [vp]
            L.batch_free.restype = None
            L.server_params_default.argtypes = [C.POINTER(ServerParams)]
            L.server_params_default.restype = None
            L.server_create.argtypes = [C.POINTER(ServerParams), C.POINTER(vp)]
            L.server_create.restype = C.c_int
            L.server_submit.argtypes = [vp, C.POINTER(Job), C.POINTER(C.c_uint64)]
            L.server_submit.restype = C.c_int
            L.server_poll.argtypes = [vp, C.c_uint64, C.POINTER(JobResult)]
            L.server_poll.restype = C.c_int
            L.server_wait.argtypes = [vp, C.c_uint64, C.c_double, C.POINTER(JobResult)]
            L.server_wait.restype = C.c_int
            L.server_job_view.argtypes = [vp, C.c_uint64, C.POINTER(TsView)]
            L.server_job_view.restype = C.c_int
            L.server_release.argtypes = [vp, C.c_uint64]
            L.server_release.restype = C.c_int
            L.server_drain.argtypes = [vp]
            L.server_drain.restype = C.c_int
            L.server_stats.argtypes = [vp, C.POINTER(ServerStats)]
            L.server_stats.restype = C.c_int
            L.server_reset_stats.argtypes = [vp]
            L.server_reset_stats.restype = None
            L.server_destroy.argtypes = [vp]
            L.server_destroy.restype = None
            L.cycle_counts.argtypes = [vp, vp, vp]
            L.cycle_counts.restype = C.c_int
            L.emd_spectrum.argtypes = [vp, C.c_int32, vp, C.POINTER(EmdSpectrum)]
            L.emd_spectrum.restype = C.c_int
            L.lnms_params_default.argtypes = [C.POINTER(LnmsParams)]
            L.lnms_params_default.restype = None
            L.sim_params_default.argtypes = [C.POINTER(SimParams)]
            L.sim_params_default.restype = None
            L.lnms_decode.argtypes = [vp, C.POINTER(LnmsParams), vp, C.c_int64, vp, vp, vp, vp]
            L.lnms_decode.restype = C.c_int
            L.lnms_simulate.argtypes = [vp, C.POINTER(LnmsParams), C.POINTER(SimParams), vp, C.POINTER(SimResult), vp]
            L.lnms_simulate.restype = C.c_int
            L.union_bound_fer.argtypes = [vp, C.c_int64, vp, vp, vp, C.POINTER(IsParams), vp, C.POINTER(UnionResult),
                                          vp]
            L.union_bound_fer.restype = C.c_int
            L.measure_peaks.argtypes = [C.POINTER(Peaks), vp]
            L.measure_peaks.restype = C.c_int
            _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().tsx_strerror(int(status)).decode()


def _check(status: int, what: str):
    if status != TSX_OK:
        raise TsxError(status, what)


def _stream_handle(stream):
    """A cudaStream_t as an integer: an int, a torch stream, or None (the
    current torch stream when torch has CUDA, else the legacy default)."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# ---------------------------------------------------------------------------
# the entry points, same names as the C ABI
# ---------------------------------------------------------------------------
class Code:
    """A loaded code (device-resident tables); frees itself on deletion."""

    def __init__(self, handle, info: CodeInfo):
        self.h = handle
        self.info = {k: getattr(info, k) for k, _ in CodeInfo._fields_}

    def __del__(self):
        if getattr(self, "h", None):
            lib().free_code(self.h)
            self.h = None


def load_code(code, stream=None) -> Code:
    """load_code(): `code` has the fields of synth.Code (kind, Z, shifts, n,
    m, row_ptr, col_idx)."""
    d = CodeDesc()
    keep = []
    if code.kind == "qc":
        s = _i32(code.shifts)
        keep.append(s)
        d.kind, d.m_b, d.n_b, d.Z = TSX_CODE_QC, s.shape[0], s.shape[1], int(code.Z)
        d.shifts = s.ctypes.data_as(I32)
    else:
        rp, ci = _i32(code.row_ptr), _i32(code.col_idx)
        keep += [rp, ci]
        d.kind, d.n, d.m = TSX_CODE_CSR, int(code.n), int(code.m)
        d.row_ptr, d.col_idx = rp.ctypes.data_as(I32), ci.ctypes.data_as(I32)
    h = C.c_void_p()
    _check(lib().load_code(C.byref(d), _stream_handle(stream), C.byref(h)), "load_code")
    info = CodeInfo()
    _check(lib().code_info(h, C.byref(info)), "code_info")
    return Code(h, info)


def free_code(code: Code):
    if code.h:
        lib().free_code(code.h)
        code.h = None


def code_info(code: Code) -> dict:
    return dict(code.info)


def enum_params_default() -> EnumParams:
    p = EnumParams()
    lib().enum_params_default(C.byref(p))
    return p


def make_params(**kw) -> EnumParams:
    p = enum_params_default()
    for k, v in kw.items():
        if k == "decoder" and isinstance(v, str):
            v = DECODERS[v]
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


class TsList:
    """Results of one enumerate_ts call (device-resident until viewed)."""

    def __init__(self, handle, code: Code):
        self.h = handle
        self.code = code  # keeps the code alive

    def __del__(self):
        if getattr(self, "h", None):
            lib().free_ts_list(self.h)
            self.h = None


def enumerate_ts(code: Code, params=None, stream=None, **kw) -> TsList:
    p = params if isinstance(params, EnumParams) else make_params(**(params or {}), **kw)
    h = C.c_void_p()
    _check(lib().enumerate_ts(code.h, C.byref(p), _stream_handle(stream), C.byref(h)), "enumerate_ts")
    return TsList(h, code)


def _arr(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def ts_list_view(lst: TsList, check: bool = True, keys: bool = True) -> dict:
    """Synchronizes, copies the results out; returns numpy arrays:
    per TS: a, b, orbit, count, thr, thr_f, flags, the canonical keys as
    key_vars (concatenated) with key_off [n_ts + 1], and with keys=True also
    keys (a list of tuples, built on the host); per candidate: cand_vars
    [N,4], cand_thr, cand_thr_f, cand_ts, cand_flags, cand_decodes,
    cand_iters; and stats."""
    v = TsView()
    st = lib().ts_list_view(lst.h, C.byref(v))
    if check:
        _check(st, "ts_list_view")
    return _view_dict(v, st, keys)


def _view_dict(v, st, keys=True) -> dict:
    nts, nc = int(v.n_ts), int(v.n_cand)
    out = {"status": st, "stats": {k: getattr(v.stats, k) for k, _ in EnumStats._fields_}}
    for k in ("a", "b", "orbit", "count", "thr", "flags"):
        out[k] = _arr(getattr(v, k), nts, np.int32)
    out["thr_f"] = _arr(v.thr_f, nts, np.float32)
    off = _arr(v.var_off, nts + 1, np.int64) if nts else np.zeros(1, np.int64)
    vars_ = _arr(v.vars, int(off[-1]), np.int32)
    out["key_vars"], out["key_off"] = vars_, off
    if keys:
        flat, o = vars_.tolist(), off.tolist()
        out["keys"] = [tuple(flat[o[i]:o[i + 1]]) for i in range(nts)]
    out["cand_vars"] = _arr(v.cand_vars, 4 * nc, np.int32).reshape(nc, 4)
    for k in ("cand_thr", "cand_ts", "cand_flags", "cand_decodes", "cand_iters"):
        out[k] = _arr(getattr(v, k), nc, np.int32)
    out["cand_thr_f"] = _arr(v.cand_thr_f, nc, np.float32)
    return out


def ts_list_stats(lst: TsList, check: bool = True) -> dict:
    s = EnumStats()
    st = lib().ts_list_stats(lst.h, C.byref(s))
    if check:
        _check(st, "ts_list_stats")
    return {k: getattr(s, k) for k, _ in EnumStats._fields_}


def free_ts_list(lst: TsList):
    if lst.h:
        lib().free_ts_list(lst.h)
        lst.h = None


def tune_tile(code: Code, params=None, stream=None, **kw):
    """tune_tile(): returns (tuned EnumParams, decode ms of the best tile)."""
    p = params if isinstance(params, EnumParams) else make_params(**(params or {}), **kw)
    t = EnumParams()
    ms = C.c_float()
    _check(lib().tune_tile(code.h, C.byref(p), _stream_handle(stream), C.byref(t), C.byref(ms)), "tune_tile")
    return t, float(ms.value)


class Batch:
    """A batch of codes enumerated together (batch_create)."""

    def __init__(self, handle, codes):
        self.h = handle
        self.codes = list(codes)  # keeps the codes alive

    def __len__(self):
        return int(lib().batch_size(self.h))

    @property
    def multi_launch(self) -> bool:
        return bool(lib().batch_multi_launch(self.h))

    @property
    def decode_launches(self) -> int:
        return int(lib().batch_decode_launches(self.h))

    def __del__(self):
        if getattr(self, "h", None):
            lib().batch_free(self.h)
            self.h = None


def batch_create(codes, params, stream=None) -> Batch:
    """batch_create(): codes is a list of Code, params one EnumParams (or
    dict) for all of them or a list with one per code."""
    n = len(codes)
    if isinstance(params, (list, tuple)):
        ps = [p if isinstance(p, EnumParams) else make_params(**p) for p in params]
    else:
        p0 = params if isinstance(params, EnumParams) else make_params(**(params or {}))
        ps = [p0] * n
    if len(ps) != n:
        raise ValueError("one parameter set per code")
    harr = (C.c_void_p * n)(*[c.h for c in codes])
    parr = (EnumParams * n)(*ps)
    h = C.c_void_p()
    _check(lib().batch_create(harr, parr, n, _stream_handle(stream), C.byref(h)), "batch_create")
    return Batch(h, codes)


def batch_run(batch: Batch, stream=None):
    _check(lib().batch_run(batch.h, _stream_handle(stream)), "batch_run")


def batch_view(batch: Batch, i: int, check: bool = True, keys: bool = True) -> dict:
    v = TsView()
    st = lib().batch_view(batch.h, int(i), C.byref(v))
    if check:
        _check(st, "batch_view")
    return _view_dict(v, st, keys)


def batch_stats(batch: Batch, check: bool = True) -> dict:
    s = EnumStats()
    st = lib().batch_stats(batch.h, C.byref(s))
    if check:
        _check(st, "batch_stats")
    return {k: getattr(s, k) for k, _ in EnumStats._fields_}


def batch_free(batch: Batch):
    if batch.h:
        lib().batch_free(batch.h)
        batch.h = None


def is_params_default() -> IsParams:
    p = IsParams()
    lib().is_params_default(C.byref(p))
    return p


def is_fer_estimate(code: Code, ts_vars, stream=None, record: bool = False, **kw) -> dict:
    """is_fer_estimate(): importance-sampling FER toward the trapping set
    ts_vars.  Keyword arguments set tsx_is_params fields.  With record, the
    per-sample failure flags and log-weights are returned too."""
    p = is_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    T = _i32(ts_vars)
    r = IsResult()
    n = int(p.n_samples)
    fail = np.zeros(n, dtype=np.uint8) if record else None
    logw = np.zeros(n, dtype=np.float64) if record else None
    _check(lib().is_fer_estimate(code.h, T.ctypes.data_as(C.c_void_p), T.size, C.byref(p), _stream_handle(stream),
                                 C.byref(r), fail.ctypes.data_as(C.c_void_p) if record else None,
                                 logw.ctypes.data_as(C.c_void_p) if record else None), "is_fer_estimate")
    out = {k: getattr(r, k) for k, _ in IsResult._fields_}
    if record:
        out["fail"], out["logw"] = fail, logw
    return out


def decode_thresholds_noalloc(code: Code, cand_vars_ptr: int, n_cand: int, thr_ptr: int, thr_f_ptr, decodes_ptr: int,
                              iters_ptr: int, params=None, stream=None, check: bool = True, **kw) -> int:
    """decode_thresholds_noalloc(): decodes caller-given candidate sets with
    no device allocation; all pointers are device addresses (ints) of the
    caller's buffers (thr_f_ptr may be None).  Returns the status."""
    p = params if isinstance(params, EnumParams) else make_params(**(params or {}), **kw)
    st = lib().decode_thresholds_noalloc(code.h, C.byref(p), cand_vars_ptr, int(n_cand), thr_ptr, thr_f_ptr,
                                         decodes_ptr, iters_ptr, _stream_handle(stream))
    if check:
        _check(st, "decode_thresholds_noalloc")
    return st


def _struct_dict(x) -> dict:
    out = {}
    for k, _ in x._fields_:
        v = getattr(x, k)
        out[k] = _struct_dict(v) if isinstance(v, C.Structure) else v
    return out


def server_params_default() -> ServerParams:
    p = ServerParams()
    lib().server_params_default(C.byref(p))
    return p


class Server:
    """The serving runtime (server_create ... server_destroy).  Codes given to
    submit_* must stay alive until their jobs complete (the server keeps a
    reference until the job is released)."""

    def __init__(self, **kw):
        p = server_params_default()
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown server parameter {k}")
            setattr(p, k, v)
        h = C.c_void_p()
        _check(lib().server_create(C.byref(p), C.byref(h)), "server_create")
        self.h = h
        self.params = p
        self._keep = {}

    def _submit(self, job, keep) -> int:
        jid = C.c_uint64()
        _check(lib().server_submit(self.h, C.byref(job), C.byref(jid)), "server_submit")
        self._keep[jid.value] = keep
        return int(jid.value)

    def submit_enumerate(self, code: Code, params=None, **kw) -> int:
        p = params if isinstance(params, EnumParams) else make_params(**(params or {}), **kw)
        job = Job(kind=TSX_JOB_ENUMERATE, code=code.h, enum_params=p)
        return self._submit(job, code)

    def submit_is_fer(self, code: Code, ts_vars, **kw) -> int:
        p = is_params_default()
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        T = _i32(ts_vars)
        job = Job(kind=TSX_JOB_IS_FER, code=code.h, is_params=p, ts_vars=T.ctypes.data_as(C.c_void_p), a=T.size)
        return self._submit(job, code)

    def poll(self, jid: int):
        """None while queued or running, else the result dict."""
        r = JobResult()
        st = lib().server_poll(self.h, jid, C.byref(r))
        if st == TSX_EAGAIN:
            return None
        if st == TSX_ENOTFOUND:
            _check(st, "server_poll")
        return _struct_dict(r)

    def wait(self, jid: int, timeout_ms: float = -1.0):
        r = JobResult()
        st = lib().server_wait(self.h, jid, float(timeout_ms), C.byref(r))
        if st == TSX_EAGAIN:
            return None
        if st == TSX_ENOTFOUND:
            _check(st, "server_wait")
        return _struct_dict(r)

    def view(self, jid: int, check: bool = True, keys: bool = True) -> dict:
        v = TsView()
        st = lib().server_job_view(self.h, jid, C.byref(v))
        if check:
            _check(st, "server_job_view")
        return _view_dict(v, st, keys)

    def release(self, jid: int):
        _check(lib().server_release(self.h, jid), "server_release")
        self._keep.pop(jid, None)

    def drain(self):
        _check(lib().server_drain(self.h), "server_drain")

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().server_stats(self.h, C.byref(s)), "server_stats")
        return _struct_dict(s)

    def reset_stats(self):
        lib().server_reset_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def measure_peaks(stream=None) -> dict:
    """measure_peaks(): per-SM-clock issue rates measured on the current device."""
    p = Peaks()
    _check(lib().measure_peaks(C.byref(p), _stream_handle(stream)), "measure_peaks")
    return {k: getattr(p, k) for k, _ in Peaks._fields_}


def cycle_counts(code: Code):
    """cycle_counts(): the 4- and 6-cycles through every variable node (int64 arrays of n)."""
    n = int(code.info["n"])
    c4 = np.zeros(n, dtype=np.int64)
    c6 = np.zeros(n, dtype=np.int64)
    _check(lib().cycle_counts(code.h, c4.ctypes.data_as(C.c_void_p), c6.ctypes.data_as(C.c_void_p)), "cycle_counts")
    return c4, c6


def emd_spectrum(code: Code, lmax: int, stream=None) -> dict:
    """emd_spectrum(): closed walks from the representatives per length
    (walks[l]) and the class-weighted counts count2l[l, e]; count2l / (2l) is
    the number of cycles of length 2l with EMD e (per circulant orbit for a QC
    code)."""
    out = EmdSpectrum()
    _check(lib().emd_spectrum(code.h, int(lmax), _stream_handle(stream), C.byref(out)), "emd_spectrum")
    walks = np.array(out.walks[:], dtype=np.int64)
    count2l = np.array([row[:] for row in out.count2l], dtype=np.int64)
    return {"lmax": int(out.lmax), "walks": walks, "count2l": count2l, "ms": float(out.ms)}


def lnms_params(**kw) -> LnmsParams:
    p = LnmsParams()
    lib().lnms_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def lnms_decode(code: Code, llr_ptr: int, n_frames: int, fail_ptr: int, iters_ptr=None, x_ptr=None, stream=None,
                **kw) -> None:
    """lnms_decode(): the layered simulation decoder on caller frames; every
    pointer is a device address (int) of the caller's buffers."""
    p = lnms_params(**kw)
    _check(lib().lnms_decode(code.h, C.byref(p), llr_ptr, int(n_frames), fail_ptr, iters_ptr, x_ptr,
                             _stream_handle(stream)), "lnms_decode")


def lnms_simulate(code: Code, stream=None, record: bool = False, **kw) -> dict:
    """lnms_simulate(): frame-error simulation with the layered decoder.
    Keyword arguments set tsx_lnms_params and tsx_sim_params fields; with
    record, the per-frame failure flags are returned as well."""
    lp = LnmsParams()
    lib().lnms_params_default(C.byref(lp))
    sp = SimParams()
    lib().sim_params_default(C.byref(sp))
    for k, v in kw.items():
        if hasattr(lp, k):
            setattr(lp, k, v)
        elif hasattr(sp, k):
            setattr(sp, k, v)
        else:
            raise TypeError(f"unknown parameter {k}")
    r = SimResult()
    fail = np.zeros(int(sp.max_frames), dtype=np.uint8) if record else None
    _check(lib().lnms_simulate(code.h, C.byref(lp), C.byref(sp), _stream_handle(stream), C.byref(r),
                               fail.ctypes.data_as(C.c_void_p) if record else None), "lnms_simulate")
    out = {k: getattr(r, k) for k, _ in SimResult._fields_}
    if record:
        out["fail"] = fail[:int(r.frames)]
    return out


def union_bound_fer(code: Code, sets, mult, stream=None, **kw) -> dict:
    """union_bound_fer(): sum over the sets of mult * the importance-sampling
    FER toward the set (job key job_key + i for set i); keyword arguments set
    tsx_is_params fields."""
    p = is_params_default()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    sets = [np.asarray(t, dtype=np.int32) for t in sets]
    off = np.zeros(len(sets) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(t) for t in sets])
    flat = np.ascontiguousarray(np.concatenate(sets) if sets else np.zeros(0, np.int32), dtype=np.int32)
    m = np.ascontiguousarray(np.asarray(mult, dtype=np.float64))
    fer = np.zeros(len(sets), dtype=np.float64)
    r = UnionResult()
    _check(lib().union_bound_fer(code.h, len(sets), flat.ctypes.data_as(C.c_void_p), off.ctypes.data_as(C.c_void_p),
                                 m.ctypes.data_as(C.c_void_p), C.byref(p), _stream_handle(stream), C.byref(r),
                                 fer.ctypes.data_as(C.c_void_p)), "union_bound_fer")
    out = {k: getattr(r, k) for k, _ in UnionResult._fields_}
    out["fer"] = fer
    return out
