"""CPU oracle for the modified Cole impulse method -- TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded C (``oracle.c``) behind a ctypes wrapper.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never does and shares
no code with it.  Codes are accepted as duck-typed objects with the fields of
``synth.Code`` (kind, Z, shifts, n, m, row_ptr, col_idx).
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
F32P = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
U8P = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, so float results match
    the source's operation order on every host)."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp = os.path.join(_BUILD, "machine.txt")
    try:
        same = open(stamp).read().strip() == platform.machine()
    except OSError:
        same = False
    if force or not same or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(platform.machine())
    return _LIB


class _IsParams(C.Structure):
    _fields_ = [("ebn0_db", C.c_double), ("rate", C.c_double), ("mu", C.c_double), ("job", C.c_uint64),
                ("K", C.c_int), ("sat", C.c_int), ("alpha_num", C.c_int), ("alpha_shift", C.c_int)]


class _Params(C.Structure):
    _fields_ = [("decoder", C.c_int), ("K", C.c_int), ("base_llr", C.c_int), ("sat", C.c_int),
                ("alpha_num", C.c_int), ("alpha_shift", C.c_int), ("amp_steps", C.c_int),
                ("spa_clip", C.c_float), ("spa_amax", C.c_float), ("list_mode", C.c_int), ("kstart", C.c_int),
                ("spa_libm", C.c_int), ("budget_wref", C.c_int), ("budget_kmin", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.og_from_qc.restype = vp
            L.og_from_qc.argtypes = [C.c_int, C.c_int, C.c_int, I32P]
            L.og_from_csr.restype = vp
            L.og_from_csr.argtypes = [C.c_int, C.c_int, I32P, I32P]
            L.og_free.argtypes = [vp]
            for f in ("og_n", "og_m", "og_E", "og_girth"):
                getattr(L, f).argtypes = [vp]
                getattr(L, f).restype = C.c_int
            for f in ("og_vdeg", "og_cdeg"):
                getattr(L, f).argtypes = [vp, C.c_int]
                getattr(L, f).restype = C.c_int
            for f in ("og_vadj", "og_cadj"):
                getattr(L, f).argtypes = [vp, C.c_int, C.c_int]
                getattr(L, f).restype = C.c_int
            L.og_ball4.argtypes = [vp, C.c_int, I32P]
            L.og_ball4.restype = C.c_int
            L.og_canon.argtypes = [vp, I32P, C.c_int, I32P]
            L.og_canon.restype = C.c_int
            L.og_candidates.argtypes = [vp, C.c_int, C.c_int]
            L.og_candidates.restype = vp
            L.og_cands_count.argtypes = [vp]
            L.og_cands_count.restype = C.c_size_t
            L.og_cands_copy.argtypes = [vp, I32P]
            L.og_cands_free.argtypes = [vp]
            L.og_decode_nms.argtypes = [vp, I32P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                        U8P, C.POINTER(C.c_int), I32P, I32P, vp]
            L.og_decode_nms.restype = C.c_int
            L.og_decode_lnms.argtypes = [vp, I32P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, U8P,
                                         C.POINTER(C.c_int)]
            L.og_decode_lnms.restype = C.c_int
            L.og_decode_spa.argtypes = [vp, F32P, C.c_int, C.c_float, C.c_int, U8P,
                                        C.POINTER(C.c_int), I32P, C.c_int]
            L.og_decode_spa.restype = C.c_int
            L.og_spa_posterior.argtypes = [vp, F32P, C.c_int, C.c_float, F32P]
            L.og_tree.argtypes = [vp, U8P]
            L.og_ts_closure.argtypes = [vp, U8P, U8P]
            L.og_classify.argtypes = [vp, U8P, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]
            L.og_extract.argtypes = [vp, U8P, I32P, C.c_int, U8P]
            L.og_extract.restype = C.c_int
            L.og_enumerate.argtypes = [vp, C.POINTER(_Params), I32P, C.c_size_t]
            L.og_enumerate.restype = vp
            L.og_res_nts.argtypes = [vp]
            L.og_res_nts.restype = C.c_int
            L.og_res_cand.argtypes = [vp, I32P, F32P, I32P, I32P, I32P, I32P]
            L.og_res_ts.argtypes = [vp, C.c_int, I32P, C.POINTER(C.c_float), I32P]
            L.og_res_ts.restype = C.c_int
            L.og_res_free.argtypes = [vp]
            I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
            L.og_res_stats.argtypes = [vp, I64P]
            L.og_cycles_from.argtypes = [vp, C.c_int, C.c_int, I64P, vp]
            L.og_tanhf.argtypes = [C.c_float]
            L.og_tanhf.restype = C.c_float
            L.og_atanhf.argtypes = [C.c_float]
            L.og_atanhf.restype = C.c_float
            U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
            F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
            L.og_philox4x32_10.argtypes = [U32P, U32P, U32P]
            L.og_logf.argtypes = [C.c_float]
            L.og_logf.restype = C.c_float
            L.og_sincos2pi.argtypes = [C.c_float, C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.og_normals4.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, F32P]
            L.og_is_samples.argtypes = [C.c_void_p, I32P, C.c_int, C.POINTER(_IsParams), C.c_uint64, C.c_int,
                                        U8P, F64P]
            L.og_lnms_frames.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_int,
                                         C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, U8P, I32P, I32P]
            L.og_is_quant.argtypes = [C.c_float, C.c_float, C.c_int]
            L.og_is_quant.restype = C.c_int
            L.og_is_channel.argtypes = [C.c_void_p, I32P, C.c_int, C.POINTER(_IsParams), C.c_uint64, I32P, F32P]
            _lib = L
    return _lib


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) of a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().og_philox4x32_10(c, k, out)
    return out


def logf(x: float) -> float:
    return float(lib().og_logf(float(x)))


def sincos2pi(t: float):
    s, c = C.c_float(), C.c_float()
    lib().og_sincos2pi(float(t), C.byref(s), C.byref(c))
    return s.value, c.value


def normals4(job: int, sample: int, quad: int) -> np.ndarray:
    g = np.zeros(4, dtype=np.float32)
    lib().og_normals4(int(job), int(sample), int(quad), g)
    return g


def is_quant(y: float, cq: float, sat: int) -> int:
    """The importance-sampling channel quantizer: round-half-away(y * cq) in
    single precision, saturated to [-sat, sat]."""
    return int(lib().og_is_quant(float(y), float(cq), int(sat)))


def tanhf(x: float) -> float:
    """The sum-product decoder's single-precision tanh (series, IEEE ops)."""
    return float(lib().og_tanhf(float(x)))


def atanhf(x: float) -> float:
    """The sum-product decoder's single-precision atanh (series, IEEE ops)."""
    return float(lib().og_atanhf(float(x)))


@dataclass
class TS:
    """One distinct trapping set: (a, b), canonical key, orbit size, etc."""
    a: int
    b: int
    key: tuple
    orbit: int
    elementary: bool
    count: int
    thr: int
    thr_f: float
    kind: int  # 1 = Tree(X), 2 = Tree(TS(X)); list mode: 3 = both


@dataclass
class Enumeration:
    cands: np.ndarray     # [N, 5] size, v0..v3 (canonical keys, -1 padded)
    thr: np.ndarray       # int32 [N], -1 = no failure
    thr_f: np.ndarray     # float32 [N], -1 = no failure
    ts: np.ndarray        # int32 [N], index into ``ts_list`` or -1
    which: np.ndarray     # int32 [N], 0 none/acyclic, 1 Tree(X), 2 Tree(TS(X))
    decodes: np.ndarray   # int32 [N]
    iters: np.ndarray     # int32 [N], iterations summed over the candidate's decodes
    ts_list: list
    converged: int = 0    # decodes that ended in the all-zero word
    converged_iterations: int = 0
    kstart: int = 0       # list mode: the first iteration of the lists


class Graph:
    """The oracle's own Tanner graph (Sec. II, eqs. 1-2)."""

    def __init__(self, code):
        L = lib()
        self.code = code
        self.Z = int(code.Z) if code.kind == "qc" else 0
        if code.kind == "qc":
            s = np.ascontiguousarray(code.shifts, dtype=np.int32)
            self.h = L.og_from_qc(s.shape[0], s.shape[1], int(code.Z), s)
        else:
            self.h = L.og_from_csr(int(code.n), int(code.m),
                                   np.ascontiguousarray(code.row_ptr, dtype=np.int32),
                                   np.ascontiguousarray(code.col_idx, dtype=np.int32))
        self.n, self.m, self.E = L.og_n(self.h), L.og_m(self.h), L.og_E(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().og_free(self.h)
            self.h = None

    # --- structure -----------------------------------------------------
    def vn_checks(self, v):
        L = lib()
        return [L.og_vadj(self.h, v, i) for i in range(L.og_vdeg(self.h, v))]

    def check_vns(self, c):
        L = lib()
        return [L.og_cadj(self.h, c, p) for p in range(L.og_cdeg(self.h, c))]

    def dense(self) -> np.ndarray:
        H = np.zeros((self.m, self.n), dtype=np.uint8)
        for c in range(self.m):
            H[c, self.check_vns(c)] = 1
        return H

    def girth(self) -> int:
        return lib().og_girth(self.h)

    def ball4(self, v) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int32)
        k = lib().og_ball4(self.h, int(v), out)
        return out[:k].copy()

    def canon(self, T):
        T = np.ascontiguousarray(np.asarray(T, dtype=np.int32))
        key = np.empty(max(1, T.size), dtype=np.int32)
        orbit = lib().og_canon(self.h, T, T.size, key)
        return tuple(int(x) for x in key[:T.size]), orbit

    def candidates(self, max_size=3, cycle_len=0) -> np.ndarray:
        L = lib()
        h = L.og_candidates(self.h, max_size, cycle_len)
        n = L.og_cands_count(h)
        out = np.empty((n, 5), dtype=np.int32)
        if n:
            L.og_cands_copy(h, out)
        L.og_cands_free(h)
        return out

    # --- decoders -------------------------------------------------------
    def decode_nms(self, Lv, K, sat=511, alpha_num=3, alpha_shift=2, wstart=None, trace=False):
        Lv = np.ascontiguousarray(np.asarray(Lv, dtype=np.int32))
        ws = max(1, self.girth() // 2) if wstart is None else wstart
        xb = np.zeros(self.n, dtype=np.uint8)
        kl = C.c_int()
        ut = np.zeros(K + 1, dtype=np.int32)
        P = np.zeros(self.n, dtype=np.int32)
        xt = np.zeros((K + 1, self.n), dtype=np.uint8) if trace else None
        f = lib().og_decode_nms(self.h, Lv, K, sat, alpha_num, alpha_shift, ws, xb, C.byref(kl), ut, P,
                                xt.ctypes.data_as(C.c_void_p) if trace else None)
        self.last_P = P
        # with trace, self.last_trace[k] = x_k for k = 0..K_last
        self.last_trace = xt[: kl.value + 1] if trace else None
        return bool(f), xb, kl.value, ut[: kl.value + 1]

    def decode_lnms(self, Lv, K=20, llr_bits=4, c2v_bits=4, v2c_bits=6, alpha_num=3, alpha_shift=2):
        """The quantized layered normalized min-sum of the paper's simulations:
        returns (failed, x, iterations run)."""
        Lv = np.ascontiguousarray(np.asarray(Lv, dtype=np.int32))
        x = np.zeros(self.n, dtype=np.uint8)
        kl = C.c_int()
        f = lib().og_decode_lnms(self.h, Lv, K, llr_bits, c2v_bits, v2c_bits, alpha_num, alpha_shift, x,
                                 C.byref(kl))
        return bool(f), x, kl.value

    def lnms_frames(self, *, ebn0_db, rate=None, llr_scale=1.0, job=0, f0=0, n=100, K=20, llr_bits=4, c2v_bits=4,
                    v2c_bits=6, alpha_num=3, alpha_shift=2):
        """Frames of the layered decoder's frame-error simulation: per frame the
        failure flag, iterations and the Hamming weight of the decision."""
        r = (1.0 - self.m / self.n) if rate is None else rate
        fail = np.zeros(n, dtype=np.uint8)
        it = np.zeros(n, dtype=np.int32)
        w = np.zeros(n, dtype=np.int32)
        lib().og_lnms_frames(self.h, float(ebn0_db), float(r), float(llr_scale), int(job), int(f0), int(n), K,
                             llr_bits, c2v_bits, v2c_bits, alpha_num, alpha_shift, fail, it, w)
        return fail, it, w

    def decode_spa(self, Lv, K, clip=30.0, wstart=None, libm=False):
        Lv = np.ascontiguousarray(np.asarray(Lv, dtype=np.float32))
        ws = max(1, self.girth() // 2) if wstart is None else wstart
        xb = np.zeros(self.n, dtype=np.uint8)
        kl = C.c_int()
        ut = np.zeros(K + 1, dtype=np.int32)
        f = lib().og_decode_spa(self.h, Lv, K, clip, ws, xb, C.byref(kl), ut, 1 if libm else 0)
        return bool(f), xb, kl.value, ut[: kl.value + 1]

    def spa_posterior(self, Lv, K, clip=30.0):
        Lv = np.ascontiguousarray(np.asarray(Lv, dtype=np.float32))
        P = np.zeros(self.n, dtype=np.float32)
        lib().og_spa_posterior(self.h, Lv, K, clip, P)
        return P

    # --- sieving --------------------------------------------------------
    def _ind(self, S):
        x = np.zeros(self.n, dtype=np.uint8)
        x[np.asarray(list(S), dtype=np.int64)] = 1
        return x

    def tree(self, S):
        x = self._ind(S)
        lib().og_tree(self.h, x)
        return set(np.flatnonzero(x).tolist())

    def ts_closure(self, S):
        x = self._ind(S)
        out = np.zeros(self.n, dtype=np.uint8)
        lib().og_ts_closure(self.h, x, out)
        return set(np.flatnonzero(out).tolist())

    def classify(self, T):
        a, b, e = C.c_int(), C.c_int(), C.c_int()
        lib().og_classify(self.h, self._ind(T), C.byref(a), C.byref(b), C.byref(e))
        return a.value, b.value, bool(e.value)

    def extract(self, xstar, I):
        xs = np.ascontiguousarray(np.asarray(xstar, dtype=np.uint8))
        Ia = np.ascontiguousarray(np.asarray(I, dtype=np.int32))
        T = np.zeros(self.n, dtype=np.uint8)
        which = lib().og_extract(self.h, xs, Ia, Ia.size, T)
        return which, set(np.flatnonzero(T).tolist())

    # --- importance-sampling FER ----------------------------------------
    def is_samples(self, T, *, ebn0_db, rate=None, mu=1.0, job=0, s0=0, n=1000, K=20, sat=511,
                   alpha_num=3, alpha_shift=2):
        """Per-sample failure flags and log-weights of the mean-shift IS estimator."""
        Ta = np.ascontiguousarray(np.sort(np.asarray(list(T), dtype=np.int32)))
        r = (1.0 - self.m / self.n) if rate is None else rate
        p = _IsParams(float(ebn0_db), float(r), float(mu), int(job), K, sat, alpha_num, alpha_shift)
        fail = np.zeros(n, dtype=np.uint8)
        logw = np.zeros(n, dtype=np.float64)
        lib().og_is_samples(self.h, Ta, Ta.size, C.byref(p), int(s0), int(n), fail, logw)
        return fail, logw

    def is_channel(self, T, *, ebn0_db, rate=None, mu=1.0, job=0, sample=0, sat=511):
        """The quantized channel LLRs and the drawn noise (before the shift) of one sample."""
        Ta = np.ascontiguousarray(np.sort(np.asarray(list(T), dtype=np.int32)))
        r = (1.0 - self.m / self.n) if rate is None else rate
        p = _IsParams(float(ebn0_db), float(r), float(mu), int(job), 20, sat, 3, 2)
        L = np.zeros(self.n, dtype=np.int32)
        nv = np.zeros(self.n, dtype=np.float32)
        lib().og_is_channel(self.h, Ta, Ta.size, C.byref(p), int(sample), L, nv)
        return L, nv

    # --- cycles -----------------------------------------------------------
    def cycle_walks(self, v, lmax, emd=False):
        """Closed walks from v around simple cycles of l = 2..lmax variable
        nodes (each cycle through v twice, one per direction): walks[l], and
        with emd, hist[l, e] by the cycle's EMD e."""
        walks = np.zeros(lmax + 1, dtype=np.int64)
        hist = np.zeros((lmax + 1) * 128, dtype=np.int64) if emd else None
        lib().og_cycles_from(self.h, int(v), int(lmax), walks,
                             hist.ctypes.data_as(C.c_void_p) if emd else None)
        return (walks, hist.reshape(lmax + 1, 128)) if emd else walks

    def emd_spectrum(self, lmax, starts=None):
        """Sum over the start nodes (QC: the orbit representatives (j,0);
        general: every node) of the closed walks by length and EMD; dividing
        by 2l gives cycles per circulant orbit (QC) or cycles (general)."""
        if starts is None:
            starts = [j * self.Z for j in range(self.n // self.Z)] if self.Z else range(self.n)
        hist = np.zeros((lmax + 1, 128), dtype=np.int64)
        walks = np.zeros(lmax + 1, dtype=np.int64)
        for v in starts:
            w, h = self.cycle_walks(v, lmax, emd=True)
            hist += h
            walks += w
        return walks, hist

    # --- the whole method -----------------------------------------------
    def enumerate(self, cands=None, *, decoder="nms", K=20, base_llr=16, sat=511, alpha_num=3,
                  alpha_shift=2, amp_steps=10, spa_clip=30.0, spa_amax=64.0, max_size=3,
                  cycle_len=0, list_mode=False, kstart=0, spa_libm=False, budget_wref=0,
                  budget_kmin=1) -> Enumeration:
        """list_mode (min-sum): every non-empty set of the ordered list S1(x_k),
        S2(x_k), k = kstart (0: floor(girth/2); -1: ceil of the average
        iterations of the converged decodes of a first stage) .. K_last, of the
        decode at the threshold is a trapping set; per trapping set, count =
        candidates whose list holds it and kind = 1 (S1), 2 (S2) or 3 (both);
        the per-candidate ts index is -1 in this mode.  budget_wref > 0: the
        cycle-density iteration budget of each candidate."""
        if cands is None:
            cands = self.candidates(max_size, cycle_len)
        cands = np.ascontiguousarray(np.asarray(cands, dtype=np.int32).reshape(-1, 5))
        p = _Params(0 if decoder == "nms" else 1, K, base_llr, sat, alpha_num, alpha_shift,
                    amp_steps, spa_clip, spa_amax, 1 if list_mode else 0, kstart, 1 if spa_libm else 0,
                    budget_wref, budget_kmin)
        L = lib()
        h = L.og_enumerate(self.h, C.byref(p), cands, cands.shape[0])
        N = cands.shape[0]
        thr = np.empty(N, np.int32); thr_f = np.empty(N, np.float32)
        ts = np.empty(N, np.int32); which = np.empty(N, np.int32)
        dec = np.empty(N, np.int32); it = np.empty(N, np.int32)
        if N:
            L.og_res_cand(h, thr, thr_f, ts, which, dec, it)
        out = []
        info = np.empty(7, np.int32)
        key = np.empty(self.n, np.int32)
        tf = C.c_float()
        for i in range(L.og_res_nts(h)):
            a = L.og_res_ts(h, i, info, C.byref(tf), key)
            out.append(TS(a=int(info[0]), b=int(info[1]), key=tuple(int(x) for x in key[:a]),
                          orbit=int(info[2]), elementary=bool(info[3]), count=int(info[4]),
                          thr=int(info[5]), thr_f=float(tf.value), kind=int(info[6])))
        st = np.zeros(3, dtype=np.int64)
        L.og_res_stats(h, st)
        L.og_res_free(h)
        return Enumeration(cands, thr, thr_f, ts, which, dec, it, out, int(st[0]), int(st[1]), int(st[2]))
