"""ctypes wrapper around the plain-C oracle (pc_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg.  The product path never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "pc_oracle.c")]
_HDR = [os.path.join(_HERE, "pc_oracle.h")]
_lock = threading.Lock()
_lib = None

F32, F64 = 0, 1
PRED_LORENZO, PRED_MLP, PRED_MLP_BF16, PRED_MLP64 = 0, 1, 2, 3
ERR = {0: "ok", -1: "arg", -2: "dtype", -3: "nonfinite", -4: "capacity", -5: "corrupt", -8: "eb_range"}
LMAX = 24
BATCH = 256


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, IEEE semantics."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + _HDR)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Consts(C.Structure):
    _fields_ = [("dtype", C.c_int), ("eb", C.c_double), ("abs_min", C.c_double), ("abs_max", C.c_double),
                ("trivial", C.c_int), ("step64", C.c_double), ("step32", C.c_float), ("inv32", C.c_float),
                ("ebdn32", C.c_float), ("stepd", C.c_double), ("invd", C.c_double), ("ebdnd", C.c_double),
                ("Kp", C.c_int32), ("Kn", C.c_int32), ("Zq", C.c_int32), ("S", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("eb", C.c_double), ("block", C.c_int * 3), ("pred", C.c_int), ("stencil", C.c_int),
                ("h1", C.c_int), ("h2", C.c_int), ("m", C.c_int), ("s_in", C.c_int),
                ("weights", C.c_void_p), ("qnet", C.c_void_p), ("codebook", C.c_void_p), ("codebook_n", C.c_int),
                ("literal", C.c_int), ("eq_period", C.c_int), ("lossless", C.c_int)]


class Dump(C.Structure):
    _fields_ = [("dq", C.c_void_p), ("ok", C.c_void_p), ("codes", C.c_void_p), ("nnflag", C.c_void_p),
                ("hist", C.c_void_p), ("lens", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u64p = C.POINTER(C.c_uint64)
            L.orc_L32.restype = C.c_float; L.orc_L32.argtypes = [C.c_float]
            L.orc_E32.restype = C.c_float; L.orc_E32.argtypes = [C.c_float]
            L.orc_L64.restype = C.c_double; L.orc_L64.argtypes = [C.c_double]
            L.orc_E64.restype = C.c_double; L.orc_E64.argtypes = [C.c_double]
            L.orc_mix64.restype = C.c_uint64; L.orc_mix64.argtypes = [C.c_uint64, C.c_uint64]
            L.orc_crc32.restype = C.c_uint32; L.orc_crc32.argtypes = [C.c_void_p, C.c_size_t]
            L.orc_stats.restype = C.c_int
            L.orc_stats.argtypes = [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_int)]
            L.orc_make_consts.restype = C.c_int
            L.orc_make_consts.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                          C.POINTER(Consts)]
            L.orc_recon32.restype = C.c_float; L.orc_recon32.argtypes = [C.c_int32, C.POINTER(Consts)]
            L.orc_recon64.restype = C.c_double; L.orc_recon64.argtypes = [C.c_int32, C.POINTER(Consts)]
            L.orc_transform32.restype = None
            L.orc_transform32.argtypes = [C.c_float, C.POINTER(Consts), C.POINTER(C.c_int32), C.POINTER(C.c_int)]
            L.orc_transform64.restype = None
            L.orc_transform64.argtypes = [C.c_double, C.POINTER(Consts), C.POINTER(C.c_int32), C.POINTER(C.c_int)]
            L.orc_lz_weight.restype = C.c_int; L.orc_lz_weight.argtypes = [C.c_int, C.c_int]
            L.orc_mlp_nweights.restype = C.c_int; L.orc_mlp_nweights.argtypes = [C.c_int] * 3
            L.orc_mlp_fwd32.restype = C.c_float
            L.orc_mlp_fwd32.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
            L.orc_mlp_pred32.restype = C.c_int32
            L.orc_mlp_pred32.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
            L.orc_mlp_fwd64.restype = C.c_double
            L.orc_mlp_fwd64.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
            L.orc_mlp_pred64.restype = C.c_int32
            L.orc_mlp_pred64.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
            L.orc_val_size.restype = C.c_uint64
            L.orc_val_size.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_uint64, C.c_int, C.c_int]
            L.orc_val_hist.restype = None
            L.orc_val_hist.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_uint64, C.c_int, C.c_void_p]
            L.orc_sample_codebook.restype = C.c_int
            L.orc_sample_codebook.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p]
            L.orc_sample_codebook_for.restype = C.c_int
            L.orc_sample_codebook_for.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, C.POINTER(C.c_int),
                                                  C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                                  C.c_uint64, C.c_uint32, C.c_int, C.c_void_p]
            L.orc_lz_bound.restype = C.c_uint64
            L.orc_lz_bound.argtypes = [C.c_uint64]
            L.orc_lz_encode.restype = C.c_uint64
            L.orc_lz_encode.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p]
            L.orc_lz_decode.restype = C.c_int
            L.orc_lz_decode.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64]
            L.orc_coverage_m.restype = C.c_int
            L.orc_coverage_m.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_uint64, C.c_double]
            L.orc_train_select.restype = C.c_int
            L.orc_train_select.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, C.POINTER(C.c_int), C.c_int,
                                           C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_void_p,
                                           C.POINTER(C.c_int)]
            L.orc_block_codes.restype = C.c_int
            L.orc_block_codes.argtypes = [C.c_void_p, u64p, C.c_int, C.POINTER(Consts), C.POINTER(Params), C.c_uint64,
                                          C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.orc_pred_report.restype = C.c_int
            L.orc_pred_report.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, C.POINTER(C.c_int), C.c_int,
                                          C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
            L.orc_huffman_lengths.restype = C.c_int
            L.orc_huffman_lengths.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_canonical_codes.restype = C.c_int
            L.orc_canonical_codes.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            L.orc_compress_bound.restype = C.c_uint64
            L.orc_compress_bound.argtypes = [u64p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int]
            L.orc_compress.restype = C.c_int
            L.orc_compress.argtypes = [C.c_void_p, u64p, C.c_int, C.POINTER(Params), C.c_void_p, C.c_uint64,
                                       u64p, C.POINTER(Dump)]
            L.orc_read_header.restype = C.c_int
            L.orc_read_header.argtypes = [C.c_void_p, C.c_uint64, u64p, C.POINTER(C.c_int)]
            L.orc_decompress.restype = C.c_int
            L.orc_decompress.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64]
            L.orc_count_samples.restype = C.c_int
            L.orc_count_samples.argtypes = [u64p, C.POINTER(C.c_int), C.c_uint64, C.c_uint32, u64p, u64p]
            L.orc_gather_samples.restype = C.c_int
            L.orc_gather_samples.argtypes = [C.c_void_p, u64p, C.c_int, C.POINTER(Consts), C.POINTER(C.c_int),
                                             C.c_int, C.c_uint64, C.c_uint32] + [C.c_void_p] * 6
            L.orc_input_shift.restype = C.c_int
            L.orc_input_shift.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64]
            L.orc_init_weights.restype = None
            L.orc_init_weights.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64]
            L.orc_batch_grad.restype = None
            L.orc_batch_grad.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]
            L.orc_sgd_update.restype = None
            L.orc_sgd_update.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float]
            L.orc_train_epoch.restype = None
            L.orc_train_epoch.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_uint64, C.c_float, C.c_float, C.c_uint64]
            L.orc_val_cost.restype = C.c_uint64
            L.orc_val_cost.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_uint64, C.c_int]
            L.orc_train.restype = C.c_int
            L.orc_train.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, C.POINTER(C.c_int), C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_uint64, C.c_uint32, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_int), C.c_void_p]
            L.orc_qnet_len.restype = C.c_int; L.orc_qnet_len.argtypes = [C.c_int] * 3
            L.orc_mlp_pred_q.restype = C.c_int32; L.orc_mlp_pred_q.argtypes = [C.c_void_p, C.c_void_p]
            L.orc_qnet_build.restype = C.c_int
            L.orc_qnet_build.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                         C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p]
            L.orc_quantize.restype = C.c_int
            L.orc_quantize.argtypes = [C.c_void_p, u64p, C.c_int, C.c_double, C.POINTER(C.c_int), C.c_int, C.c_int,
                                       C.c_int, C.c_uint64, C.c_uint32, C.c_void_p, C.c_int, C.c_void_p]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims(x: np.ndarray):
    shp = list(x.shape)
    while len(shp) < 3:
        shp.insert(0, 1)
    if len(shp) != 3:
        raise ValueError("fields are 1-D, 2-D or 3-D")
    return (C.c_uint64 * 3)(*shp)


def _dtype_code(x: np.ndarray) -> int:
    if x.dtype == np.float32:
        return F32
    if x.dtype == np.float64:
        return F64
    raise TypeError("float32 or float64 field expected")


# ---------------------------------------------------------------- numerics
def L32(y): return lib().orc_L32(float(y))
def E32(t): return lib().orc_E32(float(t))
def L64(y): return lib().orc_L64(float(y))
def E64(t): return lib().orc_E64(float(t))
def mix64(seed, i): return lib().orc_mix64(seed, i)


def crc32(b: bytes) -> int:
    buf = np.frombuffer(b, dtype=np.uint8).copy()
    return lib().orc_crc32(_p(buf), len(b))


def stats(x: np.ndarray):
    x = np.ascontiguousarray(x)
    mn, mx, tr = C.c_double(), C.c_double(), C.c_int()
    st = lib().orc_stats(_p(x), x.size, _dtype_code(x), C.byref(mn), C.byref(mx), C.byref(tr))
    return st, mn.value, mx.value, tr.value


def make_consts(dtype: int, amin: float, amax: float, trivial: int, eb: float):
    c = Consts()
    st = lib().orc_make_consts(dtype, amin, amax, trivial, eb, C.byref(c))
    return st, c


def consts_for(x: np.ndarray, eb: float) -> Consts:
    st, mn, mx, tr = stats(x)
    assert st == 0, ERR.get(st)
    st, c = make_consts(_dtype_code(x), mn, mx, tr, eb)
    assert st == 0, ERR.get(st)
    return c


def transform(x: np.ndarray, c: Consts):
    """Per-point (dq, ok) for a float32 or float64 array."""
    flat = np.ascontiguousarray(x).ravel()
    dq = np.empty(flat.size, np.int32)
    ok = np.empty(flat.size, np.uint8)
    L = lib()
    q, o = C.c_int32(), C.c_int()
    f = L.orc_transform32 if flat.dtype == np.float32 else L.orc_transform64
    for i, v in enumerate(flat.tolist()):
        f(v, C.byref(c), C.byref(q), C.byref(o))
        dq[i] = q.value
        ok[i] = o.value
    return dq.reshape(x.shape), ok.reshape(x.shape)


def recon(q: int, c: Consts, dtype: int = F32):
    L = lib()
    return L.orc_recon32(int(q), C.byref(c)) if dtype == F32 else L.orc_recon64(int(q), C.byref(c))


def lz_weight(k: int, i: int) -> int:
    return lib().orc_lz_weight(k, i)


def mlp_nweights(k: int, h1: int, h2: int) -> int:
    return lib().orc_mlp_nweights(k, h1, h2)


def mlp_fwd32(w: np.ndarray, k, h1, h2, s_in, v) -> float:
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(v, np.int32)
    return lib().orc_mlp_fwd32(_p(w), k, h1, h2, s_in, _p(v))


def mlp_pred32(w: np.ndarray, k, h1, h2, s_in, v) -> int:
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(v, np.int32)
    return lib().orc_mlp_pred32(_p(w), k, h1, h2, s_in, _p(v))


def mlp_fwd64(w: np.ndarray, k, h1, h2, s_in, v) -> float:
    """The FP32 weights evaluated in FP64 (the reporting predictor)."""
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(v, np.int32)
    return lib().orc_mlp_fwd64(_p(w), k, h1, h2, s_in, _p(v))


def mlp_pred64(w: np.ndarray, k, h1, h2, s_in, v) -> int:
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(v, np.int32)
    return lib().orc_mlp_pred64(_p(w), k, h1, h2, s_in, _p(v))


def pred_report(x: np.ndarray, eb: float, w, s_in: int, block=(8, 8, 8), k=7, h1=16, h2=16, qnet=None, m=16):
    """Prediction error of Lorenzo and of the FP64, FP32 and fixed-point forms of one network over every
    non-anchor point of a field (the oracle's orc_pred_report).  Returns a dict."""
    x = np.ascontiguousarray(x)
    w = np.ascontiguousarray(w, np.float32)
    q = None if qnet is None else np.ascontiguousarray(qnet, np.int64)
    out = np.zeros(13, np.float64)
    b = (C.c_int * 3)(*block)
    st = lib().orc_pred_report(_p(x), _dims(x), _dtype_code(x), eb, b, k, h1, h2, s_in, _p(w),
                               None if q is None else _p(q), m, _p(out))
    assert st == 0, st
    n = max(out[0], 1.0)
    names = ["lorenzo", "fp64", "fp32", "fixed_point"]
    return {"points": int(out[0]),
            "rms_residual": {nm: float(np.sqrt(out[1 + i] / n)) for i, nm in enumerate(names)},
            "rms_vs_fp64": {"fp32": float(np.sqrt(out[5] / n)), "fixed_point": float(np.sqrt(out[6] / n))},
            "frac_differs_from_fp64": {"fp32": out[7] / n, "fixed_point": out[8] / n},
            "bits_proxy_per_point": {nm: out[9 + i] / n for i, nm in enumerate(names)}}


# ------------------------------------------------ fixed-point (BF16) perceptron
def qnet_len(k: int, h1: int, h2: int) -> int:
    return lib().orc_qnet_len(k, h1, h2)


def mlp_pred_q(q: np.ndarray, v) -> int:
    """Prediction of the fixed-point network q (int64 layout of orc_qnet_len)."""
    q = np.ascontiguousarray(q, np.int64)
    v = np.ascontiguousarray(v, np.int32)
    return lib().orc_mlp_pred_q(_p(q), _p(v))


def qnet_build(w, k, h1, h2, s_in, tin, tuse, vin=None, vuse=None) -> np.ndarray:
    """Quantize FP32 weights with shifts chosen from the given (used) sample inputs."""
    w = np.ascontiguousarray(w, np.float32)
    tin = np.ascontiguousarray(tin, np.int32).reshape(-1)
    tuse = np.ascontiguousarray(tuse, np.uint8)
    if vin is None:
        vin = np.zeros(k, np.int32); vuse = np.zeros(1, np.uint8); nv = 0
    else:
        vin = np.ascontiguousarray(vin, np.int32).reshape(-1); vuse = np.ascontiguousarray(vuse, np.uint8)
        nv = vuse.size
    q = np.zeros(qnet_len(k, h1, h2), np.int64)
    st = lib().orc_qnet_build(_p(w), k, h1, h2, s_in, _p(tin), _p(tuse), tuse.size, _p(vin), _p(vuse), nv, _p(q))
    assert st == 0
    return q


def quantize(x: np.ndarray, eb: float, w, s_in: int, block=(8, 8, 8), k=7, h1=16, h2=16, seed=0,
             thr32=None) -> np.ndarray:
    """Fixed-point form of the trained perceptron w, shifts from the training phase's samples."""
    x = np.ascontiguousarray(x)
    if thr32 is None:
        thr32 = int(0.1 * 2 ** 32)
    w = np.ascontiguousarray(w, np.float32)
    q = np.zeros(qnet_len(k, h1, h2), np.int64)
    b = (C.c_int * 3)(*block)
    st = lib().orc_quantize(_p(x), _dims(x), _dtype_code(x), eb, b, k, h1, h2, seed, thr32, _p(w), s_in, _p(q))
    assert st == 0, st
    return q


def huffman_lengths(hist: np.ndarray, lmax: int = LMAX, with_order: bool = False):
    """Code lengths per symbol; with_order also returns the code order (most frequent first)."""
    h = np.ascontiguousarray(hist, np.uint64)
    out = np.zeros(h.size, np.uint8)
    order = np.zeros(max(h.size, 1), np.uint32)
    n = lib().orc_huffman_lengths(_p(h), h.size, lmax, _p(out), _p(order))
    if with_order:
        return out, order[:n].copy()
    return out


def canonical_codes(lens: np.ndarray, order=None) -> np.ndarray:
    """Code words along `order` (default: by length, then symbol, as in RFC 1951)."""
    ln = np.ascontiguousarray(lens, np.uint8)
    if order is None:
        used = np.flatnonzero(ln)
        order = used[np.lexsort((used, ln[used]))]
    order = np.ascontiguousarray(order, np.uint32)
    out = np.zeros(ln.size, np.uint32)
    st = lib().orc_canonical_codes(_p(order), order.size, _p(ln), _p(out))
    assert st == 0, "lengths must not decrease along the order"
    return out


def _params(eb, block, pred, stencil, h1, h2, m, s_in, w, q=None, cb=None):
    p = Params()
    p.codebook = None if cb is None else cb.ctypes.data
    p.codebook_n = 0 if cb is None else cb.size
    p.eb = eb
    p.block[:] = list(block)
    p.pred = pred
    p.stencil = stencil
    p.h1, p.h2, p.m, p.s_in = h1, h2, m, s_in
    p.weights = None if w is None else w.ctypes.data
    p.qnet = None if q is None else q.ctypes.data
    return p


def compress_bound(shape3, dtype: int, block, m: int = 16, nweights: int = 0) -> int:
    d = (C.c_uint64 * 3)(*shape3)
    b = (C.c_int * 3)(*block)
    return lib().orc_compress_bound(d, dtype, b, m, nweights)


def compress(x: np.ndarray, eb: float, block=(8, 8, 8), weights=None, stencil=7, h1=16, h2=16,
             m: int = 16, s_in: int = 0, dump: bool = False, qnet=None, fp64: bool = False, codebook=None,
             literal: bool = False, eq_period: int = 0, lossless: bool = False):
    """Compress with the oracle.  Returns (status, bytes[, dump dict]).  `qnet` selects the
    fixed-point (BF16) perceptron form instead of the FP32 weights; fp64=True evaluates the
    FP32 weights in FP64 (the reporting predictor, which only the oracle encodes with).
    `codebook` (uint32 list, sym | len << 16) compresses with that sample codebook: codes
    outside it become balance points and the stream precedes the balance values.
    literal=True: the paper-literal data selection (predict from true values; float32 only),
    with a deliberate equilibrium point every eq_period points of each block (0: none).
    lossless=True: the lossless stage over the bitstream bytes."""
    x = np.ascontiguousarray(x)
    dims = _dims(x)
    dt = _dtype_code(x)
    w = None if weights is None else np.ascontiguousarray(weights, np.float32)
    q = None if qnet is None else np.ascontiguousarray(qnet, np.int64)
    nw = 0 if w is None else w.size
    if w is not None:
        assert nw == mlp_nweights(stencil, h1, h2)
    if q is not None:
        assert q.size == qnet_len(stencil, h1, h2)
        nw = 2 * q.size
    pred = PRED_MLP_BF16 if q is not None else (PRED_MLP if w is not None else PRED_LORENZO)
    if fp64 and w is not None and q is None:
        pred = PRED_MLP64
    cb = None if codebook is None else np.ascontiguousarray(codebook, np.uint32)
    p = _params(eb, block, pred, stencil, h1, h2, m, s_in, w, q, cb)
    p.literal = int(bool(literal))
    p.eq_period = int(eq_period)
    p.lossless = int(bool(lossless))
    cap = compress_bound(tuple(dims), dt, block, m, nw)
    out = np.zeros(cap, np.uint8)
    size = C.c_uint64()
    d = None
    dobj = None
    if dump:
        nb = [(dims[i] + block[i] - 1) // block[i] for i in range(3)]
        nblocks = nb[0] * nb[1] * nb[2]
        bvol = block[0] * block[1] * block[2]
        d = dict(dq=np.zeros(x.size, np.int32), ok=np.zeros(x.size, np.uint8),
                 codes=np.zeros(nblocks * bvol, np.uint16), nnflag=np.zeros(nblocks, np.uint8),
                 hist=np.zeros(1 << m, np.uint64), lens=np.zeros(1 << m, np.uint8))
        dobj = Dump(*[d[k].ctypes.data for k in ("dq", "ok", "codes", "nnflag", "hist", "lens")])
    st = lib().orc_compress(_p(x), dims, dt, C.byref(p), _p(out), cap, C.byref(size),
                            C.byref(dobj) if dobj is not None else None)
    blob = out[: size.value].tobytes() if st == 0 else b""
    if dump:
        return st, blob, d
    return st, blob


def block_codes(x: np.ndarray, consts, bi: int, eb: float, block=(8, 8, 8), weights=None, stencil=7, h1=16, h2=16,
                m: int = 16, s_in: int = 0, qnet=None):
    """Codes (as stored) and perceptron flag of block bi, from the field's constants `consts`
    (consts_for of the whole field); only the block's points are transformed."""
    x = np.ascontiguousarray(x)
    w = None if weights is None else np.ascontiguousarray(weights, np.float32)
    q = None if qnet is None else np.ascontiguousarray(qnet, np.int64)
    pred = PRED_MLP_BF16 if q is not None else (PRED_MLP if w is not None else PRED_LORENZO)
    p = _params(eb, block, pred, stencil, h1, h2, m, s_in, w, q)
    codes = np.zeros(block[0] * block[1] * block[2], np.uint16)
    usen, npts = C.c_int(), C.c_int()
    st = lib().orc_block_codes(_p(x), _dims(x), _dtype_code(x), C.byref(consts), C.byref(p), int(bi), _p(codes),
                               C.byref(usen), C.byref(npts))
    assert st == 0, st
    return codes[: npts.value], bool(usen.value)


def read_header(blob: bytes):
    buf = np.frombuffer(blob, np.uint8).copy()
    dims = (C.c_uint64 * 3)()
    dt = C.c_int()
    st = lib().orc_read_header(_p(buf), len(blob), dims, C.byref(dt))
    return st, tuple(dims), dt.value


def decompress(blob: bytes):
    """Decompress with the oracle.  Returns (status, array or None)."""
    st, dims, dt = read_header(blob)
    if st:
        return st, None
    if dt not in (F32, F64):
        return -5, None
    n = dims[0] * dims[1] * dims[2]
    if n > (1 << 34):
        return -5, None
    out = np.zeros(n, np.float32 if dt == F32 else np.float64)
    buf = np.frombuffer(blob, np.uint8).copy()
    st = lib().orc_decompress(_p(buf), len(blob), _p(out), n)
    if st:
        return st, None
    return 0, out.reshape(dims)


# ---------------------------------------------------------------- training
def count_samples(shape3, block, seed: int, thr32: int):
    d = (C.c_uint64 * 3)(*shape3)
    b = (C.c_int * 3)(*block)
    nt, nv = C.c_uint64(), C.c_uint64()
    st = lib().orc_count_samples(d, b, seed, thr32, C.byref(nt), C.byref(nv))
    assert st == 0
    return nt.value, nv.value


def gather_samples(x: np.ndarray, eb: float, block, k: int, seed: int, thr32: int):
    x = np.ascontiguousarray(x)
    dims = _dims(x)
    c = consts_for(x, eb)
    nt, nv = count_samples(tuple(dims), block, seed, thr32)
    tin = np.zeros((max(nt, 1), k), np.int32); ttg = np.zeros(max(nt, 1), np.int32); tus = np.zeros(max(nt, 1), np.uint8)
    vin = np.zeros((max(nv, 1), k), np.int32); vtg = np.zeros(max(nv, 1), np.int32); vus = np.zeros(max(nv, 1), np.uint8)
    b = (C.c_int * 3)(*block)
    st = lib().orc_gather_samples(_p(x), dims, _dtype_code(x), C.byref(c), b, k, seed, thr32,
                                  _p(tin), _p(ttg), _p(tus), _p(vin), _p(vtg), _p(vus))
    assert st == 0
    return (tin[:nt], ttg[:nt], tus[:nt]), (vin[:nv], vtg[:nv], vus[:nv])


def input_shift(tg: np.ndarray, use: np.ndarray) -> int:
    tg = np.ascontiguousarray(tg, np.int32); use = np.ascontiguousarray(use, np.uint8)
    return lib().orc_input_shift(_p(tg), _p(use), tg.size)


def init_weights(k, h1, h2, seed) -> np.ndarray:
    w = np.zeros(mlp_nweights(k, h1, h2), np.float32)
    lib().orc_init_weights(_p(w), k, h1, h2, seed)
    return w


def batch_grad(w, k, h1, h2, s_in, inp, tg, use) -> np.ndarray:
    w = np.ascontiguousarray(w, np.float32)
    inp = np.ascontiguousarray(inp, np.int32); tg = np.ascontiguousarray(tg, np.int32)
    use = np.ascontiguousarray(use, np.uint8)
    B = tg.size
    assert 1 <= B <= BATCH
    g = np.zeros_like(w)
    lib().orc_batch_grad(_p(w), k, h1, h2, s_in, _p(inp), _p(tg), _p(use), B, _p(g))
    return g


def sgd_update(w, g, k, h1, h2, lr, lam) -> np.ndarray:
    w = np.array(w, np.float32, copy=True)
    g = np.ascontiguousarray(g, np.float32)
    lib().orc_sgd_update(_p(w), _p(g), k, h1, h2, lr, lam)
    return w


def train_epoch(w, k, h1, h2, s_in, inp, tg, use, lr, lam, max_steps=None) -> np.ndarray:
    w = np.array(w, np.float32, copy=True)
    inp = np.ascontiguousarray(inp, np.int32); tg = np.ascontiguousarray(tg, np.int32)
    use = np.ascontiguousarray(use, np.uint8)
    ms = (1 << 64) - 1 if max_steps is None else int(max_steps)
    lib().orc_train_epoch(_p(w), k, h1, h2, s_in, _p(inp), _p(tg), _p(use), tg.size, lr, lam, ms)
    return w


def val_cost(w, k, h1, h2, s_in, inp, tg, use, m=16) -> int:
    inp = np.ascontiguousarray(inp, np.int32); tg = np.ascontiguousarray(tg, np.int32)
    use = np.ascontiguousarray(use, np.uint8)
    wp = None if w is None else _p(np.ascontiguousarray(w, np.float32))
    return lib().orc_val_cost(wp, k, h1, h2, s_in, _p(inp), _p(tg), _p(use), tg.size, m)


def val_size(w, k, h1, h2, s_in, inp, tg, use, m=16, value_bits=32) -> int:
    """Simulated compressed size (bits) of a predictor on validation samples (Section IV.C)."""
    inp = np.ascontiguousarray(inp, np.int32); tg = np.ascontiguousarray(tg, np.int32)
    use = np.ascontiguousarray(use, np.uint8)
    wp = None if w is None else _p(np.ascontiguousarray(w, np.float32))
    return lib().orc_val_size(wp, k, h1, h2, s_in, _p(inp), _p(tg), _p(use), tg.size, m, value_bits)


def val_hist(w, k, h1, h2, s_in, inp, tg, use, m=16) -> np.ndarray:
    """Validation histogram of one predictor (w None: Lorenzo) at m code bits."""
    inp = np.ascontiguousarray(inp, np.int32); tg = np.ascontiguousarray(tg, np.int32)
    use = np.ascontiguousarray(use, np.uint8)
    wp = None if w is None else _p(np.ascontiguousarray(w, np.float32))
    h = np.zeros(1 << m, np.uint64)
    lib().orc_val_hist(wp, k, h1, h2, s_in, _p(inp), _p(tg), _p(use), tg.size, m, _p(h))
    return h


def sample_codebook(hist, m=16, span_fill=False) -> np.ndarray:
    """The training phase's Huffman code from a validation histogram: uint32 list
    (sym | len << 16) in container order.  span_fill: every code inside the sampled span
    gets a code word."""
    h = np.ascontiguousarray(hist, np.uint64)
    assert h.size == 1 << m
    out = np.zeros(1 << m, np.uint32)
    n = lib().orc_sample_codebook(_p(h), m, int(bool(span_fill)), _p(out))
    return out[:n].copy()


def sample_codebook_for(x: np.ndarray, eb: float, block=(8, 8, 8), k=7, h1=16, h2=16, s_in=0, weights=None, m=16,
                        seed=0, thr32=None, span_fill=False) -> np.ndarray:
    """Sample codebook of field x for the FP32 weights (None: Lorenzo), validation samples drawn
    as the training phase draws them."""
    x = np.ascontiguousarray(x)
    if thr32 is None:
        thr32 = int(0.1 * 2 ** 32)
    w = None if weights is None else np.ascontiguousarray(weights, np.float32)
    out = np.zeros(1 << m, np.uint32)
    b = (C.c_int * 3)(*block)
    n = lib().orc_sample_codebook_for(_p(x), _dims(x), _dtype_code(x), eb, b, k, h1, h2, s_in,
                                      None if w is None else _p(w), m, seed, thr32, int(bool(span_fill)), _p(out))
    assert n > 0, n
    return out[:n].copy()


def lz_encode(data: bytes) -> bytes:
    """The lossless stage's section for a byte string (length a multiple of 4)."""
    src = np.frombuffer(bytes(data), np.uint8).copy()
    cap = lib().orc_lz_bound(src.size)
    out = np.zeros(cap, np.uint8)
    n = lib().orc_lz_encode(_p(src) if src.size else None, src.size, _p(out))
    return out[:n].tobytes()


def lz_decode(section: bytes, raw_bytes: int):
    """Inverse of lz_encode: (status, bytes)."""
    sec = np.frombuffer(bytes(section), np.uint8).copy()
    out = np.zeros(max(raw_bytes, 1), np.uint8)
    st = lib().orc_lz_decode(_p(sec), sec.size, _p(out), raw_bytes)
    return st, out[:raw_bytes].tobytes()


def coverage_m(w, k, h1, h2, s_in, inp, tg, use, eb) -> int:
    inp = np.ascontiguousarray(inp, np.int32); tg = np.ascontiguousarray(tg, np.int32)
    use = np.ascontiguousarray(use, np.uint8)
    wp = None if w is None else _p(np.ascontiguousarray(w, np.float32))
    return lib().orc_coverage_m(wp, k, h1, h2, s_in, _p(inp), _p(tg), _p(use), tg.size, eb)


def train_select(x: np.ndarray, eb: float, block=(8, 8, 8), k=7, h1=16, h2=16, m=16, seed=0, thr32=None,
                 lrs=None, lams=None):
    """Training phase with selection by simulated compression and the coverage rule for m.
    Returns (chosen index or -1, weights [H, nw], s_in, simulated sizes [H + 1], m)."""
    x = np.ascontiguousarray(x)
    if thr32 is None:
        thr32 = int(0.1 * 2 ** 32)
    if lrs is None:
        lrs, lams = default_grid()
    lrs = np.ascontiguousarray(lrs, np.float32); lams = np.ascontiguousarray(lams, np.float32)
    H = lrs.size
    W = np.zeros((H, mlp_nweights(k, h1, h2)), np.float32)
    sizes = np.zeros(H + 1, np.uint64)
    s_in, m_out = C.c_int(), C.c_int()
    b = (C.c_int * 3)(*block)
    best = lib().orc_train_select(_p(x), _dims(x), _dtype_code(x), eb, b, k, h1, h2, m, seed, thr32, H, _p(lrs),
                                  _p(lams), _p(W), C.byref(s_in), _p(sizes), C.byref(m_out))
    return best, W, s_in.value, sizes, m_out.value


DEFAULT_LRS = [3e-3, 1e-2, 3e-2, 1e-1]
DEFAULT_LAMS = [0.0, 1e-5, 1e-4, 1e-3]


def default_grid():
    lrs = np.array([lr for lr in DEFAULT_LRS for _ in DEFAULT_LAMS], np.float32)
    lams = np.array([lm for _ in DEFAULT_LRS for lm in DEFAULT_LAMS], np.float32)
    return lrs, lams


def train(x: np.ndarray, eb: float, block=(8, 8, 8), k=7, h1=16, h2=16, m=16, seed=0,
          thr32=None, lrs=None, lams=None):
    """Full training phase.  Returns (chosen index or -1, weights [H, nw], s_in, costs [H+1])."""
    x = np.ascontiguousarray(x)
    dims = _dims(x)
    if thr32 is None:
        thr32 = int(0.1 * 2 ** 32)
    if lrs is None:
        lrs, lams = default_grid()
    lrs = np.ascontiguousarray(lrs, np.float32); lams = np.ascontiguousarray(lams, np.float32)
    H = lrs.size
    nw = mlp_nweights(k, h1, h2)
    W = np.zeros((H, nw), np.float32)
    costs = np.zeros(H + 1, np.uint64)
    s_in = C.c_int()
    b = (C.c_int * 3)(*block)
    best = lib().orc_train(_p(x), dims, _dtype_code(x), eb, b, k, h1, h2, m, seed, thr32, H,
                           _p(lrs), _p(lams), _p(W), C.byref(s_in), _p(costs))
    return best, W, s_in.value, costs
