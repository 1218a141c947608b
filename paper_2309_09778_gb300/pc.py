"""Python binding of the C ABI in include/pc.h (argument marshalling only).

Every function here has the name of the C entry point it calls and only turns
torch tensors / numpy arrays into pointers and sizes; every step of the method
runs in the CUDA library.  PyTorch supplies device memory and streams.  If the
library has not been built the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpc.so")
_lib = None
_lock = threading.Lock()

PC_F32, PC_F64 = 0, 1
PC_PRED_LORENZO, PC_PRED_MLP_FP32, PC_PRED_MLP_BF16 = 0, 1, 2
STATUS = {0: "PC_OK", -1: "PC_ERR_ARG", -2: "PC_ERR_DTYPE", -3: "PC_ERR_NONFINITE", -4: "PC_ERR_CAPACITY",
          -5: "PC_ERR_CORRUPT", -6: "PC_ERR_TIMEOUT", -7: "PC_ERR_CUDA", -8: "PC_ERR_EB_RANGE"}
SYMBOLS = ["pc_mlp_nweights", "pc_compress_bound", "pc_compress_workspace_size", "pc_compress",
           "pc_header_info", "pc_decompress", "pc_decompress_noalloc", "pc_compress_host", "pc_decompress_host",
           "pc_train_workspace_size", "pc_train", "pc_compress_workspace_layout", "pc_profile_enable",
           "pc_profile_read", "pc_profile_stage_name", "pc_strerror", "pc_compress_batch_workspace_size",
           "pc_compress_batch", "pc_decompress_batch_workspace_size", "pc_decompress_batch", "pc_train_select"]


# (lr, lambda) grid trained side by side in the training phase (Section IV.C
# trains several hyperparameter sets concurrently and keeps the best); the
# paper gives no values, these are ours.
DEFAULT_LRS = (3e-3, 1e-2, 3e-2, 1e-1)
DEFAULT_LAMS = (0.0, 1e-5, 1e-4, 1e-3)


def default_grid():
    lrs = np.array([lr for lr in DEFAULT_LRS for _ in DEFAULT_LAMS], np.float32)
    lams = np.array([lm for _ in DEFAULT_LRS for lm in DEFAULT_LAMS], np.float32)
    return lrs, lams


class PcError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


class pc_params(C.Structure):
    _fields_ = [("eb_rel", C.c_double), ("block", C.c_int * 3), ("pred", C.c_int), ("stencil", C.c_int),
                ("hidden", C.c_int * 2), ("m", C.c_int), ("s_in", C.c_int), ("h_weights", C.c_void_p),
                ("h_qnet", C.c_void_p), ("seed", C.c_ulonglong), ("train_samples", C.c_longlong),
                ("ndims", C.c_int), ("codebook_n", C.c_int), ("h_codebook", C.c_void_p), ("literal", C.c_int),
                ("eq_period", C.c_int), ("lossless", C.c_int)]


def lib():
    """Load libpc.so (built by __graft_entry__.build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
            L = C.CDLL(LIB_PATH)
            sz = C.c_size_t
            szp = C.POINTER(C.c_size_t)
            vp = C.c_void_p
            P = C.POINTER(pc_params)
            L.pc_mlp_nweights.restype = C.c_int
            L.pc_mlp_nweights.argtypes = [C.c_int, C.c_int, C.c_int]
            L.pc_compress_bound.restype = sz
            L.pc_compress_bound.argtypes = [szp, C.c_int, P]
            L.pc_compress_workspace_size.restype = C.c_int
            L.pc_compress_workspace_size.argtypes = [szp, C.c_int, P, szp]
            L.pc_compress_workspace_layout.restype = C.c_int
            L.pc_compress_workspace_layout.argtypes = [szp, C.c_int, P, szp, szp, szp]
            L.pc_compress.restype = C.c_int
            L.pc_compress.argtypes = [vp, szp, C.c_int, P, vp, sz, szp, vp, sz, vp]
            L.pc_header_info.restype = C.c_int
            L.pc_header_info.argtypes = [vp, sz, szp, C.POINTER(C.c_int), szp]
            L.pc_decompress.restype = C.c_int
            L.pc_decompress.argtypes = [vp, sz, vp, sz, szp, C.POINTER(C.c_int), vp, sz, vp]
            L.pc_decompress_noalloc.restype = C.c_int
            L.pc_decompress_noalloc.argtypes = [vp, sz, vp, sz, szp, C.POINTER(C.c_int), vp]
            L.pc_compress_host.restype = C.c_int
            L.pc_compress_host.argtypes = [vp, szp, C.c_int, P, vp, sz, szp, vp, vp, sz, vp, sz, vp]
            L.pc_decompress_host.restype = C.c_int
            L.pc_decompress_host.argtypes = [vp, sz, vp, sz, szp, C.POINTER(C.c_int), vp, sz, vp, vp, sz, vp]
            if hasattr(L, "pc_train"):
                L.pc_train_workspace_size.restype = C.c_int
                L.pc_train_workspace_size.argtypes = [szp, C.c_int, P, C.c_uint, C.c_int, szp]
                L.pc_train.restype = C.c_int
                L.pc_train.argtypes = [vp, szp, C.c_int, P, C.c_ulonglong, C.c_uint, C.c_int, vp, vp, vp,
                                       C.POINTER(C.c_int), C.POINTER(C.c_int), vp, vp, sz, vp]
            if hasattr(L, "pc_train_select"):
                L.pc_sample_codebook.restype = C.c_int
                L.pc_sample_codebook.argtypes = [vp, szp, C.c_int, P, C.c_ulonglong, C.c_uint, C.c_int, vp,
                                                 C.POINTER(C.c_int), vp, sz, vp]
                L.pc_train_select.restype = C.c_int
                L.pc_train_select.argtypes = [vp, szp, C.c_int, P, C.c_ulonglong, C.c_uint, C.c_int, vp, vp, vp,
                                              C.POINTER(C.c_int), C.POINTER(C.c_int), vp, C.POINTER(C.c_int), vp, sz,
                                              vp]
            if hasattr(L, "pc_quantize"):
                L.pc_qnet_len.restype = C.c_int
                L.pc_qnet_len.argtypes = [C.c_int, C.c_int, C.c_int]
                L.pc_quantize.restype = C.c_int
                L.pc_quantize.argtypes = [vp, szp, C.c_int, P, C.c_ulonglong, C.c_uint, vp, vp, sz, vp]
            L.pc_compress_batch_workspace_size.restype = C.c_int
            L.pc_compress_batch_workspace_size.argtypes = [C.c_int, szp, C.POINTER(C.c_int), P, szp, szp]
            L.pc_compress_batch.restype = C.c_int
            L.pc_compress_batch.argtypes = [C.c_int, C.POINTER(C.c_void_p), szp, C.POINTER(C.c_int), P, vp, sz, szp,
                                            szp, vp, sz, vp]
            L.pc_decompress_batch_workspace_size.restype = C.c_int
            L.pc_decompress_batch_workspace_size.argtypes = [C.c_int, C.POINTER(C.c_void_p), szp]
            L.pc_decompress_batch.restype = C.c_int
            L.pc_decompress_batch.argtypes = [C.c_int, vp, szp, szp, C.POINTER(C.c_void_p), szp, vp, sz, vp]
            L.pc_profile_enable.restype = C.c_int
            L.pc_profile_enable.argtypes = [C.c_int]
            L.pc_profile_read.restype = C.c_int
            L.pc_profile_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]
            L.pc_profile_stage_name.restype = C.c_char_p
            L.pc_profile_stage_name.argtypes = [C.c_int]
            L.pc_strerror.restype = C.c_char_p
            L.pc_strerror.argtypes = [C.c_int]
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != 0:
        raise PcError(st, where)


def _dims3(shape):
    shp = [int(s) for s in shape]
    while len(shp) < 3:
        shp.insert(0, 1)
    if len(shp) != 3:
        raise ValueError("fields are 1-D, 2-D or 3-D")
    return (C.c_size_t * 3)(*shp)


def _dtype_of(t) -> int:
    s = str(t.dtype)
    if s.endswith("float32"):
        return PC_F32
    if s.endswith("float64"):
        return PC_F64
    raise TypeError("float32 or float64 field expected")


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def make_params(eb_rel: float, block=(8, 8, 8), pred: int = PC_PRED_LORENZO, stencil: int = 7,
                hidden=(16, 16), m: int = 16, s_in: int = 0, weights=None, qnet=None, seed: int = 0,
                train_samples: int = 0, ndims: int = 0, codebook=None, literal: bool = False, eq_period: int = 0,
                lossless: bool = False):
    """Fill a pc_params struct; the weights, network and codebook arrays are kept alive on the
    struct.  With a perceptron form and no weights (or network), pc_compress trains one on the
    device; with a codebook (uint32 list from pc_sample_codebook) it compresses in one pass."""
    p = pc_params()
    p.literal = int(bool(literal))
    p.eq_period = int(eq_period)
    p.lossless = int(bool(lossless))
    p.seed = int(seed)
    p.train_samples = int(train_samples)
    p.ndims = int(ndims)
    if codebook is not None:
        cb = np.ascontiguousarray(np.asarray(codebook, dtype=np.uint32))
        p._cb = cb
        p.h_codebook = cb.ctypes.data
        p.codebook_n = int(cb.size)
    else:
        p.h_codebook = None
        p.codebook_n = 0
    p.eb_rel = float(eb_rel)
    p.block[:] = [int(b) for b in block]
    p.pred = int(pred)
    p.stencil = int(stencil)
    p.hidden[:] = [int(h) for h in hidden]
    p.m = int(m)
    p.s_in = int(s_in)
    if weights is not None:
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
        p._w = w
        p.h_weights = w.ctypes.data
    else:
        p.h_weights = None
    if qnet is not None:
        q = np.ascontiguousarray(np.asarray(qnet, dtype=np.int64))
        p._q = q
        p.h_qnet = q.ctypes.data
    else:
        p.h_qnet = None
    return p


def pc_mlp_nweights(k: int, h1: int, h2: int) -> int:
    return lib().pc_mlp_nweights(k, h1, h2)


def pc_compress_bound(shape, dtype: int, params: pc_params) -> int:
    return int(lib().pc_compress_bound(_dims3(shape), dtype, C.byref(params)))


def pc_compress_workspace_size(shape, dtype: int, params: pc_params) -> int:
    ws = C.c_size_t()
    _check(lib().pc_compress_workspace_size(_dims3(shape), dtype, C.byref(params), C.byref(ws)),
           "pc_compress_workspace_size")
    return ws.value


def pc_compress_workspace_layout(shape, dtype: int, params: pc_params):
    a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
    _check(lib().pc_compress_workspace_layout(_dims3(shape), dtype, C.byref(params), C.byref(a), C.byref(b),
                                              C.byref(c)), "pc_compress_workspace_layout")
    return a.value, b.value, c.value


def pc_compress(field, params: pc_params, out, ws, stream=None) -> int:
    """field: device tensor; out, ws: device uint8 tensors.  Returns bytes written."""
    size = C.c_size_t()
    st = lib().pc_compress(C.c_void_p(field.data_ptr()), _dims3(field.shape), _dtype_of(field), C.byref(params),
                           C.c_void_p(out.data_ptr()), out.numel(), C.byref(size), C.c_void_p(ws.data_ptr()),
                           ws.numel(), _stream_ptr(stream))
    _check(st, "pc_compress")
    return size.value


def pc_header_info(header: bytes):
    buf = np.frombuffer(bytes(header[:256]), np.uint8).copy()
    dims = (C.c_size_t * 3)()
    dt = C.c_int()
    ws = C.c_size_t()
    _check(lib().pc_header_info(buf.ctypes.data_as(C.c_void_p), buf.size, dims, C.byref(dt), C.byref(ws)),
           "pc_header_info")
    return tuple(dims), dt.value, ws.value


def pc_decompress(blob, in_size: int, out, ws, stream=None):
    """blob: device uint8 tensor holding in_size bytes; out: device tensor with room for the field."""
    dims = (C.c_size_t * 3)()
    dt = C.c_int()
    st = lib().pc_decompress(C.c_void_p(blob.data_ptr()), int(in_size), C.c_void_p(out.data_ptr()),
                             out.numel() * out.element_size(), dims, C.byref(dt), C.c_void_p(ws.data_ptr()),
                             ws.numel(), _stream_ptr(stream))
    _check(st, "pc_decompress")
    return tuple(dims), dt.value


def pc_decompress_noalloc(blob, in_size: int, out, stream=None):
    """Decompress without a caller workspace (fixed built-in scratch, see include/pc.h)."""
    dims = (C.c_size_t * 3)()
    dt = C.c_int()
    st = lib().pc_decompress_noalloc(C.c_void_p(blob.data_ptr()), int(in_size), C.c_void_p(out.data_ptr()),
                                     out.numel() * out.element_size(), dims, C.byref(dt), _stream_ptr(stream))
    _check(st, "pc_decompress_noalloc")
    return tuple(dims), dt.value


def pc_compress_host(h_field: np.ndarray, params: pc_params, h_out: np.ndarray, d_field_stage, d_out_stage, ws,
                     stream=None) -> int:
    size = C.c_size_t()
    st = lib().pc_compress_host(h_field.ctypes.data_as(C.c_void_p), _dims3(h_field.shape), _dtype_of(h_field),
                                C.byref(params), h_out.ctypes.data_as(C.c_void_p), h_out.nbytes, C.byref(size),
                                C.c_void_p(d_field_stage.data_ptr()), C.c_void_p(d_out_stage.data_ptr()),
                                d_out_stage.numel(), C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream))
    _check(st, "pc_compress_host")
    return size.value


def pc_decompress_host(h_in: np.ndarray, in_size: int, h_field: np.ndarray, d_in_stage, d_field_stage, ws,
                       stream=None):
    dims = (C.c_size_t * 3)()
    dt = C.c_int()
    st = lib().pc_decompress_host(h_in.ctypes.data_as(C.c_void_p), int(in_size), h_field.ctypes.data_as(C.c_void_p),
                                  h_field.nbytes, dims, C.byref(dt), C.c_void_p(d_in_stage.data_ptr()),
                                  d_in_stage.numel(), C.c_void_p(d_field_stage.data_ptr()), C.c_void_p(ws.data_ptr()),
                                  ws.numel(), _stream_ptr(stream))
    _check(st, "pc_decompress_host")
    return tuple(dims), dt.value


def pc_train_workspace_size(shape, dtype: int, params: pc_params, thr32: int, nmodels: int) -> int:
    ws = C.c_size_t()
    _check(lib().pc_train_workspace_size(_dims3(shape), dtype, C.byref(params), int(thr32), int(nmodels),
                                         C.byref(ws)), "pc_train_workspace_size")
    return ws.value


def pc_train(field, params: pc_params, seed: int, thr32: int, lrs, lams, ws, stream=None):
    """Returns (weights [nmodels, nw] float32, s_in, chosen index or -1, costs [nmodels + 1])."""
    lrs = np.ascontiguousarray(lrs, np.float32)
    lams = np.ascontiguousarray(lams, np.float32)
    H = lrs.size
    nw = pc_mlp_nweights(params.stencil, params.hidden[0], params.hidden[1])
    W = np.zeros((H, nw), np.float32)
    costs = np.zeros(H + 1, np.uint64)
    s_in = C.c_int()
    chosen = C.c_int()
    st = lib().pc_train(C.c_void_p(field.data_ptr()), _dims3(field.shape), _dtype_of(field), C.byref(params),
                        int(seed), int(thr32), H, lrs.ctypes.data_as(C.c_void_p), lams.ctypes.data_as(C.c_void_p),
                        W.ctypes.data_as(C.c_void_p), C.byref(s_in), C.byref(chosen),
                        costs.ctypes.data_as(C.c_void_p), C.c_void_p(ws.data_ptr()), ws.numel(),
                        _stream_ptr(stream))
    _check(st, "pc_train")
    return W, s_in.value, chosen.value, costs


def pc_train_select(field, params: pc_params, seed: int, thr32: int, lrs, lams, ws, stream=None):
    """Training with selection by simulated compression and the coverage rule for m.
    Returns (weights [nmodels, nw], s_in, chosen or -1, simulated sizes [nmodels + 1], m)."""
    lrs = np.ascontiguousarray(lrs, np.float32)
    lams = np.ascontiguousarray(lams, np.float32)
    H = lrs.size
    nw = pc_mlp_nweights(params.stencil, params.hidden[0], params.hidden[1])
    W = np.zeros((H, nw), np.float32)
    sizes = np.zeros(H + 1, np.uint64)
    s_in, chosen, m = C.c_int(), C.c_int(), C.c_int()
    st = lib().pc_train_select(C.c_void_p(field.data_ptr()), _dims3(field.shape), _dtype_of(field), C.byref(params),
                               int(seed), int(thr32), H, lrs.ctypes.data_as(C.c_void_p),
                               lams.ctypes.data_as(C.c_void_p), W.ctypes.data_as(C.c_void_p), C.byref(s_in),
                               C.byref(chosen), sizes.ctypes.data_as(C.c_void_p), C.byref(m),
                               C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream))
    _check(st, "pc_train_select")
    return W, s_in.value, chosen.value, sizes, m.value


def pc_sample_codebook(field, params: pc_params, seed: int, thr32: int, ws, stream=None,
                       span_fill: bool = False) -> np.ndarray:
    """Sample codebook of the training phase for params' predictor (FP32 weights, or Lorenzo):
    uint32 list (sym | length << 16) in container order.  span_fill: every code inside the
    sampled span gets a code word."""
    out = np.zeros(1 << params.m, np.uint32)
    n = C.c_int()
    st = lib().pc_sample_codebook(C.c_void_p(field.data_ptr()), _dims3(field.shape), _dtype_of(field),
                                  C.byref(params), int(seed), int(thr32), int(bool(span_fill)),
                                  out.ctypes.data_as(C.c_void_p),
                                  C.byref(n), C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream))
    _check(st, "pc_sample_codebook")
    return out[: n.value].copy()


def pc_qnet_len(k: int, h1: int, h2: int) -> int:
    return lib().pc_qnet_len(k, h1, h2)


def pc_quantize(field, params: pc_params, seed: int, thr32: int, ws, stream=None) -> np.ndarray:
    """Fixed-point (BF16) network from params' FP32 weights and s_in; returns int64 [pc_qnet_len]."""
    q = np.zeros(pc_qnet_len(params.stencil, params.hidden[0], params.hidden[1]), np.int64)
    st = lib().pc_quantize(C.c_void_p(field.data_ptr()), _dims3(field.shape), _dtype_of(field), C.byref(params),
                           int(seed), int(thr32), q.ctypes.data_as(C.c_void_p), C.c_void_p(ws.data_ptr()),
                           ws.numel(), _stream_ptr(stream))
    _check(st, "pc_quantize")
    return q


def _batch_args(fields, params):
    n = len(fields)
    dims = (C.c_size_t * (3 * n))(*[d for f in fields for d in _dims3(f.shape)])
    dts = (C.c_int * n)(*[_dtype_of(f) for f in fields])
    ps = (pc_params * n)(*params)
    return n, dims, dts, ps


def pc_compress_batch_workspace_size(fields, params):
    """(workspace bytes, output bytes) of a batched compression of these fields."""
    n, dims, dts, ps = _batch_args(fields, params)
    ws, ob = C.c_size_t(), C.c_size_t()
    _check(lib().pc_compress_batch_workspace_size(n, dims, dts, ps, C.byref(ws), C.byref(ob)),
           "pc_compress_batch_workspace_size")
    return ws.value, ob.value


def pc_compress_batch(fields, params, out, ws, stream=None):
    """Compress device tensors `fields` (each with its pc_params) into the uint8 device buffer `out`.
    Returns (offsets [n + 1], sizes [n])."""
    n, dims, dts, ps = _batch_args(fields, params)
    ptrs = (C.c_void_p * n)(*[f.data_ptr() for f in fields])
    offs = (C.c_size_t * (n + 1))()
    sizes = (C.c_size_t * n)()
    st = lib().pc_compress_batch(n, ptrs, dims, dts, ps, C.c_void_p(out.data_ptr()), out.numel(), offs, sizes,
                                 C.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream))
    _check(st, "pc_compress_batch")
    return list(offs), list(sizes)


def pc_decompress_batch_workspace_size(headers):
    """headers: list of 256-byte host copies of the containers' headers."""
    bufs = [np.frombuffer(bytes(h[:256]), np.uint8).copy() for h in headers]
    ptrs = (C.c_void_p * len(bufs))(*[b.ctypes.data for b in bufs])
    ws = C.c_size_t()
    _check(lib().pc_decompress_batch_workspace_size(len(bufs), ptrs, C.byref(ws)), "pc_decompress_batch_workspace_size")
    return ws.value


def pc_decompress_batch(blob, offsets, sizes, outs, ws, stream=None):
    n = len(outs)
    offs = (C.c_size_t * n)(*offsets[:n])
    szs = (C.c_size_t * n)(*sizes)
    ptrs = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    caps = (C.c_size_t * n)(*[o.numel() * o.element_size() for o in outs])
    st = lib().pc_decompress_batch(n, C.c_void_p(blob.data_ptr()), offs, szs, ptrs, caps, C.c_void_p(ws.data_ptr()),
                                   ws.numel(), _stream_ptr(stream))
    _check(st, "pc_decompress_batch")


def pc_profile_enable(on: bool) -> None:
    _check(lib().pc_profile_enable(1 if on else 0), "pc_profile_enable")


def pc_profile_read() -> dict:
    """Per-stage device milliseconds and launch counts since the last read."""
    ms = (C.c_double * 32)()
    n = (C.c_longlong * 32)()
    k = lib().pc_profile_read(ms, n, 32)
    return {lib().pc_profile_stage_name(i).decode(): (ms[i], n[i]) for i in range(k)}


def pc_strerror(status: int) -> str:
    return lib().pc_strerror(int(status)).decode()


# ---------------------------------------------------------------- convenience
def compress(field, params: pc_params, stream=None):
    """Allocate output and workspace with torch, compress, return the exact-size device blob."""
    import torch
    dt = _dtype_of(field)
    cap = pc_compress_bound(field.shape, dt, params)
    if cap == 0:
        raise PcError(-1, "pc_compress_bound")
    out = torch.empty(cap, dtype=torch.uint8, device=field.device)
    ws = torch.empty(pc_compress_workspace_size(field.shape, dt, params), dtype=torch.uint8, device=field.device)
    n = pc_compress(field, params, out, ws, stream)
    return out[:n]


def decompress(blob, stream=None):
    """Decompress a device blob; returns a device tensor of the stored shape and dtype."""
    import torch
    hdr = blob[:256].cpu().numpy().tobytes()
    dims, dt, wsb = pc_header_info(hdr)
    out = torch.empty(tuple(dims), dtype=torch.float32 if dt == PC_F32 else torch.float64, device=blob.device)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=blob.device)
    pc_decompress(blob, blob.numel(), out, ws, stream)
    return out
