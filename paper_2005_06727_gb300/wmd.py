"""Thin Python binding of the C ABI in ``include/wmd.h`` (ctypes).

This module only marshals arguments: every step of the method runs in the
CUDA library ``libwmd_gb300.so``.  There is no CPU fallback; if the library is
missing the import of a function raises :class:`WMDError`.

Names follow the C entry points: ``corpus_load`` / :class:`Corpus`,
``Corpus.query`` (``wmd_query``), ``Corpus.query_device``
(``wmd_query_device``), ``Corpus.query_device_tol`` (``wmd_query_device_tol``),
``Corpus.query_device_topk`` and ``topk`` (``wmd_query_device_topk``,
``wmd_topk``), ``Corpus.query_dense`` (``wmd_query_dense``),
``Corpus.build_kernel_matrix``, ``Corpus.sinkhorn_loop``, ``query_batch``,
:class:`Server` and ``compact_query``.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwmd_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "wmd.h")

WMD_OK = 0
WMD_ERR_INVALID_ARG = 1
WMD_ERR_OUT_OF_MEMORY = 2
WMD_ERR_CUDA = 3
WMD_ERR_NOT_READY = 4
WMD_ERR_TIMEOUT = 5
WMD_ERR_SHUTDOWN = 6
WMD_ERR_UNSUPPORTED = 7
WMD_ERR_RANGE = 8

CDIST_TENSOR_CORES = 0
CDIST_CUDA_CORES = 1

PREC_FP32 = 0
PREC_BF16_K = 1
MAX_VR = 256

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "NOT_READY",
           5: "TIMEOUT", 6: "SHUTDOWN", 7: "UNSUPPORTED", 8: "RANGE"}


class WMDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"wmd status {_STATUS.get(status, status)}: {msg}")
        self.status = status


class ServerOptions(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("slots", C.c_int32), ("mem_budget", C.c_size_t),
                ("max_pending", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("cancelled", C.c_int64),
                ("batches", C.c_int64), ("max_batch_seen", C.c_int64), ("pending", C.c_int64),
                ("in_flight_batches", C.c_int64)]


class CorpusInfo(C.Structure):
    _fields_ = [("V", C.c_int64), ("d", C.c_int32), ("N", C.c_int64), ("nnz", C.c_int64),
                ("U", C.c_int64), ("device", C.c_int32), ("device_bytes", C.c_size_t),
                ("cdist_kernel", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("device", C.c_int32), ("use_graphs", C.c_int32), ("cdist_kernel", C.c_int32),
                ("autotune_cache", C.c_char_p), ("wait_limit_cycles", C.c_int64),
                ("server", ServerOptions)]


_lib = None

_P = C.c_void_p
_SIGS = {
    "wmd_last_error": (C.c_char_p, []),
    "wmd_version": (C.c_char_p, []),
    "wmd_measure_fp32_peak": (C.c_int, [C.c_int32, C.c_int32, _P]),
    "wmd_compact_query": (C.c_int, [_P, _P, C.c_int32, C.c_int64, _P, _P, _P]),
    "wmd_options_default": (None, [_P]),
    "wmd_corpus_load": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P, C.c_int64, C.c_int64,
                                  _P, _P]),
    "wmd_corpus_free": (None, [_P]),
    "wmd_shard_plan": (C.c_int, [_P, _P, C.c_int64, C.c_int64, C.c_int32, _P]),
    "wmd_corpus_load_shard": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P, C.c_int64, C.c_int64,
                                        C.c_int64, C.c_int64, _P, _P]),
    "wmd_corpus_get_info": (C.c_int, [_P, _P]),
    "wmd_corpus_set_wait_limit": (C.c_int, [_P, C.c_int64]),
    "wmd_query": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, C.c_int, _P]),
    "wmd_workspace_bytes": (C.c_size_t, [_P, C.c_int32, C.c_int]),
    "wmd_build_kernel_matrix": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int, _P,
                                          C.c_size_t, _P]),
    "wmd_sinkhorn_loop": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int, _P, C.c_size_t, _P, _P]),
    "wmd_query_device": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, C.c_int, _P,
                                   C.c_size_t, _P, _P]),
    "wmd_query_device_tol": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, C.c_float,
                                       C.c_int, _P, C.c_size_t, _P, _P, _P]),
    "wmd_topk": (C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P]),
    "wmd_query_device_topk": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, C.c_int, _P,
                                        C.c_size_t, _P, C.c_int32, _P, _P, _P]),
    "wmd_dense_workspace_bytes": (C.c_size_t, [_P, C.c_int32]),
    "wmd_dense_load_c": (C.c_int, [_P, _P, C.c_size_t, _P]),
    "wmd_query_dense": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, _P, C.c_size_t, _P,
                                  _P]),
    "wmd_query_device_noalloc": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, C.c_int,
                                           _P, _P]),
    "wmd_query_batch": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, C.c_int32, C.c_int, _P]),
    "wmd_loop_width": (C.c_int32, [C.c_int32]),
    "wmd_loop_variant_count": (C.c_int32, [C.c_int32]),
    "wmd_set_loop_variant": (C.c_int, [_P, C.c_int32, C.c_int, C.c_int32]),
    "wmd_get_loop_variant": (C.c_int32, [_P, C.c_int32, C.c_int]),
    "wmd_set_loop_partition": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32]),
    "wmd_get_loop_partition": (C.c_int32, [_P, C.c_int32, C.c_int32]),
    "wmd_autotune": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, C.c_int, _P]),
    "wmd_server_create": (C.c_int, [_P, _P, _P]),
    "wmd_serve_submit": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.c_int32, C.c_int, _P]),
    "wmd_serve_poll": (C.c_int, [_P, C.c_uint64, _P, C.c_int64]),
    "wmd_serve_cancel": (C.c_int, [_P, C.c_uint64]),
    "wmd_server_get_stats": (C.c_int, [_P, _P]),
    "wmd_server_destroy": (None, [_P]),
}


def lib():
    """Load ``libwmd_gb300.so`` (built by ``paper_2005_06727_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise WMDError(WMD_ERR_CUDA, f"CUDA library not built: {LIB_PATH} is missing "
                                         "(run paper_2005_06727_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_functions() -> list[str]:
    """Names of the functions declared in include/wmd.h."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wmd_[a-z_0-9]+)\s*\(", src)))


def _check(st: int):
    if st != WMD_OK:
        raise WMDError(st, lib().wmd_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    # the raw address: the arguments are declared c_void_p, which takes an int;
    # a ctypes view of a writable contiguous buffer gives it in about half the
    # time of ndarray.ctypes (which builds a helper object on every access)
    if not a.size:
        return None
    try:
        return C.addressof(C.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):  # read-only or strided
        return a.ctypes.data


def measure_fp32_peak(device: int = 0, packed: bool = True) -> float:
    """``wmd_measure_fp32_peak``: the device's measured FP32 FMA rate in
    TFLOP/s (packed FFMA2 or scalar FFMA)."""
    out = C.c_double(0.0)
    _check(lib().wmd_measure_fp32_peak(int(device), 1 if packed else 0, C.byref(out)))
    return float(out.value)


def loop_width(v_r: int) -> int:
    """``wmd_loop_width``: the fused loop's tile width for v_r query words."""
    return int(lib().wmd_loop_width(int(v_r)))


def loop_variant_count(v_r: int) -> int:
    """``wmd_loop_variant_count``."""
    return int(lib().wmd_loop_variant_count(int(v_r)))


def compact_query(q_ids, q_w, V: int):
    """``wmd_compact_query``: drop zero weights (I = r > 0) and validate."""
    ids = np.ascontiguousarray(q_ids, dtype=np.int32)
    w = np.ascontiguousarray(q_w, dtype=np.float32)
    if ids.shape != w.shape:
        raise WMDError(WMD_ERR_INVALID_ARG, "ids and weights differ in length")
    out_ids = np.zeros(max(ids.size, 1), np.int32)
    out_w = np.zeros(max(ids.size, 1), np.float32)
    vr = C.c_int32(0)
    _check(lib().wmd_compact_query(_ptr(ids), _ptr(w), ids.size, V, _ptr(out_ids), _ptr(out_w),
                                   C.byref(vr)))
    return out_ids[:vr.value].copy(), out_w[:vr.value].copy()


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    """Device pointer of a torch tensor (or a raw int)."""
    if t is None:
        return None
    if isinstance(t, int):
        return C.c_void_p(t)
    return C.c_void_p(t.data_ptr())


def options(device: int = 0, use_graphs: bool = True, cdist_kernel: int = CDIST_TENSOR_CORES,
            autotune_cache: str | None = None, wait_limit_cycles: int = 0, **server) -> Options:
    """A ``wmd_options`` from ``wmd_options_default`` with the given fields
    (``server`` keywords: max_batch, slots, mem_budget, max_pending)."""
    o = Options()
    lib().wmd_options_default(C.byref(o))
    o.device = int(device)
    o.use_graphs = 1 if use_graphs else 0
    o.cdist_kernel = int(cdist_kernel)
    o.autotune_cache = autotune_cache.encode() if autotune_cache else None
    o.wait_limit_cycles = int(wait_limit_cycles)
    for k, v in server.items():
        if k not in {f for f, _ in ServerOptions._fields_}:
            raise TypeError(f"unknown option {k}")
        setattr(o.server, k, int(v))
    return o


class Corpus:
    """``wmd_corpus``: embeddings and the V x N CSR ``c`` resident on a GPU."""

    def __init__(self, vecs, row_ptr, doc_idx, val, N: int, device: int = 0, **opts):
        vecs = np.ascontiguousarray(vecs, dtype=np.float32)
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        doc_idx = np.ascontiguousarray(doc_idx, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float32)
        V, d = vecs.shape
        o = options(device=device, **opts)
        h = C.c_void_p()
        _check(lib().wmd_corpus_load(_ptr(vecs), V, d, _ptr(row_ptr), _ptr(doc_idx), _ptr(val),
                                     int(N), int(val.size), C.byref(o), C.byref(h)))
        self._adopt(h)

    @classmethod
    def _from_handle(cls, h):
        """A Corpus owning a handle returned by another loading call."""
        self = cls.__new__(cls)
        self._adopt(h)
        return self

    def _adopt(self, h):
        self._h = h
        info = CorpusInfo()
        _check(lib().wmd_corpus_get_info(self._h, C.byref(info)))
        self.V, self.d, self.N, self.nnz, self.U = info.V, info.d, info.N, info.nnz, info.U
        self.device = info.device
        self.device_bytes = info.device_bytes
        self.cdist_kernel = "tensor cores (tcgen05)" if info.cdist_kernel == CDIST_TENSOR_CORES \
            else "CUDA cores (float32 FMA)"

    @classmethod
    def from_synth(cls, vecs, corpus, device: int = 0, **opts):
        return cls(vecs, corpus.row_ptr, corpus.doc_idx, corpus.val, corpus.N, device, **opts)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().wmd_corpus_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- host path
    def query(self, q_ids, q_w, lam: float, max_iter: int, prec: int = PREC_FP32,
              out: np.ndarray | None = None) -> np.ndarray:
        """``wmd_query``: host buffers in, WMD[N] (float64) out."""
        ids = np.ascontiguousarray(q_ids, dtype=np.int32)
        w = np.ascontiguousarray(q_w, dtype=np.float32)
        if out is None:
            out = np.empty(self.N, np.float64)
        elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size < self.N:
            raise ValueError("out must be a C-contiguous float64 array of N values")
        _check(lib().wmd_query(self._h, _ptr(ids), _ptr(w), ids.size, float(lam), int(max_iter),
                               int(prec), _ptr(out)))
        return out

    def set_wait_limit(self, cycles: int):
        """``wmd_corpus_set_wait_limit`` (0 = the default, about 2 s)."""
        _check(lib().wmd_corpus_set_wait_limit(self._h, int(cycles)))

    def set_loop_variant(self, v_r: int, variant: int, prec: int = PREC_FP32):
        """``wmd_set_loop_variant``."""
        _check(lib().wmd_set_loop_variant(self._h, int(v_r), int(prec), int(variant)))

    def loop_variant(self, v_r: int, prec: int = PREC_FP32) -> int:
        """``wmd_get_loop_variant``."""
        return int(lib().wmd_get_loop_variant(self._h, int(v_r), int(prec)))

    def set_loop_partition(self, v_r: int, variant: int, fill: int):
        """``wmd_set_loop_partition``: team-size fill (50, 75, 100 or 200) of
        v_r's class and tile variant."""
        _check(lib().wmd_set_loop_partition(self._h, int(v_r), int(variant), int(fill)))

    def loop_partition(self, v_r: int, variant: int) -> int:
        """``wmd_get_loop_partition``."""
        return int(lib().wmd_get_loop_partition(self._h, int(v_r), int(variant)))

    def autotune(self, q_ids, q_w, lam: float, max_iter: int, prec: int = PREC_FP32) -> int:
        """``wmd_autotune``: returns the chosen fused-loop variant."""
        ids = np.ascontiguousarray(q_ids, dtype=np.int32)
        w = np.ascontiguousarray(q_w, dtype=np.float32)
        chosen = C.c_int32(-1)
        _check(lib().wmd_autotune(self._h, _ptr(ids), _ptr(w), ids.size, float(lam), int(max_iter),
                                  int(prec), C.byref(chosen)))
        return int(chosen.value)

    def query_batch(self, queries, lam, max_iter: int, prec: int = PREC_FP32) -> np.ndarray:
        """``wmd_query_batch``: ``queries`` is a list of (ids, weights); ``lam``
        one value or one per query.  Returns an (nq, N) float64 array."""
        nq = len(queries)
        lens = [len(np.atleast_1d(q[0])) for q in queries]
        q_ptr = np.zeros(nq + 1, np.int64)
        np.cumsum(lens, out=q_ptr[1:])
        ids = np.ascontiguousarray(np.concatenate([np.asarray(q[0], np.int32).ravel() for q in queries])
                                   if nq else np.zeros(0, np.int32), dtype=np.int32)
        w = np.ascontiguousarray(np.concatenate([np.asarray(q[1], np.float32).ravel() for q in queries])
                                 if nq else np.zeros(0, np.float32), dtype=np.float32)
        lams = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float32), (nq,)), np.float32)
        out = np.empty((nq, self.N), np.float64)
        _check(lib().wmd_query_batch(self._h, nq, _ptr(q_ptr), _ptr(ids), _ptr(w), _ptr(lams),
                                     int(max_iter), int(prec), _ptr(out) if out.size else None))
        return out

    # -------------------------------------------------------------- device path
    def workspace_bytes(self, v_r: int, prec: int = PREC_FP32) -> int:
        return int(lib().wmd_workspace_bytes(self._h, int(v_r), int(prec)))

    def build_kernel_matrix(self, d_ids, d_w, v_r, lam, prec, ws, ws_bytes, stream=None):
        _check(lib().wmd_build_kernel_matrix(self._h, _dptr(d_ids), _dptr(d_w), int(v_r),
                                             float(lam), int(prec), _dptr(ws), int(ws_bytes),
                                             _stream_ptr(stream)))

    def sinkhorn_loop(self, v_r, max_iter, prec, ws, ws_bytes, d_out, stream=None):
        _check(lib().wmd_sinkhorn_loop(self._h, int(v_r), int(max_iter), int(prec), _dptr(ws),
                                       int(ws_bytes), _dptr(d_out), _stream_ptr(stream)))

    def query_device(self, d_ids, d_w, v_r, lam, max_iter, prec, ws, ws_bytes, d_out,
                     stream=None):
        _check(lib().wmd_query_device(self._h, _dptr(d_ids), _dptr(d_w), int(v_r), float(lam),
                                      int(max_iter), int(prec), _dptr(ws), int(ws_bytes),
                                      _dptr(d_out), _stream_ptr(stream)))

    def query_device_tol(self, d_ids, d_w, v_r, lam, max_iter, tol, prec, ws, ws_bytes, d_out,
                         d_iters=None, stream=None):
        """``wmd_query_device_tol``: stop each document once x stops changing
        (relative change <= tol), at most max_iter bodies; ``d_iters``
        (device int32 [N], optional) receives the bodies each document ran."""
        _check(lib().wmd_query_device_tol(self._h, _dptr(d_ids), _dptr(d_w), int(v_r), float(lam),
                                          int(max_iter), float(tol), int(prec), _dptr(ws),
                                          int(ws_bytes), _dptr(d_out), _dptr(d_iters),
                                          _stream_ptr(stream)))

    def query_device_topk(self, d_ids, d_w, v_r, lam, max_iter, prec, ws, ws_bytes, d_out, k,
                          d_idx, d_val, stream=None):
        """``wmd_query_device_topk``: WMD[N] into ``d_out`` and the k nearest
        documents (ascending) into ``d_idx`` (int64) and ``d_val`` (float64)."""
        _check(lib().wmd_query_device_topk(self._h, _dptr(d_ids), _dptr(d_w), int(v_r), float(lam),
                                           int(max_iter), int(prec), _dptr(ws), int(ws_bytes),
                                           _dptr(d_out), int(k), _dptr(d_idx), _dptr(d_val),
                                           _stream_ptr(stream)))

    # -------------------------------------------------------------- dense comparator
    def dense_workspace_bytes(self, v_r: int) -> int:
        """``wmd_dense_workspace_bytes``."""
        return int(lib().wmd_dense_workspace_bytes(self._h, int(v_r)))

    def dense_load_c(self, ws, ws_bytes, stream=None):
        """``wmd_dense_load_c``: the dense U x N c at the start of ``ws``."""
        _check(lib().wmd_dense_load_c(self._h, _dptr(ws), int(ws_bytes), _stream_ptr(stream)))

    def query_dense(self, d_ids, d_w, v_r, lam, max_iter, ws, ws_bytes, d_out, stream=None):
        """``wmd_query_dense``: Algorithm 1 in its dense form (cuBLAS GEMMs)."""
        _check(lib().wmd_query_dense(self._h, _dptr(d_ids), _dptr(d_w), int(v_r), float(lam),
                                     int(max_iter), _dptr(ws), int(ws_bytes), _dptr(d_out),
                                     _stream_ptr(stream)))


def topk(d_wmd, N: int, k: int, d_idx, d_val, stream=None):
    """``wmd_topk``: the k smallest of ``d_wmd[:N]`` (device float64) and their
    document ids, ascending; ties to the lower id, NaN last."""
    _check(lib().wmd_topk(_dptr(d_wmd), int(N), int(k), _dptr(d_idx), _dptr(d_val),
                          _stream_ptr(stream)))


def query_device_noalloc(corpus: "Corpus", d_ids, d_w, v_r, lam, max_iter, prec, d_out,
                         stream=None):
    """``wmd_query_device_noalloc``: the device path without a workspace.

    For callers that may not allocate device memory: the library's built-in
    16 MiB scratch array stands in for the workspace.  Calls share that array,
    so they must not overlap on the GPU."""
    _check(lib().wmd_query_device_noalloc(corpus.handle, _dptr(d_ids), _dptr(d_w), int(v_r),
                                          float(lam), int(max_iter), int(prec), _dptr(d_out),
                                          _stream_ptr(stream)))


class DeviceQuery:
    """Device buffers (torch) for the stream-ordered path of one query."""

    def __init__(self, corpus: Corpus, q_ids, q_w, prec: int = PREC_FP32):
        import torch
        ids, w = compact_query(q_ids, q_w, corpus.V)
        dev = torch.device("cuda", corpus.device)
        self.v_r = int(ids.size)
        self.prec = prec
        self.ids = torch.from_numpy(ids).to(dev)
        self.w = torch.from_numpy(w).to(dev)
        self.ws_bytes = corpus.workspace_bytes(self.v_r, prec)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.out = torch.empty(max(corpus.N, 1), dtype=torch.float64, device=dev)
        self.corpus = corpus

    def run(self, lam: float, max_iter: int, stream=None):
        self.corpus.query_device(self.ids, self.w, self.v_r, lam, max_iter, self.prec, self.ws,
                                 self.ws_bytes, self.out, stream)
        return self.out


class Server:
    """``wmd_server``: continuous batching of queries against a corpus."""

    def __init__(self, corpus: Corpus, max_batch: int = 64, slots: int = 2,
                 mem_budget: int = 8 << 30, max_pending: int = 65536):
        opt = ServerOptions(int(max_batch), int(slots), int(mem_budget), int(max_pending))
        h = C.c_void_p()
        _check(lib().wmd_server_create(corpus.handle, C.byref(opt), C.byref(h)))
        self._h = h
        self.corpus = corpus

    def submit(self, q_ids, q_w, lam: float, max_iter: int, prec: int = PREC_FP32) -> int:
        ids = np.ascontiguousarray(q_ids, dtype=np.int32)
        w = np.ascontiguousarray(q_w, dtype=np.float32)
        t = C.c_uint64(0)
        _check(lib().wmd_serve_submit(self._h, _ptr(ids), _ptr(w), ids.size, float(lam),
                                      int(max_iter), int(prec), C.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, timeout_us: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.corpus.N, np.float64)
        _check(lib().wmd_serve_poll(self._h, C.c_uint64(ticket), _ptr(out) if out.size else None,
                                    int(timeout_us)))
        return out

    def cancel(self, ticket: int):
        _check(lib().wmd_serve_cancel(self._h, C.c_uint64(ticket)))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().wmd_server_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().wmd_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
