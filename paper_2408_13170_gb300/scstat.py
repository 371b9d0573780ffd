"""Python binding of the C ABI in include/scstat.h (argument marshalling only).

Every function here forwards to libscstat.so; all arithmetic of the
statistic runs in the library's CUDA kernels.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); complex data are complex128.
If the library cannot be built or loaded, the import of a function raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

SCS_OK, SCS_EINVAL, SCS_ENOMEM, SCS_ECUDA, SCS_ENODATA, SCS_ETIMEOUT, SCS_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
SCS_FP64, SCS_MIXED = 0, 1
SCS_EQUAL_WIDTH, SCS_EQUAL_SNR2 = 0, 1

_lock = threading.Lock()
_lib = None


class ScsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"scstat error {code}: {msg}")
        self.code = code


def lib():
    """The loaded libscstat.so (built on first use)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.scs_create.argtypes = [ctypes.POINTER(P), I, I]
        L.scs_create.restype = I
        L.scs_destroy.argtypes = [P]
        L.scs_destroy.restype = None
        L.scs_last_error.argtypes = [P]
        L.scs_last_error.restype = ctypes.c_char_p
        L.scs_set_path.argtypes = [P, I]
        L.scs_set_path.restype = I
        L.scs_set_data.argtypes = [P, I, P, P, P, P, D, D, I64, D]
        L.scs_set_data.restype = I
        L.scs_set_segments.argtypes = [P, I, I, I]
        L.scs_set_segments.restype = I
        L.scs_eval_stat.argtypes = [P, I, P, I64, P, P, P, P]
        L.scs_eval_stat.restype = I
        L.scs_waveform.argtypes = [P, I, P, P, P, P]
        L.scs_waveform.restype = I
        L.scs_inject.argtypes = [P, I, P, D, P]
        L.scs_inject.restype = I
        L.scs_support.argtypes = [P, I, P, I64, P, P, P, P]
        L.scs_support.restype = I
        L.scs_segment_edges.argtypes = [P, I, P, I64, P, P]
        L.scs_segment_edges.restype = I
        L.scs_set_profiling.argtypes = [P, I]
        L.scs_set_profiling.restype = I
        L.scs_last_timings.argtypes = [P, P]
        L.scs_last_timings.restype = I
        L.scs_eval_stat_noalloc.argtypes = [P, I, P, I64, P, P]
        L.scs_eval_stat_noalloc.restype = I
        L.scs_batch_eval.argtypes = [P, P, P, I, P, P, P]
        L.scs_batch_eval.restype = I
        _lib = L
        return L


def _ptr(x):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


_CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream


def _stream(s):
    """cudaStream_t handle of a torch stream (or an int).  torch reports the
    default stream as handle 0, which the C ABI reads as "the context's own
    stream"; it is passed as cudaStreamLegacy so the work stays ordered with
    torch's default stream."""
    if s is None:
        return None
    h = getattr(s, "cuda_stream", s)
    return _CUDA_STREAM_LEGACY if h == 0 else h


def _check(ctx, rc):
    if rc != SCS_OK:
        msg = lib().scs_last_error(ctx).decode(errors="replace") if ctx else ""
        raise ScsError(rc, msg)


# ------------------------------------------------------- the C entry points
def scs_create(device: int = 0, path: int = SCS_MIXED):
    h = ctypes.c_void_p()
    rc = lib().scs_create(ctypes.byref(h), device, path)
    if rc != SCS_OK:
        raise ScsError(rc, "scs_create failed")
    return h


def scs_destroy(ctx):
    lib().scs_destroy(ctx)


def scs_last_error(ctx) -> str:
    return lib().scs_last_error(ctx).decode(errors="replace")


def scs_set_path(ctx, path: int):
    _check(ctx, lib().scs_set_path(ctx, path))


def scs_set_data(ctx, stream_id, A, E, S_A, S_E, f_first, df, K, T_obs):
    _check(ctx, lib().scs_set_data(ctx, stream_id, _ptr(A), _ptr(E), _ptr(S_A), _ptr(S_E),
                                   float(f_first), float(df), int(K), float(T_obs)))


def scs_set_segments(ctx, stream_id, N, mode):
    _check(ctx, lib().scs_set_segments(ctx, stream_id, int(N), int(mode)))


def scs_eval_stat(ctx, stream_id, params, P, stat, seg_x=None, seg_hh=None, cuda_stream=None):
    _check(ctx, lib().scs_eval_stat(ctx, stream_id, _ptr(params), int(P), _ptr(stat),
                                    _ptr(seg_x), _ptr(seg_hh), _stream(cuda_stream)))


def scs_batch_eval(ctx, stream_ids, P_offsets, params, stat, cuda_stream=None):
    """Items i: particles P_offsets[i]..P_offsets[i+1]-1 on stream stream_ids[i]."""
    sids = np.ascontiguousarray(stream_ids, dtype=np.int32)
    offs = np.ascontiguousarray(P_offsets, dtype=np.int64)
    _check(ctx, lib().scs_batch_eval(ctx, _ptr(sids), _ptr(offs), len(sids), _ptr(params),
                                     _ptr(stat), _stream(cuda_stream)))


def scs_waveform(ctx, stream_id, theta, hA, hE, cuda_stream=None):
    _check(ctx, lib().scs_waveform(ctx, stream_id, _ptr(theta), _ptr(hA), _ptr(hE),
                                   _stream(cuda_stream)))


def scs_inject(ctx, stream_id, theta, snr):
    hh = ctypes.c_double()
    _check(ctx, lib().scs_inject(ctx, stream_id, _ptr(theta), float(snr), ctypes.byref(hh)))
    return hh.value


def scs_support(ctx, stream_id, params, P, k_lo, k_hi, log2_stride=None, cuda_stream=None):
    _check(ctx, lib().scs_support(ctx, stream_id, _ptr(params), int(P), _ptr(k_lo),
                                  _ptr(k_hi), _ptr(log2_stride), _stream(cuda_stream)))


def scs_segment_edges(ctx, stream_id, params, P, edges, cuda_stream=None):
    _check(ctx, lib().scs_segment_edges(ctx, stream_id, _ptr(params), int(P), _ptr(edges),
                                        _stream(cuda_stream)))


def scs_eval_stat_noalloc(ctx, stream_id, params, P, stat, cuda_stream=None):
    """scs_eval_stat with scratch from the library's fixed device array (no
    allocation); params and stat must be CUDA tensors."""
    _check(ctx, lib().scs_eval_stat_noalloc(ctx, stream_id, _ptr(params), int(P), _ptr(stat),
                                            _stream(cuda_stream)))


def scs_set_profiling(ctx, enable: bool):
    _check(ctx, lib().scs_set_profiling(ctx, 1 if enable else 0))


def scs_last_timings(ctx):
    """ms of (set-up + work list, segment edges, main kernel, fix-up)."""
    out = np.zeros(4)
    _check(ctx, lib().scs_last_timings(ctx, out.ctypes.data))
    return out


# ------------------------------------------------------ numpy convenience
class Context:
    """Owns one scs_ctx; thin numpy-facing wrappers of the entry points."""

    def __init__(self, device: int = 0, path: int = SCS_MIXED):
        self.h = scs_create(device, path)

    def close(self):
        if self.h:
            scs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_path(self, path):
        scs_set_path(self.h, path)

    def set_data(self, stream_id, data):
        A = np.ascontiguousarray(data["A"], dtype=np.complex128)
        E = np.ascontiguousarray(data["E"], dtype=np.complex128)
        SA = np.ascontiguousarray(data["SA"], dtype=np.float64)
        SE = data.get("SE")
        SE = None if SE is None else np.ascontiguousarray(SE, dtype=np.float64)
        scs_set_data(self.h, stream_id, A, E, SA, SE, data["f_first"], data["df"], data["K"],
                     data["T_obs"])

    def set_segments(self, stream_id, N, mode):
        scs_set_segments(self.h, stream_id, N, mode)

    def eval(self, stream_id, params, N=None, segments=False):
        params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 8)
        P = params.shape[0]
        stat = np.empty(P)
        if segments:
            sx = np.empty((P, N))
            sh = np.empty((P, N))
            scs_eval_stat(self.h, stream_id, params, P, stat, sx, sh)
            return stat, sx, sh
        scs_eval_stat(self.h, stream_id, params, P, stat)
        return stat

    def batch_eval(self, stream_ids, params_list):
        """One launch over several streams; returns one stat array per item."""
        params_list = [np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 8)
                       for p in params_list]
        offs = np.concatenate([[0], np.cumsum([len(p) for p in params_list])])
        allp = np.ascontiguousarray(np.vstack(params_list))
        stat = np.empty(len(allp))
        scs_batch_eval(self.h, stream_ids, offs, allp, stat)
        return [stat[offs[i]:offs[i + 1]] for i in range(len(params_list))]

    def waveform(self, stream_id, theta, K):
        hA = np.empty(K, np.complex128)
        hE = np.empty(K, np.complex128)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        scs_waveform(self.h, stream_id, th, hA, hE)
        return hA, hE

    def inject(self, stream_id, theta, snr):
        return scs_inject(self.h, stream_id, np.ascontiguousarray(theta, dtype=np.float64), snr)

    def support(self, stream_id, params):
        params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 8)
        P = params.shape[0]
        lo = np.empty(P, np.int64)
        hi = np.empty(P, np.int64)
        l2 = np.empty(P, np.int32)
        scs_support(self.h, stream_id, params, P, lo, hi, l2)
        return lo, hi, l2

    def edges(self, stream_id, params, N):
        params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 8)
        P = params.shape[0]
        e = np.empty((P, N + 1), np.int64)
        scs_segment_edges(self.h, stream_id, params, P, e)
        return e
