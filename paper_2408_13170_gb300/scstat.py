"""Python binding of the C ABI in include/scstat.h (argument marshalling only).

Every function here forwards to libscstat.so; all arithmetic of the
statistic runs in the library's CUDA kernels.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); complex data are complex128.
If the library cannot be built or loaded, the import of a function raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SCS_OK, SCS_EINVAL, SCS_ENOMEM, SCS_ECUDA, SCS_ENODATA, SCS_ETIMEOUT, SCS_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6)
SCS_FP64, SCS_MIXED, SCS_SPLINE = 0, 1, 2
SCS_EQUAL_WIDTH, SCS_EQUAL_SNR2 = 0, 1
# test-only models (scs_debug_set_model)
SCS_MODEL_TF2, SCS_MODEL_NEWTONIAN, SCS_MODEL_LINEAR_CHIRP = 0, 1, 2
SCS_RESPONSE_TDI, SCS_RESPONSE_IDENTITY = 0, 1

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
        # SCS_DEBUG=1: the build with index checks (scs_debug_error)
        path = _build.build(debug=os.environ.get("SCS_DEBUG") == "1")
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
        L.scs_debug_set_model.argtypes = [P, I, I]
        L.scs_debug_set_model.restype = I
        L.scs_set_spline.argtypes = [P, I]
        L.scs_set_spline.restype = I
        L.scs_set_data.argtypes = [P, I, P, P, P, P, D, D, I64, D]
        L.scs_set_data.restype = I
        L.scs_set_data_aet.argtypes = [P, I, P, P, P, P, P, P, D, D, I64, D]
        L.scs_set_data_aet.restype = I
        L.scs_set_segments.argtypes = [P, I, I, I]
        L.scs_set_segments.restype = I
        L.scs_eval_stat.argtypes = [P, I, P, I64, P, P, P, P]
        L.scs_eval_stat.restype = I
        L.scs_waveform.argtypes = [P, I, P, P, P, P]
        L.scs_waveform.restype = I
        L.scs_waveform_aet.argtypes = [P, I, P, P, P, P, P]
        L.scs_waveform_aet.restype = I
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
        L.scs_last_counters.argtypes = [P, P, I]
        L.scs_last_counters.restype = I
        L.scs_debug_error.argtypes = [P, P, P]
        L.scs_debug_error.restype = I
        L.scs_eval_stat_noalloc.argtypes = [P, I, P, I64, P, P]
        L.scs_eval_stat_noalloc.restype = I
        L.scs_batch_eval.argtypes = [P, P, P, I, P, P, P]
        L.scs_batch_eval.restype = I
        L.scs_eval_loglike.argtypes = [P, I, P, I64, P, P, P, P, P]
        L.scs_eval_loglike.restype = I
        L.scs_set_tile.argtypes = [P, I, I]
        L.scs_set_tile.restype = I
        L.scs_autotune.argtypes = [P, I, P, I64, P, P, P]
        L.scs_autotune.restype = I
        U64 = ctypes.c_uint64
        L.scs_pso_create.argtypes = [P, I, P, P, P, P, U64, P]
        L.scs_pso_set_hyper.argtypes = [P, I, D, D, D, P, P]
        L.scs_pso_run.argtypes = [P, I, I, P]
        L.scs_pso_get.argtypes = [P, P, P, P, P, P, P, P, P, P]
        L.scs_pso_set.argtypes = [P, P, P, P, P, P, P, I64, P]
        L.scs_pso_save.argtypes = [P, P, P, P]
        L.scs_pso_load.argtypes = [P, P, ctypes.c_size_t, P]
        L.scs_pso_set_convergence.argtypes = [P, D, I]
        L.scs_pso_status.argtypes = [P, P, P, P]
        L.scs_pso_reset_bests.argtypes = [P, P]
        L.scs_pso_layout.argtypes = [P, P, P, P]
        L.scs_kmeans.argtypes = [P, P, I64, P, P, I, I, P, P, P]
        L.scs_pso_regroup.argtypes = [P, I, I, P]
        L.scs_pso_search.argtypes = [P, P, I, P, I, I, I, P, P]
        for f in ("scs_pso_create", "scs_pso_set_hyper", "scs_pso_run", "scs_pso_get",
                  "scs_pso_set", "scs_pso_save", "scs_pso_load", "scs_pso_set_convergence",
                  "scs_pso_status", "scs_pso_reset_bests", "scs_pso_layout", "scs_kmeans",
                  "scs_pso_regroup", "scs_pso_search"):
            getattr(L, f).restype = I
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


def scs_set_spline(ctx, max_log2_spacing: int):
    """Largest node spacing (log2 bins) of the SCS_SPLINE path."""
    _check(ctx, lib().scs_set_spline(ctx, max_log2_spacing))


def scs_debug_set_model(ctx, waveform: int, response: int):
    """Test-only: switch waveform / response to a closed-form test model."""
    _check(ctx, lib().scs_debug_set_model(ctx, waveform, response))


def scs_set_data(ctx, stream_id, A, E, S_A, S_E, f_first, df, K, T_obs):
    _check(ctx, lib().scs_set_data(ctx, stream_id, _ptr(A), _ptr(E), _ptr(S_A), _ptr(S_E),
                                   float(f_first), float(df), int(K), float(T_obs)))


def scs_set_data_aet(ctx, stream_id, A, E, T, S_A, S_E, S_T, f_first, df, K, T_obs):
    _check(ctx, lib().scs_set_data_aet(ctx, stream_id, _ptr(A), _ptr(E), _ptr(T), _ptr(S_A),
                                       _ptr(S_E), _ptr(S_T), float(f_first), float(df), int(K),
                                       float(T_obs)))


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


def scs_waveform_aet(ctx, stream_id, theta, hA, hE, hT, cuda_stream=None):
    _check(ctx, lib().scs_waveform_aet(ctx, stream_id, _ptr(theta), _ptr(hA), _ptr(hE),
                                       _ptr(hT), _stream(cuda_stream)))


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


# Table III of the paper: (Omega, Phi_P, Phi_G) and the minimum velocities per
# rung N of the segment ladder, with eps re-ordered to this library's parameter
# order (Mc, q, f0, lambda, beta, iota, psi, e0); the paper's eps for eta is
# applied to q and its eps for f_low to f0.
TABLE3_HYPER = {
    100: (0.5, 0.2, 0.3, (0.1, 0.05, 5e-8, 0.1, 0.1, 0.2, 0.1, 0.1)),
    50: (0.5, 0.2, 0.4, (0.01, 0.05, 1e-8, 0.01, 0.01, 0.2, 0.1, 0.1)),
    10: (0.3, 0.2, 0.5, (0.001, 0.05, 1e-8, 0.001, 0.001, 0.01, 0.1, 0.1)),
    1: (0.72, 1.193, 1.193, (0.0,) * 8),
}


def table3_hyper(N: int):
    """Table III row of the ladder rung closest to N (ties: the larger N)."""
    rung = min(sorted(TABLE3_HYPER, reverse=True), key=lambda r: abs(r - N))
    return TABLE3_HYPER[rung]


def scs_pso_create(ctx, stream_ids, swarm_offsets, prior_lo, prior_hi, seed, cuda_stream=None):
    sids = np.ascontiguousarray(stream_ids, dtype=np.int32)
    offs = np.ascontiguousarray(swarm_offsets, dtype=np.int64)
    lo = np.ascontiguousarray(prior_lo, dtype=np.float64)
    hi = np.ascontiguousarray(prior_hi, dtype=np.float64)
    _check(ctx, lib().scs_pso_create(ctx, len(sids), _ptr(sids), _ptr(offs), _ptr(lo),
                                     _ptr(hi), int(seed), _stream(cuda_stream)))


def scs_pso_set_hyper(ctx, swarm, Omega, PhiP, PhiG, eps, cuda_stream=None):
    e = np.ascontiguousarray(eps, dtype=np.float64)
    _check(ctx, lib().scs_pso_set_hyper(ctx, int(swarm), float(Omega), float(PhiP),
                                        float(PhiG), _ptr(e), _stream(cuda_stream)))


def scs_pso_run(ctx, iters, use_graph=True, cuda_stream=None):
    _check(ctx, lib().scs_pso_run(ctx, int(iters), 1 if use_graph else 0,
                                  _stream(cuda_stream)))


def scs_pso_get(ctx, pos=None, vel=None, best_pos=None, best_val=None, swarm_pos=None,
                swarm_val=None, stat=None, cuda_stream=None):
    it = ctypes.c_int64()
    _check(ctx, lib().scs_pso_get(ctx, _ptr(pos), _ptr(vel), _ptr(best_pos), _ptr(best_val),
                                  _ptr(swarm_pos), _ptr(swarm_val), _ptr(stat),
                                  ctypes.byref(it), _stream(cuda_stream)))
    return it.value


def scs_pso_set(ctx, pos=None, vel=None, best_pos=None, best_val=None, swarm_pos=None,
                swarm_val=None, iteration=0, cuda_stream=None):
    _check(ctx, lib().scs_pso_set(ctx, _ptr(pos), _ptr(vel), _ptr(best_pos), _ptr(best_val),
                                  _ptr(swarm_pos), _ptr(swarm_val), int(iteration),
                                  _stream(cuda_stream)))


def scs_pso_save(ctx, cuda_stream=None) -> bytes:
    n = ctypes.c_size_t()
    _check(ctx, lib().scs_pso_save(ctx, None, ctypes.byref(n), _stream(cuda_stream)))
    buf = ctypes.create_string_buffer(n.value)
    _check(ctx, lib().scs_pso_save(ctx, buf, ctypes.byref(n), _stream(cuda_stream)))
    return buf.raw[:n.value]


def scs_pso_load(ctx, blob: bytes, cuda_stream=None):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(ctx, lib().scs_pso_load(ctx, buf, len(blob), _stream(cuda_stream)))


def scs_eval_loglike(ctx, stream_id, params, P, loglike, amp=None, overlap=None, hh=None,
                     cuda_stream=None):
    _check(ctx, lib().scs_eval_loglike(ctx, stream_id, _ptr(params), int(P), _ptr(amp),
                                       _ptr(loglike), _ptr(overlap), _ptr(hh),
                                       _stream(cuda_stream)))


def scs_set_tile(ctx, stream_id, log2_chunk):
    _check(ctx, lib().scs_set_tile(ctx, stream_id, int(log2_chunk)))


def scs_autotune(ctx, stream_id, params, P, cuda_stream=None):
    """Times every tile on these particles; returns (chosen log2_chunk, ms[4])."""
    best = ctypes.c_int()
    ms = np.zeros(4)
    _check(ctx, lib().scs_autotune(ctx, stream_id, _ptr(params), int(P), ctypes.byref(best),
                                   ms.ctypes.data, _stream(cuda_stream)))
    return best.value, ms


def scs_pso_set_convergence(ctx, delta=2.0, window=50):
    _check(ctx, lib().scs_pso_set_convergence(ctx, float(delta), int(window)))


def scs_pso_layout(ctx):
    """(stream_ids[S], swarm_offsets[S + 1]) of the current swarms."""
    n = ctypes.c_int()
    _check(ctx, lib().scs_pso_layout(ctx, ctypes.byref(n), None, None))
    sids = np.empty(n.value, np.int32)
    offs = np.empty(n.value + 1, np.int64)
    _check(ctx, lib().scs_pso_layout(ctx, ctypes.byref(n), _ptr(sids), _ptr(offs)))
    return sids, offs


def scs_pso_status(ctx, cuda_stream=None):
    """(all converged, converged[S], iteration)."""
    S = len(scs_pso_layout(ctx)[0])
    conv = np.zeros(S, np.int32)
    it = ctypes.c_int64()
    rc = lib().scs_pso_status(ctx, _ptr(conv), ctypes.byref(it), _stream(cuda_stream))
    if rc < 0:
        _check(ctx, rc)
    return rc == 1, conv.astype(bool), it.value


def scs_pso_reset_bests(ctx, cuda_stream=None):
    _check(ctx, lib().scs_pso_reset_bests(ctx, _stream(cuda_stream)))


def scs_kmeans(ctx, pos, prior_lo, prior_hi, k, iters, cuda_stream=None):
    """(labels[P], centroids[k, 9]) of P x 8 positions."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 8)
    lo = np.ascontiguousarray(prior_lo, dtype=np.float64)
    hi = np.ascontiguousarray(prior_hi, dtype=np.float64)
    lab = np.empty(len(pos), np.int32)
    cen = np.empty((k, 9))
    _check(ctx, lib().scs_kmeans(ctx, _ptr(pos), len(pos), _ptr(lo), _ptr(hi), int(k),
                                 int(iters), _ptr(lab), _ptr(cen), _stream(cuda_stream)))
    return lab, cen


def scs_pso_regroup(ctx, n_clusters, iters=10, cuda_stream=None):
    _check(ctx, lib().scs_pso_regroup(ctx, int(n_clusters), int(iters), _stream(cuda_stream)))


def scs_pso_search(ctx, ladder, hyper_rows, n_clusters, chunk_iters, max_iters,
                   cuda_stream=None):
    """Runs the ladder; returns the iterations spent on each rung."""
    lad = np.ascontiguousarray(ladder, dtype=np.int32)
    rows = np.ascontiguousarray(hyper_rows, dtype=np.float64).reshape(len(lad), 11)
    its = np.zeros(len(lad), np.int64)
    _check(ctx, lib().scs_pso_search(ctx, _ptr(lad), len(lad), _ptr(rows), int(n_clusters),
                                     int(chunk_iters), int(max_iters), _ptr(its),
                                     _stream(cuda_stream)))
    return its


def scs_set_profiling(ctx, enable: bool):
    _check(ctx, lib().scs_set_profiling(ctx, 1 if enable else 0))


def scs_last_counters(ctx):
    """(particles, particles whose equal-SNR^2 edges took the FP64 fallback
    or -1) of the last profiled evaluation."""
    out = np.zeros(2, np.int64)
    _check(ctx, lib().scs_last_counters(ctx, _ptr(out), 2))
    return int(out[0]), int(out[1])


def scs_debug_error(ctx):
    """(is a debug build, failed check number or 0, its index or -1): reads
    and clears the index-check record of the debug build."""
    chk, idx = ctypes.c_int(0), ctypes.c_longlong(-1)
    rc = lib().scs_debug_error(ctx, ctypes.byref(chk), ctypes.byref(idx))
    if rc not in (SCS_OK, SCS_EUNSUPPORTED):
        _check(ctx, rc)
    return rc == SCS_OK, chk.value, idx.value


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

    def set_model(self, waveform, response):
        scs_debug_set_model(self.h, waveform, response)

    def set_data(self, stream_id, data):
        A = np.ascontiguousarray(data["A"], dtype=np.complex128)
        E = np.ascontiguousarray(data["E"], dtype=np.complex128)
        SA = np.ascontiguousarray(data["SA"], dtype=np.float64)
        SE = data.get("SE")
        SE = None if SE is None else np.ascontiguousarray(SE, dtype=np.float64)
        if data.get("T") is not None:   # the third TDI channel with its PSD
            T = np.ascontiguousarray(data["T"], dtype=np.complex128)
            ST = np.ascontiguousarray(data["ST"], dtype=np.float64)
            scs_set_data_aet(self.h, stream_id, A, E, T, SA, SE, ST, data["f_first"],
                             data["df"], data["K"], data["T_obs"])
            return
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

    def loglike(self, stream_id, params, amp=None):
        """(log L_N, O_N, <h|h>) per particle (Sec. II.B)."""
        params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 8)
        P = params.shape[0]
        L, O, H = np.empty(P), np.empty(P), np.empty(P)
        a = None if amp is None else np.ascontiguousarray(amp, dtype=np.float64)
        scs_eval_loglike(self.h, stream_id, params, P, L, a, O, H)
        return L, O, H

    def batch_eval(self, stream_ids, params_list):
        """One launch over several streams; returns one stat array per item."""
        params_list = [np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 8)
                       for p in params_list]
        offs = np.concatenate([[0], np.cumsum([len(p) for p in params_list])])
        allp = np.ascontiguousarray(np.vstack(params_list))
        stat = np.empty(len(allp))
        scs_batch_eval(self.h, stream_ids, offs, allp, stat)
        return [stat[offs[i]:offs[i + 1]] for i in range(len(params_list))]

    def waveform(self, stream_id, theta, K, want_T=False):
        hA = np.empty(K, np.complex128)
        hE = np.empty(K, np.complex128)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        if want_T:
            hT = np.empty(K, np.complex128)
            scs_waveform_aet(self.h, stream_id, th, hA, hE, hT)
            return hA, hE, hT
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

    # --------------------------------------------------------------- swarm
    def pso_create(self, stream_ids, swarm_sizes, prior_lo, prior_hi, seed):
        """Swarm s has swarm_sizes[s] particles and searches stream stream_ids[s]."""
        offs = np.concatenate([[0], np.cumsum(swarm_sizes)]).astype(np.int64)
        scs_pso_create(self.h, stream_ids, offs, prior_lo, prior_hi, seed)
        self._pso_P, self._pso_S = int(offs[-1]), len(offs) - 1

    def pso_set_hyper(self, Omega, PhiP, PhiG, eps, swarm=-1):
        scs_pso_set_hyper(self.h, swarm, Omega, PhiP, PhiG, eps)

    def pso_run(self, iters, use_graph=True):
        scs_pso_run(self.h, iters, use_graph)

    def pso_get(self):
        P = self._pso_P
        S = len(scs_pso_layout(self.h)[0])
        st = dict(pos=np.empty((P, 8)), vel=np.empty((P, 8)), best_pos=np.empty((P, 8)),
                  best_val=np.empty(P), swarm_pos=np.empty((S, 8)), swarm_val=np.empty(S),
                  stat=np.empty(P))
        st["iteration"] = scs_pso_get(self.h, **st)
        return st

    def pso_set(self, state):
        keys = ("pos", "vel", "best_pos", "best_val", "swarm_pos", "swarm_val")
        arrs = {k: np.ascontiguousarray(state[k], dtype=np.float64) for k in keys}
        scs_pso_set(self.h, iteration=state["iteration"], **arrs)

    def pso_save(self) -> bytes:
        return scs_pso_save(self.h)

    def pso_load(self, blob: bytes):
        scs_pso_load(self.h, blob)
        P, S = np.frombuffer(blob, np.int64, 2, 8)
        self._pso_P, self._pso_S = int(P), int(S)

    def pso_search(self, ladder, n_clusters=0, chunk_iters=10, max_iters=200):
        """The hierarchical search with the Table III row of each rung."""
        rows = [np.concatenate([[om, pp, pg], eps])
                for om, pp, pg, eps in (table3_hyper(N) for N in ladder)]
        return scs_pso_search(self.h, ladder, rows, n_clusters, chunk_iters, max_iters)
