"""FP64 CPU oracle for the semi-coherent statistic (test infrastructure only).

This package is the independent reference that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
legs of ``bench.py`` may import it; the product package never does, and it
imports nothing from the product package.

The arithmetic lives in ``scoracle.c`` (plain C, FP64 with double-double
phases, Neumaier sums).  This module compiles it with gcc on first use and
wraps it with ctypes.

What the oracle computes (arXiv:2408.13170):
  * inner product and segmented inner product (Sec. II.A Eq. inner_prod,
    Sec. II.B [a|b]_n);
  * x_n = max_phi [d|h e^{i phi}]_n = |z_n| (Sec. II.B Eq. semi-coherent_O);
  * Upsilon_N = sum_n x_n^2 / [h|h]_n (Sec. II.B);
  * segment boundaries: equal-width, or equal squared SNR per segment
    re-evaluated for every theta (Sec. II.B, last paragraph);
  * template h_alpha = T_alpha(theta, f) A(f) e^{-i Psi(f)} on the FFT grid
    (Sec. IV), TaylorF2 2PN circular phase and the rigid-adiabatic LISA TDI
    A/E response, optionally with the third channel T (the paper's search
    uses all three, Sec. I).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scoracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

TF2, NEWTONIAN, LINEAR_CHIRP = 0, 1, 2
TDI_AE, IDENTITY = 0, 1
EQUAL_WIDTH, EQUAL_SNR2 = 0, 1
OK, INVALID, EMPTY = 0, 1, 2
SNR2_STRIDE = 1024


def build(force: bool = False) -> str:
    """Compile scoracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I64, I = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        lib.orc_support.argtypes = [P, I, D, D, I64, D, P, P]
        lib.orc_support.restype = I
        lib.orc_time_of_freq.argtypes = [P, I, D]
        lib.orc_time_of_freq.restype = D
        lib.orc_derive.argtypes = [P, I, P]
        lib.orc_derive.restype = I
        lib.orc_phase_turns.argtypes = [P, I, D, D, I64]
        lib.orc_phase_turns.restype = D
        lib.orc_pn_terms.argtypes = [P, I, D, P, P]
        lib.orc_pn_terms.restype = I
        lib.orc_response.argtypes = [P, D, D, P, P]
        lib.orc_response.restype = I
        lib.orc_template.argtypes = [P, I, I, D, D, I64, D, D, D, P, P, P]
        lib.orc_template.restype = I
        lib.orc_eval.argtypes = [D, D, I64, D, P, P, P, P, P, P, I, I, I, I, P,
                                 I64, D, D, P, P, P, P, I]
        lib.orc_eval.restype = I
        lib.orc_inject.argtypes = [P, D, D, I64, D, P, P, P, D, P, P, P]
        lib.orc_inject.restype = D
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _theta(theta):
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    if th.size != 8:
        raise ValueError("theta must have 8 entries")
    return th


def support(theta, f_first, df, K, T_obs, waveform=TF2):
    """(status, k_lo, k_hi) of the support of one particle on the grid."""
    lib = _load()
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    st = lib.orc_support(_ptr(_theta(theta)), waveform, f_first, df, int(K),
                         T_obs, ctypes.byref(lo), ctypes.byref(hi))
    return st, lo.value, hi.value


def time_of_freq(theta, f, waveform=TF2):
    return _load().orc_time_of_freq(_ptr(_theta(theta)), waveform, float(f))


def derive(theta, waveform=TF2):
    """(status, eta, M [s], t_c [s]) of one particle."""
    out = np.zeros(4)
    st = _load().orc_derive(_ptr(_theta(theta)), waveform, _ptr(out))
    return st, out[0], out[1], out[2] + out[3]


def phase_turns(theta, f_first, df, k, waveform=TF2):
    return _load().orc_phase_turns(_ptr(_theta(theta)), waveform, f_first, df,
                                   int(k))


def pn_terms(theta, f, waveform=TF2):
    """The PN phase split by order at frequency f: (status, F[8] turns,
    T[8] seconds), T = dF/df, for the orders 0, 1, 1.5, 2, 2.5, 3, 3.5PN and
    the leading eccentric term (Sec. IV, TaylorF2Ecc read as 3.5PN TaylorF2
    plus the O(e0^2) correction)."""
    F = np.zeros(8)
    T = np.zeros(8)
    st = _load().orc_pn_terms(_ptr(_theta(theta)), waveform, float(f), _ptr(F),
                              _ptr(T))
    return st, F, T


def response(theta, f, t):
    """Links G_{1->2},G_{2->1},G_{1->3},G_{3->1},G_{2->3},G_{3->2}, X, Y, Z,
    A, E, T (complex[12]) and craft positions (3x3, seconds) at (f, t)."""
    out = np.zeros(24)
    pos = np.zeros(9)
    _load().orc_response(_ptr(_theta(theta)), float(f), float(t), _ptr(out),
                         _ptr(pos))
    return out[0::2] + 1j * out[1::2], pos.reshape(3, 3)


def template(theta, f_first, df, K, T_obs, waveform=TF2, response=TDI_AE,
             amp_scale=1.0, phase0=0.0, want_T=False):
    """(status, h_A[K], h_E[K]) complex128 over the whole grid; with want_T
    also h_T[K] (status, h_A, h_E, h_T)."""
    hA = np.zeros(2 * int(K))
    hE = np.zeros(2 * int(K))
    hT = np.zeros(2 * int(K)) if want_T else None
    st = _load().orc_template(_ptr(_theta(theta)), waveform, response,
                              f_first, df, int(K), T_obs, amp_scale, phase0,
                              _ptr(hA), _ptr(hE), _ptr(hT))
    out = (st, hA.view(np.complex128), hE.view(np.complex128))
    return out + (hT.view(np.complex128),) if want_T else out


def inject(theta, f_first, df, K, T_obs, SA, SE, snr, A, E, T=None, ST=None):
    """Adds snr * h/sqrt(<h|h>) to complex128 arrays A, E (and T, whose PSD
    is ST, when given) in place; returns <h|h> of the un-normalised template
    over the channels given."""
    assert A.dtype == np.complex128 and E.dtype == np.complex128
    assert A.flags.c_contiguous and E.flags.c_contiguous
    if T is not None:
        assert T.dtype == np.complex128 and T.flags.c_contiguous and ST is not None
        ST = np.ascontiguousarray(ST, dtype=np.float64)
    SA = np.ascontiguousarray(SA, dtype=np.float64)
    SE = None if SE is None else np.ascontiguousarray(SE, dtype=np.float64)
    return _load().orc_inject(_ptr(_theta(theta)), f_first, df, int(K), T_obs,
                              _ptr(SA), _ptr(SE), _ptr(ST if T is not None else None),
                              float(snr), _ptr(A), _ptr(E), _ptr(T))


def evaluate(data, params, N, mode=EQUAL_WIDTH, waveform=TF2,
             response=TDI_AE, amp_scale=1.0, phase0=0.0, want_segments=False,
             want_kappa=False, nthreads=0):
    """Upsilon_N for every particle.

    data: dict with f_first, df, K, T_obs, A, E (complex128[K]), SA, SE
          (float64[K]; SE may be None); optionally the third channel T
          (complex128[K]) with its PSD ST (float64[K]).
    params: (P, 8) float64.
    Returns stat[P] and, on request, seg_x[P, N], seg_hh[P, N],
    kappa[P, N+1].
    """
    lib = _load()
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 8)
    P = params.shape[0]
    A = np.ascontiguousarray(data["A"], dtype=np.complex128)
    E = np.ascontiguousarray(data["E"], dtype=np.complex128)
    SA = np.ascontiguousarray(data["SA"], dtype=np.float64)
    SE = data.get("SE")
    SE = None if SE is None else np.ascontiguousarray(SE, dtype=np.float64)
    T = data.get("T")
    ST = None
    if T is not None:
        T = np.ascontiguousarray(T, dtype=np.complex128)
        ST = np.ascontiguousarray(data["ST"], dtype=np.float64)
    stat = np.zeros(P)
    sx = np.zeros((P, N)) if want_segments else None
    sh = np.zeros((P, N)) if want_segments else None
    kap = np.zeros((P, N + 1)) if want_kappa else None
    lib.orc_eval(float(data["f_first"]), float(data["df"]), int(data["K"]),
                 float(data["T_obs"]), _ptr(A), _ptr(E), _ptr(SA), _ptr(SE),
                 _ptr(T), _ptr(ST), int(N), int(mode), int(waveform), int(response), _ptr(params),
                 P, float(amp_scale), float(phase0), _ptr(stat), _ptr(sx),
                 _ptr(sh), _ptr(kap), int(nthreads))
    out = [stat]
    if want_segments:
        out += [sx, sh]
    if want_kappa:
        out.append(kap)
    return out[0] if len(out) == 1 else tuple(out)


def inner_dd(data):
    """<d|d> = sum_alpha sum_k 4 df |d_alpha(f_k)|^2 / S_alpha(f_k) (Eq. inner_prod
    on the FFT grid), over A, E and T when the data has T."""
    SA = np.asarray(data["SA"], np.float64)
    SE = SA if data.get("SE") is None else np.asarray(data["SE"], np.float64)
    A = np.asarray(data["A"])
    E = np.asarray(data["E"])
    out = (np.sum(4.0 * data["df"] * np.abs(A) ** 2 / SA)
           + np.sum(4.0 * data["df"] * np.abs(E) ** 2 / SE))
    if data.get("T") is not None:
        out += np.sum(4.0 * data["df"] * np.abs(np.asarray(data["T"])) ** 2
                      / np.asarray(data["ST"], np.float64))
    return float(out)


def loglike(data, params, N, mode=EQUAL_WIDTH, amp=None):
    """Semi-coherent log-likelihood (Sec. II.B):
    log L_N = -<d|d>/2 - <h|h>/2 + O_N(d, h),  O_N = sum_n x_n,
    for the templates a * h(theta) (a: amplitude per particle, default 1).
    Returns (logL, O_N of the unit templates, <h|h> of the unit templates)."""
    params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 8)
    stat, sx, sh = evaluate(data, params, N, mode=mode, want_segments=True)
    a = np.ones(len(params)) if amp is None else np.asarray(amp, np.float64)
    O = sx.sum(axis=1)
    H = sh.sum(axis=1)
    L = -0.5 * inner_dd(data) - 0.5 * a * a * H + a * O
    L = np.where(np.isfinite(stat), L, -np.inf)
    return L, O, H
