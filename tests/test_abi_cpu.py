"""CPU-side checks of the C ABI library: it builds, loads without a GPU and
exports every entry point that include/scstat.h declares; argument errors
that need no device are reported as such."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header=None):
    """Functions declared by include/<header>, or by every header there."""
    inc = os.path.join(ROOT, "include")
    names = [header] if header else sorted(h for h in os.listdir(inc) if h.endswith(".h"))
    out = set()
    for h in names:
        src = open(os.path.join(inc, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        out.update(re.findall(r"\b(scs_[a-z0-9_]+)\s*\(", src))
    return sorted(out)


def test_header_declares_the_boundary():
    names = declared_functions("scstat.h")
    for want in ("scs_create", "scs_destroy", "scs_last_error", "scs_set_data",
                 "scs_set_data_aet", "scs_set_segments", "scs_eval_stat", "scs_waveform",
                 "scs_waveform_aet", "scs_inject"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2408_13170_gb300 import build
    lib = ctypes.CDLL(build.build())
    names = declared_functions()
    assert "scs_peak_probe" in names
    for name in names:
        assert hasattr(lib, name), name


def test_debug_build_compiles_and_exports_the_boundary():
    """The -DSCS_DEBUG variant (index checks, scs_debug_error) builds for
    sm_103a and exports the same entry points; its error reader refuses
    null arguments before touching a device."""
    from paper_2408_13170_gb300 import build
    path = build.build(debug=True)
    assert path.endswith("libscstat_debug.so")
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.scs_debug_error.argtypes = [ctypes.c_void_p] * 3
    assert lib.scs_debug_error(None, None, None) == -1   # SCS_EINVAL


def test_peak_probe_rejects_bad_arguments():
    """The probe checks its arguments before touching a device."""
    from paper_2408_13170_gb300 import scstat
    fn = scstat.lib().scs_peak_probe
    fn.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 3
    assert fn(0, 9, 10, None, None, None) == -1
    assert fn(0, 0, 0, None, None, None) == -1


def test_create_without_device_fails_cleanly():
    """On a host without a GPU, scs_create reports an error code (no crash);
    on a GPU host it succeeds."""
    from paper_2408_13170_gb300 import scstat
    import torch
    h = ctypes.c_void_p()
    rc = scstat.lib().scs_create(ctypes.byref(h), 0, scstat.SCS_MIXED)
    if torch.cuda.is_available():
        assert rc == scstat.SCS_OK
        scstat.lib().scs_destroy(h)
    else:
        assert rc in (scstat.SCS_EINVAL, scstat.SCS_ECUDA)
        assert not h.value
    assert scstat.lib().scs_create(ctypes.byref(h), 0, 7) == scstat.SCS_EINVAL
    assert scstat.lib().scs_create(None, 0, 0) == scstat.SCS_EINVAL


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No CPU fallback: if the library cannot be built or loaded, the
    binding raises instead of computing anything."""
    from paper_2408_13170_gb300 import scstat, build

    def broken(*a, **k):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libscstat")

    saved = scstat._lib
    monkeypatch.setattr(build, "build", broken)
    monkeypatch.setattr(scstat, "_lib", None)
    try:
        with pytest.raises(RuntimeError):
            scstat.lib()
        with pytest.raises(RuntimeError):
            scstat.Context(0)
    finally:
        scstat._lib = saved
