"""The C ABI: the library loads, exports every function include/fv.h declares,
and validates arguments on the host before touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2506_02130_gb300 import fv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fv_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2506_02130_gb300.build import build
    build()
    return fv.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"fv_plan", "fv_set_array", "fv_set_sky", "fv_execute", "fv_destroy"} <= names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(fv.SIGNATURES) >= names


def test_abi_version_and_defaults(lib):
    assert lib.fv_abi_version() == 5
    o = fv.fv_opts_default()
    assert o.precision == fv.FV_FP64 and o.eps == 1e-10 and o.upsampfac == 2.0 and o.device == -1
    assert o.transform == 0 and o.lattice_tol_m == 0.0
    assert list(o.bin_size) == [0, 0] and o.spread_method == 0 and o.heights == 0
    assert abs(o.beam_param[0] - np.radians(10)) < 1e-15 and o.beam_param[1] == 150e6


def _opts(**kw):
    o = fv.fv_opts_default()
    f = np.array([150e6]); t = np.array([0.1])
    o.n_freq, o.freq_hz = 1, f.ctypes.data_as(C.POINTER(C.c_double))
    o.n_time, o.lst_rad = 1, t.ctypes.data_as(C.POINTER(C.c_double))
    for k, v in kw.items():
        setattr(o, k, v)
    return o, (f, t)


@pytest.mark.parametrize("kw", [dict(eps=0.0), dict(eps=1e-15), dict(precision=1, eps=1e-9), dict(precision=7),
                                dict(n_freq=0), dict(beam=9), dict(dims=4), dict(upsampfac=1.1),
                                dict(kernel_width=40), dict(latitude_rad=2.0),
                                dict(precision=1, eps=1e-6, upsampfac=1.25), dict(transform=4),
                                dict(transform=3, n_basis=-1), dict(transform=3, n_basis=2),
                                dict(lattice_tol_m=-1.0), dict(spread_method=5),
                                dict(bin_size=(C.c_int * 2)(0, 65)),
                                dict(bin_size=(C.c_int * 2)(-2, 4)), dict(heights=3), dict(heights=-1)])
def test_invalid_options_rejected_before_device(lib, kw):
    o, keep = _opts(**kw)
    h = C.c_void_p()
    st = lib.fv_plan(C.byref(o), C.byref(h))
    assert st == fv.FV_ERR_ARG
    assert h.value is None
    assert lib.fv_last_error(None)


def test_null_arguments(lib):
    assert lib.fv_plan(None, None) == fv.FV_ERR_ARG
    assert lib.fv_execute(None, None, 0) == fv.FV_ERR_ARG
    assert lib.fv_destroy(None) == fv.FV_OK


def test_no_device_is_an_error_not_a_fallback(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    o, keep = _opts()
    h = C.c_void_p()
    assert lib.fv_plan(C.byref(o), C.byref(h)) == fv.FV_ERR_CUDA
    with pytest.raises(fv.FvError):
        fv.Plan.create([150e6], [0.0], 0.0)


@pytest.mark.parametrize("eps,sigma,ok", [(1e-10, 1.25, False), (1e-8, 1.25, True), (1e-14, 2.0, True),
                                          (1e-12, 1.5, False)])
def test_unreachable_tolerance_is_refused_not_clamped(lib, eps, sigma, ok):
    """A tolerance that needs a kernel wider than 16 points at the given
    upsampling factor is refused (FV_ERR_UNSUPPORTED) before any device work."""
    o, keep = _opts(eps=eps, upsampfac=sigma)
    h = C.c_void_p()
    st = lib.fv_plan(C.byref(o), C.byref(h))
    if ok:
        assert st != fv.FV_ERR_UNSUPPORTED and st != fv.FV_ERR_ARG   # FV_ERR_CUDA here (no device) or FV_OK
        if h.value:
            lib.fv_destroy(h)
    else:
        assert st == fv.FV_ERR_UNSUPPORTED
        assert b"kernel width" in lib.fv_last_error(None)
