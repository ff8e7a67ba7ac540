"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/ipp.h declares, and rejects bad arguments on the host before any CUDA
work (no GPU call is made here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ipp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ipp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2502_10783_gb300 import _abi
    return _abi.load()


def test_every_declared_symbol_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    assert L.ipp_status_string(0) == b"ok"
    assert L.ipp_status_string(1) == b"invalid argument"
    assert L.ipp_status_string(99) == b"unknown status"
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    assert L.ipp_version(C.byref(a), C.byref(b), C.byref(c)) == 0 and (a.value, b.value) == (0, 1)


def test_host_side_validation(L):
    from paper_2502_10783_gb300 import _abi
    p = _abi.BgParams(64, 64, 3, 3, 10, 100, 0, 0, 3.0, 2.5, 1.5)
    fake = C.c_void_p(0x1000)  # never dereferenced: validation fails first
    # NULL image
    assert L.ipp_bg_estimate(None, 0, 100, 100, 100, None, None, p, fake, fake, None, None, None, fake,
                             1 << 20, None) == _abi.IPP_ERR_INVALID_ARG
    assert b"img" in L.ipp_last_error_detail()
    # pitch < W
    assert L.ipp_bg_estimate(fake, 0, 100, 100, 99, None, None, p, fake, fake, None, None, None, fake,
                             1 << 20, None) == _abi.IPP_ERR_INVALID_ARG
    # workspace too small
    assert L.ipp_bg_estimate(fake, 0, 100, 100, 100, None, None, p, fake, fake, None, None, None, fake,
                             1, None) == _abi.IPP_ERR_INVALID_ARG
    # even filter, mesh too small, mesh too large
    for bad in (_abi.BgParams(64, 64, 2, 3, 10, 100, 0, 0, 3.0, 2.5, 1.5),
                _abi.BgParams(3, 64, 3, 3, 10, 100, 0, 0, 3.0, 2.5, 1.5),
                _abi.BgParams(256, 128, 3, 3, 10, 100, 0, 0, 3.0, 2.5, 1.5)):
        assert L.ipp_bg_subtract(fake, 0, 100, 100, 100, None, fake, bad, fake, 100, None,
                                 None) == _abi.IPP_ERR_INVALID_ARG
    # uint16 frame without calibration
    assert L.ipp_bg_subtract(fake, 1, 100, 100, 100, None, fake, p, fake, 100, None, None) == 1
    # detection: min_area 0, missing stats
    st = _abi.SrcStats(*([0x1000] * 10))
    d0 = _abi.DetParams(1.5, 0.0, 0, 0)
    assert L.ipp_detect_label(fake, 100, 100, 100, fake, p, d0, None, fake, fake, 10, st, fake, 1 << 30,
                              None) == 1
    st_bad = _abi.SrcStats(*([0x1000] * 9 + [0]))
    d1 = _abi.DetParams(1.5, 0.0, 5, 0)
    assert L.ipp_detect_label(fake, 100, 100, 100, fake, p, d1, None, fake, fake, 10, st_bad, fake, 1 << 30,
                              None) == 1
    # aperture: r_out <= r_in, r_out beyond the supported 16 px
    assert L.ipp_aperture_phot(fake, 100, 100, 100, fake, 10, fake, fake, _abi.PhotParams(5, 8, 8, 10),
                               fake, None, None, None, None, None) == 1
    # PSF: unknown model, stamp size out of range, beta <= 1
    assert L.ipp_psf_fit(fake, 10, 15, None, None, _abi.FitParams(7, 2.5, 50, 1e-3), fake, fake, None, None,
                         None) == 1
    assert L.ipp_psf_fit(fake, 10, 40, None, None, _abi.FitParams(0, 2.5, 50, 1e-3), fake, fake, None, None,
                         None) == 1
    assert L.ipp_psf_model_fwd(fake, 10, 15, _abi.FitParams(0, 1.0, 0, 0), fake, None) == 1
    # empty batch is a no-op
    assert L.ipp_psf_fit(fake, 0, 15, None, None, _abi.FitParams(0, 2.5, 50, 1e-3), fake, fake, None, None,
                         None) == 0
    # the spline reading: an unknown interp is refused; calls that interpolate with
    # Keys only answer NOT_SUPPORTED before anything is enqueued
    assert L.ipp_bg_subtract(fake, 0, 100, 100, 100, None, fake, _abi.BgParams(64, 64, 3, 3, 10, 100, 0, 7, 3.0,
                             2.5, 1.5), fake, 100, None, None) == _abi.IPP_ERR_INVALID_ARG
    ps = _abi.BgParams(64, 64, 3, 3, 10, 100, 0, 1, 3.0, 2.5, 1.5)
    assert L.ipp_bg_subtract(fake, 0, 100, 100, 100, None, fake, ps, fake, 100, None,
                             None) == _abi.IPP_ERR_NOT_SUPPORTED
    st_ok = _abi.SrcStats(*([0x1000] * 10))
    assert L.ipp_detect_label(fake, 100, 100, 100, fake, ps, d1, None, fake, fake, 10, st_ok, fake, 1 << 30,
                              None) == _abi.IPP_ERR_NOT_SUPPORTED


def test_workspace_queries(L):
    from paper_2502_10783_gb300 import _abi
    p = _abi.BgParams(128, 128, 3, 3, 10, 100, 0, 0, 3.0, 2.5, 1.5)
    assert L.ipp_bg_estimate_workspace_size(4096, 4096, p) >= 4 * 32 * 32 * 4
    a = L.ipp_detect_label_workspace_size(4096, 4096)
    b = L.ipp_detect_label_workspace_size(1000, 1000)
    assert a > b > 0
    assert L.ipp_extract_workspace_size(4096, 4096, p) >= a
    # the spline node tables of the mesh bkg and rms are part of it, whatever interp says
    ps = _abi.BgParams(128, 128, 3, 3, 10, 100, 0, 1, 3.0, 2.5, 1.5)
    assert L.ipp_extract_workspace_size(4096, 4096, ps) == L.ipp_extract_workspace_size(4096, 4096, p)
    assert L.ipp_detect_label_workspace_size(0, 10) == 0
