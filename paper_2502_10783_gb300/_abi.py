"""ctypes view of include/ipp.h: structs, status codes and function prototypes.

Argument marshalling only.  Loading fails loudly when libipp.so is missing:
there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

IPP_OK, IPP_ERR_INVALID_ARG, IPP_ERR_CUDA, IPP_ERR_CAPACITY = 0, 1, 2, 3
IPP_ERR_NO_VALID_MESH, IPP_ERR_TIMEOUT, IPP_ERR_NOT_SUPPORTED, IPP_ERR_DEGENERATE = 4, 5, 6, 7
IPP_F32, IPP_U16 = 0, 1
FLAG_EDGE, FLAG_WIN_NOT_CONVERGED, FLAG_ANN_FEW = 1, 2, 4
FLAG_FIT_MAXITER, FLAG_FIT_SINGULAR, FLAG_FIT_BAD_SIGMA = 8, 16, 32
EST_SIGMA, EST_MEDIAN, EST_MEAN, EST_FACTORS = 0, 1, 2, 3
PSF_MOFFAT, PSF_GAUSS = 0, 1
GRAY_LINEAR, GRAY_LOG, GRAY_POWER, GRAY_EXP = 0, 1, 2, 3

vp, i32, i64, f32, f64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_size_t


class BgParams(C.Structure):
    _fields_ = [("mesh_w", i32), ("mesh_h", i32), ("filter_w", i32), ("filter_h", i32),
                ("maxiters", i32), ("min_valid", i32), ("estimator", i32), ("interp", i32),
                ("nsigma", f64), ("median_factor", f64), ("mean_factor", f64)]


class DetParams(C.Structure):
    _fields_ = [("k", f32), ("thresh_abs", f32), ("min_area", i32), ("filter", i32)]


class CenParams(C.Structure):
    _fields_ = [("fwhm_win", f32), ("max_iter", i32), ("tol2", f32), ("reserved", i32)]


class PhotParams(C.Structure):
    _fields_ = [("r_ap", f32), ("r_in", f32), ("r_out", f32), ("min_ann", i32)]


class Wcs(C.Structure):
    _fields_ = [("crpix", f64 * 2), ("crval", f64 * 2), ("cd", f64 * 4), ("a_order", i32), ("b_order", i32),
                ("a", f64 * 36), ("b", f64 * 36)]


class ZscaleParams(C.Structure):
    _fields_ = [("n_samples", i32), ("contrast", f32), ("krej", f32), ("max_iter", i32)]


class DeblendParams(C.Structure):
    _fields_ = [("nthresh", i32), ("mincont", f32)]


class AutoParams(C.Structure):
    _fields_ = [("k_kron", f32), ("r_min", f32), ("r_kmax", f32), ("reserved", i32)]


class FitParams(C.Structure):
    _fields_ = [("model", i32), ("beta", f32), ("max_iter", i32), ("lambda0", f32)]


class SrcStats(C.Structure):
    _fields_ = [(n, vp) for n in ("area", "first", "xmin", "xmax", "ymin", "ymax", "peak", "flux",
                                  "xbar", "ybar")]


class Calib(C.Structure):
    _fields_ = [("bias_map", vp), ("bias", f32), ("reserved", i32), ("inv_flat", vp)]


class CatalogOut(C.Structure):
    _fields_ = [("mesh_bkg", vp), ("mesh_rms", vp), ("sub", vp), ("labels", vp), ("n_src_dev", vp),
                ("stats", SrcStats), ("x", vp), ("y", vp), ("cen_flags", vp), ("flux", vp),
                ("sky", vp), ("area", vp), ("n_ann", vp), ("phot_flags", vp), ("status_dev", vp)]


class FrameDesc(C.Structure):
    _fields_ = [("img", vp), ("dtype", i32), ("reserved", i32), ("W", i64), ("H", i64), ("pitch", i64),
                ("cal", C.POINTER(Calib)), ("out", CatalogOut)]


IPP_BATCH_MAX_LANES = 8
_par = [C.POINTER(BgParams), C.POINTER(DetParams), C.POINTER(CenParams), C.POINTER(PhotParams), i32]

PROTOTYPES = {
    "ipp_status_string": ([i32], C.c_char_p),
    "ipp_last_error_detail": ([], C.c_char_p),
    "ipp_version": ([vp, vp, vp], i32),
    "ipp_bg_estimate_workspace_size": ([i64, i64, C.POINTER(BgParams)], sz),
    "ipp_bg_estimate": ([vp, i32, i64, i64, i64, vp, C.POINTER(Calib), C.POINTER(BgParams), vp, vp, vp, vp,
                         vp, vp, sz, vp], i32),
    "ipp_bg_estimate_noalloc": ([vp, i32, i64, i64, i64, vp, C.POINTER(Calib), C.POINTER(BgParams), vp, vp, vp,
                                 vp], i32),
    "ipp_bg_spline_workspace_size": ([i64, i64, C.POINTER(BgParams)], C.c_size_t),
    "ipp_bg_subtract_spline": ([vp, i32, i64, i64, i64, C.POINTER(Calib), vp, C.POINTER(BgParams), vp, i64, vp,
                                vp, C.c_size_t, vp], i32),
    "ipp_bg_subtract": ([vp, i32, i64, i64, i64, C.POINTER(Calib), vp, C.POINTER(BgParams), vp, i64, vp, vp],
                        i32),
    "ipp_detect_label_workspace_size": ([i64, i64], sz),
    "ipp_detect_label": ([vp, i64, i64, i64, vp, C.POINTER(BgParams), C.POINTER(DetParams), vp, vp, vp, i32,
                          C.POINTER(SrcStats), vp, sz, vp], i32),
    "ipp_centroid": ([vp, i64, i64, i64, vp, i32, vp, vp, C.POINTER(CenParams), vp, vp, vp, vp, vp], i32),
    "ipp_aperture_phot": ([vp, i64, i64, i64, vp, i32, vp, vp, C.POINTER(PhotParams), vp, vp, vp, vp, vp, vp],
                          i32),
    "ipp_deblend_workspace_size": ([i64, i64, i32], sz),
    "ipp_deblend": ([vp, vp, i64, i64, i64, vp, i32, C.POINTER(SrcStats), C.POINTER(DeblendParams), vp, vp, vp, sz,
                     vp], i32),
    "ipp_clean_workspace_size": ([i32], sz),
    "ipp_clean": ([vp, vp, i64, i64, i64, vp, i32, vp, vp, C.POINTER(BgParams), C.POINTER(DetParams), C.c_float, vp,
                   vp, vp, sz, vp], i32),
    "ipp_auto_phot": ([vp, vp, i64, i64, i64, vp, i32, C.POINTER(SrcStats), C.POINTER(AutoParams), vp, vp, vp,
                       vp, vp, vp], i32),
    "ipp_wcs_map": ([C.POINTER(Wcs), C.POINTER(Wcs), i64, i64, i32, vp, vp, vp], i32),
    "ipp_affine_fit_workspace_size": ([], sz),
    "ipp_affine_fit": ([vp, vp, vp, vp, i64, i64, i32, vp, vp, vp, sz, vp], i32),
    "ipp_reproject_affine": ([vp, i64, i64, i64, vp, i64, i64, f32, vp, i64, vp], i32),
    "ipp_zscale": ([vp, i64, i64, i64, C.POINTER(ZscaleParams), vp, vp, vp], i32),
    "ipp_sub_apply_workspace_size": ([i32, i32, vp], sz),
    "ipp_sub_apply": ([vp, vp, i64, i64, i64, i32, i32, vp, vp, vp, i32, i32, vp, i64, vp, sz, vp], i32),
    "ipp_sub_fit_workspace_size": ([i32, i32, i32, i32, i32, vp, i32, i32], sz),
    "ipp_sub_stamps": ([vp, vp, i64, i64, i64, i32, i32, i32, i32, C.c_double, vp, vp, vp, vp, sz, vp], i32),
    "ipp_sub_normal": ([vp, vp, i64, i64, i64, vp, vp, vp, i32, i32, i32, i32, vp, vp, i32, i32, vp, vp, vp, sz, vp],
                       i32),
    "ipp_sub_solve": ([vp, vp, i32, vp, vp, vp, vp], i32),
    "ipp_sub_fit": ([vp, vp, i64, i64, i64, i32, i32, C.c_double, i32, i32, i32, vp, vp, i32, i32, vp, vp, vp, vp, vp,
                     vp, vp, sz, vp], i32),
    "ipp_gray_transform": ([vp, i64, i64, i64, i32, f32, f32, f32, vp, i64, vp], i32),
    "ipp_hist_equalize_workspace_size": ([i32], sz),
    "ipp_hist_equalize": ([vp, i64, i64, i64, i32, vp, i64, vp, sz, vp], i32),
    "ipp_stamp_cut": ([vp, i64, i64, i64, vp, i32, vp, vp, i32, vp, vp, vp, vp, vp], i32),
    "ipp_extract_workspace_size": ([i64, i64, C.POINTER(BgParams)], sz),
    "ipp_extract": ([vp, i32, i64, i64, i64, C.POINTER(Calib), C.POINTER(BgParams), C.POINTER(DetParams),
                     C.POINTER(CenParams), C.POINTER(PhotParams), i32, C.POINTER(CatalogOut), vp, sz, vp], i32),
    "ipp_batch_workspace_size": ([i64, i64, C.POINTER(BgParams), i32], sz),
    "ipp_batch_create": ([i32, C.POINTER(vp)], i32),
    "ipp_batch_destroy": ([vp], i32),
    "ipp_batch_extract": ([vp, C.POINTER(FrameDesc), i32] + _par + [vp, sz, vp], i32),
    "ipp_batch_capture": ([vp, C.POINTER(FrameDesc), i32] + _par + [vp, sz, vp], i32),
    "ipp_batch_launch": ([vp, vp], i32),
    "ipp_batch_table_workspace_size": ([C.POINTER(FrameDesc), i32, C.POINTER(BgParams)], sz),
    "ipp_batch_table_extract": ([vp, C.POINTER(FrameDesc), i32] + _par + [vp, sz, vp], i32),
    "ipp_batch_table_capture": ([vp, C.POINTER(FrameDesc), i32] + _par + [vp, sz, vp], i32),
    "ipp_batch_autotune": ([C.POINTER(FrameDesc), i32] + _par + [vp, sz, vp, C.POINTER(i32), C.POINTER(f32)],
                           i32),
    "ipp_psf_fit": ([vp, i64, i32, vp, vp, C.POINTER(FitParams), vp, vp, vp, vp, vp], i32),
    "ipp_psf_fit_dev": ([vp, vp, i64, i32, vp, vp, C.POINTER(FitParams), vp, vp, vp, vp, vp], i32),
    "ipp_psf_model_fwd": ([vp, i64, i32, C.POINTER(FitParams), vp, vp], i32),
    "ipp_psf_model_adj": ([vp, i64, i32, C.POINTER(FitParams), vp, vp, vp], i32),
}

_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libipp.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libipp.so not found at {_build.LIB}: build it with "
                               "`python -m paper_2502_10783_gb300._build`")
        L = C.CDLL(_build.LIB)
        for name, (args, res) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


class IppError(RuntimeError):
    def __init__(self, fn, status):
        L = load(False)
        detail = L.ipp_last_error_detail().decode(errors="replace")
        super().__init__(f"{fn}: {L.ipp_status_string(status).decode()} ({status}): {detail}")
        self.status = status


def check(fn: str, status: int) -> None:
    if status != IPP_OK:
        raise IppError(fn, status)
