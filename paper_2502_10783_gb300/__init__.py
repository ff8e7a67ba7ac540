"""GB300 (sm_103a) catalog path of the GPU image pre-processing method of
Cao, Jia et al. (arXiv 2502.10783): mesh background estimation and subtraction
(Sec. 2.2.2), threshold detection with connected-component labeling and
per-candidate statistics, windowed centroids and aperture photometry with a
local sky annulus (Sec. 2.2.5), and a batched differentiable PSF fit.

Every step runs in the CUDA kernels of libipp.so behind the C ABI of
include/ipp.h.  This module only marshals arguments: it allocates outputs and
workspaces with torch, passes raw device pointers and the current stream, and
raises when a call returns an error status.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _abi
from ._abi import (  # noqa: F401
    EST_FACTORS, EST_MEAN, EST_MEDIAN, EST_SIGMA, FLAG_ANN_FEW, FLAG_EDGE, FLAG_FIT_BAD_SIGMA,
    FLAG_FIT_MAXITER, FLAG_FIT_SINGULAR, FLAG_WIN_NOT_CONVERGED, GRAY_EXP, GRAY_LINEAR, GRAY_LOG, GRAY_POWER,
    IppError, PSF_GAUSS, PSF_MOFFAT,
)

__all__ = ["load", "bg_estimate", "bg_subtract", "detect_label", "centroid", "aperture_phot", "auto_phot", "deblend", "clean", "bg_subtract_spline", "sub_stamps", "sub_normal", "sub_solve", "sub_fit", "stamp_cut", "Batch",
           "gray_transform", "hist_equalize", "zscale", "sub_apply", "wcs_map", "affine_fit", "reproject_affine", "align",
           "extract", "Extractor", "psf_fit", "psf_model", "PSFModel", "BgConfig"]


def load():
    """Load (building if needed) the CUDA library; raises if it cannot."""
    return _abi.load()


def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _need_cuda(t, name, dtype=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")


@dataclass
class BgConfig:
    """Mesh background parameters (Sec. 2.2.2); defaults as in the paper (64 px meshes)."""
    mesh: int = 64
    mesh_h: int | None = None
    filter_size: int = 3
    maxiters: int = 10
    min_valid: int = 100
    nsigma: float = 3.0
    estimator: int = EST_SIGMA
    median_factor: float = 2.5
    mean_factor: float = 1.5
    interp: str = "keys"    # "keys" (Keys cubic convolution) or "spline" (natural tensor spline)

    def c(self):
        if self.interp not in ("keys", "spline"):
            raise ValueError("interp is 'keys' or 'spline'")
        return _abi.BgParams(self.mesh, self.mesh_h or self.mesh, self.filter_size, self.filter_size,
                             self.maxiters, self.min_valid, self.estimator, int(self.interp == "spline"),
                             self.nsigma, self.median_factor, self.mean_factor)

    def grid(self, W, H):
        mh = self.mesh_h or self.mesh
        return -(-W // self.mesh), -(-H // mh)


def _bgcfg(cfg, kw):
    if cfg is None:
        cfg = BgConfig(**kw)
    return cfg


def _frame(img, calib):
    if img.dtype == torch.float32:
        return _abi.IPP_F32, None
    if img.dtype in (torch.uint16, torch.int16):
        if calib is None:
            raise ValueError("uint16 frames need calib=(inv_flat, bias[, bias_map])")
        inv_flat, bias = calib[0], calib[1]
        bias_map = calib[2] if len(calib) > 2 else None
        return _abi.IPP_U16, _abi.Calib(_ptr(bias_map), float(bias), 0, _ptr(inv_flat))
    raise TypeError(f"unsupported frame dtype {img.dtype}")


def bg_estimate(img, mask=None, cfg: BgConfig | None = None, raw=False, calib=None, ws=None, **kw):
    """Filtered mesh background and rms grids, float32 [ny, nx] (ipp_bg_estimate)."""
    L = load()
    cfg = _bgcfg(cfg, kw)
    _need_cuda(img, "img")
    H, W = img.shape
    dtype, cal = _frame(img, calib)
    p = cfg.c()
    nx, ny = cfg.grid(W, H)
    dev = img.device
    bkg = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    rms = torch.empty_like(bkg)
    rb = torch.empty_like(bkg) if raw else None
    rr = torch.empty_like(bkg) if raw else None
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    need = L.ipp_bg_estimate_workspace_size(W, H, p)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    m = None if mask is None else mask.to(torch.uint8).contiguous()
    _abi.check("ipp_bg_estimate", L.ipp_bg_estimate(
        _ptr(img), dtype, W, H, img.stride(0), _ptr(m), cal, p, _ptr(bkg), _ptr(rms), _ptr(rb), _ptr(rr),
        _ptr(status), _ptr(ws), ws.numel(), _stream()))
    if raw:
        return bkg, rms, rb, rr, status
    return bkg, rms


def bg_subtract(img, mesh_bkg, cfg: BgConfig | None = None, bkg_map=False, calib=None, out=None, **kw):
    """Background-subtracted frame (ipp_bg_subtract); optionally the background map."""
    L = load()
    cfg = _bgcfg(cfg, kw)
    _need_cuda(img, "img")
    _need_cuda(mesh_bkg, "mesh_bkg", torch.float32)
    H, W = img.shape
    dtype, cal = _frame(img, calib)
    sub = out if out is not None else torch.empty((H, W), dtype=torch.float32, device=img.device)
    bmap = torch.empty_like(sub) if bkg_map else None
    _abi.check("ipp_bg_subtract", L.ipp_bg_subtract(
        _ptr(img), dtype, W, H, img.stride(0), cal, _ptr(mesh_bkg.contiguous()), cfg.c(), _ptr(sub),
        sub.stride(0), _ptr(bmap), _stream()))
    return (sub, bmap) if bkg_map else sub


def bg_subtract_spline(img, mesh_bkg, cfg: BgConfig | None = None, bkg_map=False, calib=None, out=None, ws=None,
                       **kw):
    """Background-subtracted frame with the natural-spline map (ipp_bg_subtract_spline)."""
    L = load()
    cfg = _bgcfg(cfg, kw)
    _need_cuda(img, "img")
    _need_cuda(mesh_bkg, "mesh_bkg", torch.float32)
    H, W = img.shape
    dtype, cal = _frame(img, calib)
    p = cfg.c()
    sub = out if out is not None else torch.empty((H, W), dtype=torch.float32, device=img.device)
    bmap = torch.empty_like(sub) if bkg_map else None
    need = L.ipp_bg_spline_workspace_size(W, H, p)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=img.device)
    _abi.check("ipp_bg_subtract_spline", L.ipp_bg_subtract_spline(
        _ptr(img), dtype, W, H, img.stride(0), cal, _ptr(mesh_bkg.contiguous()), p, _ptr(sub),
        sub.stride(0), _ptr(bmap), _ptr(ws), ws.numel(), _stream()))
    return (sub, bmap) if bkg_map else sub


_STAT_TYPES = dict(area=torch.int32, first=torch.int64, xmin=torch.int32, xmax=torch.int32,
                   ymin=torch.int32, ymax=torch.int32, peak=torch.float32, flux=torch.float32,
                   xbar=torch.float32, ybar=torch.float32)


def _alloc_stats(max_src, dev):
    return {k: torch.empty(max(max_src, 1), dtype=t, device=dev) for k, t in _STAT_TYPES.items()}


def _stats_c(st):
    return _abi.SrcStats(*[_ptr(st.get(k)) for k in _STAT_TYPES])


def detect_label(sub, mesh_rms=None, cfg: BgConfig | None = None, k=1.5, thresh_abs=0.0, min_area=5,
                 mask_in=None, max_src=None, ws=None, filter=0, **kw):
    """Labels, device source count and per-source stats (ipp_detect_label).

    mask_in: optional packed bit mask (uint32 words, ceil(W/32) per row) that
    replaces the threshold.  filter=1 thresholds the frame smoothed by the
    3 x 3 pyramid detection filter."""
    L = load()
    cfg = _bgcfg(cfg, kw)
    _need_cuda(sub, "sub", torch.float32)
    H, W = sub.shape
    dev = sub.device
    if max_src is None:
        max_src = max(1024, (H * W) // 64)
    labels = torch.empty((H, W), dtype=torch.int32, device=dev)
    n_src = torch.zeros(1, dtype=torch.int32, device=dev)
    st = _alloc_stats(max_src, dev)
    need = L.ipp_detect_label_workspace_size(W, H)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    mi = None
    if mask_in is not None:
        _need_cuda(mask_in, "mask_in")
        mi = mask_in.contiguous()
    rms = None if mesh_rms is None else mesh_rms.contiguous()
    _abi.check("ipp_detect_label", L.ipp_detect_label(
        _ptr(sub), W, H, sub.stride(0), _ptr(rms), cfg.c(), _abi.DetParams(k, thresh_abs, min_area, filter),
        _ptr(mi), _ptr(labels), _ptr(n_src), max_src, _stats_c(st), _ptr(ws), ws.numel(), _stream()))
    return labels, n_src, st


def centroid(sub, x0, y0, n_src=None, fwhm_win=3.0, max_iter=16, tol2=1e-8, max_src=None):
    """Windowed centroids (ipp_centroid); returns x, y, niter, flags."""
    L = load()
    _need_cuda(sub, "sub", torch.float32)
    H, W = sub.shape
    n = x0.numel() if max_src is None else max_src
    if n_src is None:
        n_src = torch.tensor([x0.numel()], dtype=torch.int32, device=sub.device)
    x = torch.empty(max(n, 1), dtype=torch.float32, device=sub.device)
    y, it = torch.empty_like(x), torch.empty(max(n, 1), dtype=torch.int32, device=sub.device)
    fl = torch.empty_like(it)
    _abi.check("ipp_centroid", L.ipp_centroid(
        _ptr(sub), W, H, sub.stride(0), _ptr(n_src), n, _ptr(x0.contiguous()), _ptr(y0.contiguous()),
        _abi.CenParams(fwhm_win, max_iter, tol2, 0), _ptr(x), _ptr(y), _ptr(it), _ptr(fl), _stream()))
    return x[:n], y[:n], it[:n], fl[:n]


def aperture_phot(sub, x, y, n_src=None, r_ap=5.0, r_in=8.0, r_out=12.0, min_ann=10, max_src=None):
    """Aperture photometry with a sky annulus (ipp_aperture_phot)."""
    L = load()
    _need_cuda(sub, "sub", torch.float32)
    H, W = sub.shape
    n = x.numel() if max_src is None else max_src
    if n_src is None:
        n_src = torch.tensor([x.numel()], dtype=torch.int32, device=sub.device)
    dev = sub.device
    out = dict(flux=torch.empty(max(n, 1), dtype=torch.float32, device=dev))
    out["sky"] = torch.empty_like(out["flux"])
    out["area"] = torch.empty_like(out["flux"])
    out["n_ann"] = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    out["flags"] = torch.empty_like(out["n_ann"])
    _abi.check("ipp_aperture_phot", L.ipp_aperture_phot(
        _ptr(sub), W, H, sub.stride(0), _ptr(n_src), n, _ptr(x.contiguous()), _ptr(y.contiguous()),
        _abi.PhotParams(r_ap, r_in, r_out, min_ann), _ptr(out["flux"]), _ptr(out["sky"]), _ptr(out["area"]),
        _ptr(out["n_ann"]), _ptr(out["flags"]), _stream()))
    return {k: v[:n] for k, v in out.items()}


def deblend(sub, labels, n_src, stats, nthresh=32, mincont=0.005, max_src=None, ws=None):
    """Deblended label map and device object count (ipp_deblend).  `labels`,
    `n_src` and `stats` as returned by detect_label."""
    L = load()
    _need_cuda(sub, "sub", torch.float32)
    _need_cuda(labels, "labels", torch.int32)
    H, W = sub.shape
    n = stats["xbar"].numel() if max_src is None else max_src
    dev = sub.device
    need = L.ipp_deblend_workspace_size(W, H, n)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    out = torch.empty((H, W), dtype=torch.int32, device=dev)
    n_out = torch.empty(1, dtype=torch.int32, device=dev)
    _abi.check("ipp_deblend", L.ipp_deblend(
        _ptr(sub), _ptr(labels.contiguous()), W, H, sub.stride(0), _ptr(n_src), n, _stats_c(stats),
        _abi.DeblendParams(nthresh, mincont), _ptr(out), _ptr(n_out), _ptr(ws), ws.numel(), _stream()))
    return out, n_out


def clean(sub, labels, n_obj, max_obj, thr_map=None, mesh_rms=None, cfg: BgConfig | None = None, k=1.5,
          thresh_abs=0.0, beta=1.0, ws=None, **kw):
    """Cleaned label map and device object count (ipp_clean).  The threshold at an
    object's peak is thr_map there, else max(k rms, thresh_abs) with rms the
    Keys interpolation of mesh_rms on the grid of cfg, else thresh_abs."""
    L = load()
    cfg = _bgcfg(cfg, kw)
    _need_cuda(sub, "sub", torch.float32)
    _need_cuda(labels, "labels", torch.int32)
    H, W = sub.shape
    dev = sub.device
    need = L.ipp_clean_workspace_size(max_obj)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    out = torch.empty((H, W), dtype=torch.int32, device=dev)
    n_out = torch.empty(1, dtype=torch.int32, device=dev)
    if thr_map is not None:
        _need_cuda(thr_map, "thr_map", torch.float32)
        thr_map = thr_map.contiguous()
    _abi.check("ipp_clean", L.ipp_clean(
        _ptr(sub), _ptr(labels.contiguous()), W, H, sub.stride(0), _ptr(n_obj), max_obj, _ptr(thr_map),
        _ptr(None if mesh_rms is None else mesh_rms.contiguous()), cfg.c(), _abi.DetParams(k, thresh_abs, 1, 0),
        float(beta), _ptr(out), _ptr(n_out), _ptr(ws), ws.numel(), _stream()))
    return out, n_out


def auto_phot(sub, labels, n_src, stats, k_kron=2.5, r_min=3.5, r_kmax=6.0, max_src=None):
    """Auto (Kron) photometry of the labelled sources (ipp_auto_phot): flux,
    area, Kron radius, moments (x2, y2, xy) and flags per source.  `labels`,
    `n_src` and `stats` as returned by detect_label."""
    L = load()
    _need_cuda(sub, "sub", torch.float32)
    _need_cuda(labels, "labels", torch.int32)
    H, W = sub.shape
    n = stats["xbar"].numel() if max_src is None else max_src
    dev = sub.device
    out = dict(flux=torch.empty(max(n, 1), dtype=torch.float32, device=dev))
    out["area"] = torch.empty_like(out["flux"])
    out["kron"] = torch.empty_like(out["flux"])
    out["shape"] = torch.empty((max(n, 1), 3), dtype=torch.float32, device=dev)
    out["flags"] = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    _abi.check("ipp_auto_phot", L.ipp_auto_phot(
        _ptr(sub), _ptr(labels.contiguous()), W, H, sub.stride(0), _ptr(n_src), n, _stats_c(stats),
        _abi.AutoParams(k_kron, r_min, r_kmax, 0), _ptr(out["flux"]), _ptr(out["area"]), _ptr(out["kron"]),
        _ptr(out["shape"]), _ptr(out["flags"]), _stream()))
    return {k: v[:n] for k, v in out.items()}


def _frame2d(img, name):
    _need_cuda(img, name, torch.float32)
    if img.dim() != 2 or img.stride(1) != 1:
        raise TypeError(f"{name} must be a 2-D tensor with unit column stride")


def gray_transform(img, kind, lo, hi, a=1000.0, out=None):
    """Value-to-gray map of the frame (ipp_gray_transform): GRAY_LINEAR, GRAY_LOG,
    GRAY_POWER or GRAY_EXP of clip((x - lo) / (hi - lo), 0, 1)."""
    L = load()
    _frame2d(img, "img")
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    _frame2d(out, "out")
    _abi.check("ipp_gray_transform", L.ipp_gray_transform(
        _ptr(img), W, H, img.stride(0), int(kind), float(lo), float(hi), float(a), _ptr(out), out.stride(0),
        _stream()))
    return out


def _sub_basis_args(sig, deg, sord, bord):
    sg = np.ascontiguousarray(sig, np.float64)
    dg = np.ascontiguousarray(deg, np.int32)
    nb = sum((int(d) + 1) * (int(d) + 2) // 2 for d in dg)
    npar = nb * (sord + 1) * (sord + 2) // 2 + ((bord + 1) * (bord + 2) // 2 if bord >= 0 else 0)
    return sg, dg, npar


def _pair(img, tmpl):
    _frame2d(img, "img")
    _frame2d(tmpl, "tmpl")
    if tmpl.shape != img.shape or tmpl.stride(0) != img.stride(0):
        raise TypeError("img and tmpl must have the same shape and row pitch")


def sub_stamps(img, tmpl, nsx=10, nsy=10, hw=10, fh=10, nsig=5.0, ws=None):
    """Candidate stamp centres of the subtraction fit (ipp_sub_stamps): device
    int32 cx, cy (nsx * nsy, the first n valid) and the device count n."""
    L = load()
    _pair(img, tmpl)
    H, W = img.shape
    dev = img.device
    dg = np.zeros(1, np.int32)
    need = L.ipp_sub_fit_workspace_size(0, nsx * nsy, int(hw), int(fh), 1, dg.ctypes.data_as(C.c_void_p), 0, -1)
    if ws is None or ws.numel() < need:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    cx = torch.empty(nsx * nsy, dtype=torch.int32, device=dev)
    cy = torch.empty_like(cx)
    n = torch.empty(1, dtype=torch.int32, device=dev)
    _abi.check("ipp_sub_stamps", L.ipp_sub_stamps(
        _ptr(img), _ptr(tmpl), W, H, img.stride(0), int(nsx), int(nsy), int(hw), int(fh), float(nsig), _ptr(cx),
        _ptr(cy), _ptr(n), _ptr(ws), ws.numel(), _stream()))
    return cx, cy, n


def sub_normal(img, tmpl, cx, cy, n, hw=10, fh=10, sig=(0.7, 1.5, 3.0), deg=(6, 4, 2), sord=2, bord=1, ws=None):
    """Normal equations (AtA, Atb) of the subtraction fit over candidates
    cx[:n], cy[:n] (ipp_sub_normal), FP64 device tensors."""
    L = load()
    _pair(img, tmpl)
    H, W = img.shape
    dev = img.device
    sg, dg, npar = _sub_basis_args(sig, deg, sord, bord)
    max_c = cx.numel()
    need = L.ipp_sub_fit_workspace_size(max_c, 0, int(hw), int(fh), len(dg), dg.ctypes.data_as(C.c_void_p),
                                        int(sord), int(bord))
    if need == 0:
        raise ValueError("bad basis description")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    AtA = torch.empty((npar, npar), dtype=torch.float64, device=dev)
    Atb = torch.empty(npar, dtype=torch.float64, device=dev)
    _abi.check("ipp_sub_normal", L.ipp_sub_normal(
        _ptr(img), _ptr(tmpl), W, H, img.stride(0), _ptr(cx.contiguous()), _ptr(cy.contiguous()), _ptr(n), max_c,
        int(hw), int(fh), len(dg), sg.ctypes.data_as(C.c_void_p), dg.ctypes.data_as(C.c_void_p), int(sord),
        int(bord), _ptr(AtA), _ptr(Atb), _ptr(ws), ws.numel(), _stream()))
    return AtA, Atb


def sub_solve(AtA, Atb):
    """Cholesky solve of the normal equations on the device (ipp_sub_solve);
    overwrites AtA (L) and Atb; returns (coef64, coef32, status) device tensors."""
    L = load()
    npar = Atb.numel()
    c64 = torch.empty(npar, dtype=torch.float64, device=Atb.device)
    c32 = torch.empty(npar, dtype=torch.float32, device=Atb.device)
    st = torch.empty(1, dtype=torch.int32, device=Atb.device)
    _abi.check("ipp_sub_solve", L.ipp_sub_solve(_ptr(AtA), _ptr(Atb), npar, _ptr(c64), _ptr(c32), _ptr(st),
                                                _stream()))
    return c64, c32, st


def sub_fit(img, tmpl, nsx=10, nsy=10, nsig=5.0, hw=10, fh=10, sig=(0.7, 1.5, 3.0), deg=(6, 4, 2), sord=2, bord=1,
            ws=None):
    """The subtraction fit on the device (ipp_sub_fit): dict of device tensors
    coef64, coef (float, the input of sub_apply), cx, cy, n and status (0 =
    solved, 1 = the normal matrix is not positive definite)."""
    L = load()
    _pair(img, tmpl)
    H, W = img.shape
    dev = img.device
    sg, dg, npar = _sub_basis_args(sig, deg, sord, bord)
    nreg = nsx * nsy
    need = L.ipp_sub_fit_workspace_size(nreg, nreg, int(hw), int(fh), len(dg), dg.ctypes.data_as(C.c_void_p),
                                        int(sord), int(bord))
    if need == 0:
        raise ValueError("bad basis description")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    o = dict(coef64=torch.empty(npar, dtype=torch.float64, device=dev),
             coef=torch.empty(npar, dtype=torch.float32, device=dev),
             cx=torch.empty(nreg, dtype=torch.int32, device=dev), cy=torch.empty(nreg, dtype=torch.int32, device=dev),
             n=torch.empty(1, dtype=torch.int32, device=dev), status=torch.empty(1, dtype=torch.int32, device=dev))
    _abi.check("ipp_sub_fit", L.ipp_sub_fit(
        _ptr(img), _ptr(tmpl), W, H, img.stride(0), int(nsx), int(nsy), float(nsig), int(hw), int(fh), len(dg),
        sg.ctypes.data_as(C.c_void_p), dg.ctypes.data_as(C.c_void_p), int(sord), int(bord), _ptr(o["coef64"]),
        _ptr(o["coef"]), _ptr(o["cx"]), _ptr(o["cy"]), _ptr(o["n"]), _ptr(o["status"]), _ptr(ws), ws.numel(),
        _stream()))
    return o


def sub_apply(img, tmpl, coef, hw=10, sig=(0.7, 1.5, 3.0), deg=(6, 4, 2), sord=2, bord=1, out=None, ws=None):
    """Difference image D = I + B - R (x) K of image subtraction (ipp_sub_apply):
    the kernel of each (2 hw + 1)^2 tile from the coefficients `coef` (kernel
    terms c[n, s], then background terms), evaluated at the tile's centre."""
    L = load()
    _frame2d(img, "img")
    _frame2d(tmpl, "tmpl")
    if tmpl.shape != img.shape or tmpl.stride(0) != img.stride(0):
        raise TypeError("img and tmpl must have the same shape and row pitch")
    H, W = img.shape
    sg = np.ascontiguousarray(sig, np.float32)
    dg = np.ascontiguousarray(deg, np.int32)
    need = L.ipp_sub_apply_workspace_size(int(hw), len(dg), dg.ctypes.data_as(C.c_void_p))
    if need == 0:
        raise ValueError("bad basis description")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    nb = sum((int(d) + 1) * (int(d) + 2) // 2 for d in dg)
    nterm = nb * (sord + 1) * (sord + 2) // 2 + ((bord + 1) * (bord + 2) // 2 if bord >= 0 else 0)
    c = torch.as_tensor(np.asarray(coef, np.float32) if not isinstance(coef, torch.Tensor) else coef,
                        dtype=torch.float32, device=img.device).contiguous()
    if c.numel() < nterm:
        raise ValueError(f"coef holds {c.numel()} values, the basis and orders need {nterm}")
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    _frame2d(out, "out")
    _abi.check("ipp_sub_apply", L.ipp_sub_apply(
        _ptr(img), _ptr(tmpl), W, H, img.stride(0), int(hw), len(dg), sg.ctypes.data_as(C.c_void_p),
        dg.ctypes.data_as(C.c_void_p), _ptr(c), int(sord), int(bord), _ptr(out), out.stride(0), _ptr(ws), ws.numel(),
        _stream()))
    return out


def zscale(img, n_samples=1000, contrast=0.25, krej=2.5, max_iter=5):
    """ZScale display limits of the frame (ipp_zscale): device float64 [2]
    (z1, z2) and device int32 [2] (samples used, good samples)."""
    L = load()
    _frame2d(img, "img")
    H, W = img.shape
    z = torch.empty(2, dtype=torch.float64, device=img.device)
    cnt = torch.empty(2, dtype=torch.int32, device=img.device)
    _abi.check("ipp_zscale", L.ipp_zscale(
        _ptr(img), W, H, img.stride(0), C.byref(_abi.ZscaleParams(n_samples, contrast, krej, max_iter)), _ptr(z),
        _ptr(cnt), _stream()))
    return z, cnt


def hist_equalize(img, nbins=4096, out=None, ws=None):
    """Histogram-equalised gray map of the frame (ipp_hist_equalize); returns the
    map and the workspace, which holds the bin counts and the cumulative
    distribution after the call."""
    L = load()
    _frame2d(img, "img")
    H, W = img.shape
    need = L.ipp_hist_equalize_workspace_size(int(nbins))
    if need == 0:
        raise ValueError(f"nbins must be 2..16384, got {nbins}")
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    _frame2d(out, "out")
    _abi.check("ipp_hist_equalize", L.ipp_hist_equalize(
        _ptr(img), W, H, img.stride(0), int(nbins), _ptr(out), out.stride(0), _ptr(ws), ws.numel(), _stream()))
    return out, ws


def _wcs(w):
    """dict(crpix, crval, cd (2 x 2), a, b (6 x 6, a[p][q] of u^p v^q), a_order,
    b_order) -> the ABI struct"""
    s = _abi.Wcs()
    s.crpix[:] = [float(v) for v in w["crpix"]]
    s.crval[:] = [float(v) for v in w["crval"]]
    s.cd[:] = [float(v) for v in np.asarray(w["cd"], np.float64).ravel()]
    for key in ("a", "b"):
        c = np.zeros((6, 6)) if w.get(key) is None else np.asarray(w[key], np.float64)
        getattr(s, key)[:] = [float(v) for v in c.ravel()]
        setattr(s, key + "_order", int(w.get(key + "_order", 0)))
    return s


def wcs_map(src_wcs, tgt_wcs, W, H, step=1, device="cuda"):
    """Target-frame pixel positions (x, y) of the source node grid (multiples of
    `step`) through both frames' WCS (ipp_wcs_map); float64 (ny, nx) each."""
    L = load()
    nx, ny = (W - 1) // step + 1, (H - 1) // step + 1
    xo = torch.empty((ny, nx), dtype=torch.float64, device=device)
    yo = torch.empty_like(xo)
    a, b = _wcs(src_wcs), _wcs(tgt_wcs)
    _abi.check("ipp_wcs_map", L.ipp_wcs_map(C.byref(a), C.byref(b), W, H, int(step), _ptr(xo), _ptr(yo),
                                            _stream()))
    return xo, yo


def affine_fit(xt, yt, x=None, y=None, grid_step=None, ws=None):
    """Partial affine (similarity) least squares of (x, y) -> (xt, yt)
    (ipp_affine_fit).  Without x, y the source points are the node grid of
    wcs_map: xt, yt of shape (ny, nx) and `grid_step`.  Returns the device
    float64 [12] (M, then its inverse, 2 x 3 each) and the device status."""
    L = load()
    _need_cuda(xt, "xt", torch.float64)
    _need_cuda(yt, "yt", torch.float64)
    dev = xt.device
    n = xt.numel()
    gnx = xt.shape[-1] if x is None else 1
    need = L.ipp_affine_fit_workspace_size()
    if ws is None or ws.numel() * ws.element_size() < need:
        ws = torch.empty((need + 7) // 8, dtype=torch.float64, device=dev)
    M = torch.empty(12, dtype=torch.float64, device=dev)
    st = torch.empty(1, dtype=torch.int32, device=dev)
    xc = None if x is None else x.contiguous()
    yc = None if y is None else y.contiguous()
    _abi.check("ipp_affine_fit", L.ipp_affine_fit(
        _ptr(xc), _ptr(yc), _ptr(xt.contiguous()), _ptr(yt.contiguous()), n, gnx, int(grid_step or 1), _ptr(M),
        _ptr(st), _ptr(ws), ws.numel() * ws.element_size(), _stream()))
    return M, st


def reproject_affine(src, Minv, Wo, Ho, fill=0.0, out=None):
    """Bilinear reprojection of `src` onto a Wo x Ho frame: output pixel (j, i)
    samples src at Minv (j, i, 1) (ipp_reproject_affine).  Minv: device float64
    [6] (e.g. affine_fit(...)[0][6:])."""
    L = load()
    _frame2d(src, "src")
    _need_cuda(Minv, "Minv", torch.float64)
    H, W = src.shape
    if out is None:
        out = torch.empty((Ho, Wo), dtype=torch.float32, device=src.device)
    _frame2d(out, "out")
    Mi = Minv.contiguous()
    _abi.check("ipp_reproject_affine", L.ipp_reproject_affine(
        _ptr(src), W, H, src.stride(0), _ptr(Mi), Wo, Ho, float(fill), _ptr(out), out.stride(0), _stream()))
    return out


def align(src, src_wcs, tgt_wcs, Wo, Ho, step=32, fill=0.0, out=None):
    """The alignment function of Sec. 2.2.3 on the GPU: map the source node grid
    into the target frame (wcs_map), estimate the partial affine transform
    (affine_fit) and reproject the source onto the Wo x Ho target grid
    (reproject_affine).  Three device calls, no host synchronisation; returns
    (image, M [12], status)."""
    H, W = src.shape
    xo, yo = wcs_map(src_wcs, tgt_wcs, W, H, step=step, device=src.device)
    M, st = affine_fit(xo, yo, grid_step=step)
    return reproject_affine(src, M[6:], Wo, Ho, fill=fill, out=out), M, st


def stamp_cut(sub, x, y, n_src=None, S=15, max_src=None):
    """S x S stamps around the positions, weights (0 off the frame), origins and
    EDGE flags (ipp_stamp_cut): the input of psf_fit."""
    L = load()
    _need_cuda(sub, "sub", torch.float32)
    H, W = sub.shape
    n = x.numel() if max_src is None else max_src
    if n_src is None:
        n_src = torch.tensor([x.numel()], dtype=torch.int32, device=sub.device)
    dev = sub.device
    m = max(n, 1)
    out = dict(stamps=torch.empty((m, S, S), dtype=torch.float32, device=dev))
    out["weights"] = torch.empty_like(out["stamps"])
    out["origin"] = torch.empty((m, 2), dtype=torch.int32, device=dev)
    out["flags"] = torch.empty(m, dtype=torch.int32, device=dev)
    _abi.check("ipp_stamp_cut", L.ipp_stamp_cut(
        _ptr(sub), W, H, sub.stride(0), _ptr(n_src), n, _ptr(x.contiguous()), _ptr(y.contiguous()), S,
        _ptr(out["stamps"]), _ptr(out["weights"]), _ptr(out["origin"]), _ptr(out["flags"]), _stream()))
    return {k: v[:n] for k, v in out.items()}


def _alloc_catalog(W, H, cfg, max_src, dev):
    """Output tensors of one frame's catalog path and their C view."""
    nx, ny = cfg.grid(W, H)
    f32, i32 = torch.float32, torch.int32
    o = dict(mesh_bkg=torch.empty((ny, nx), dtype=f32, device=dev))
    o["mesh_rms"] = torch.empty_like(o["mesh_bkg"])
    o["sub"] = torch.empty((H, W), dtype=f32, device=dev)
    o["labels"] = torch.empty((H, W), dtype=i32, device=dev)
    o["n_src"] = torch.zeros(1, dtype=i32, device=dev)
    o["status"] = torch.zeros(1, dtype=i32, device=dev)
    for key in ("x", "y", "flux", "sky", "area"):
        o[key] = torch.empty(max_src, dtype=f32, device=dev)
    for key in ("cen_flags", "n_ann", "phot_flags"):
        o[key] = torch.empty(max_src, dtype=i32, device=dev)
    stats = _alloc_stats(max_src, dev)
    c_out = _abi.CatalogOut(
        _ptr(o["mesh_bkg"]), _ptr(o["mesh_rms"]), _ptr(o["sub"]), _ptr(o["labels"]), _ptr(o["n_src"]),
        _stats_c(stats), _ptr(o["x"]), _ptr(o["y"]), _ptr(o["cen_flags"]), _ptr(o["flux"]),
        _ptr(o["sky"]), _ptr(o["area"]), _ptr(o["n_ann"]), _ptr(o["phot_flags"]), _ptr(o["status"]))
    return o, stats, c_out


class Extractor:
    """Preallocated outputs and workspace for repeated ipp_extract calls on
    frames of one shape (the per-frame path without allocations)."""

    def __init__(self, W, H, cfg: BgConfig | None = None, k=1.5, thresh_abs=0.0, min_area=5, fwhm_win=3.0,
                 cen_iter=16, tol2=1e-8, r_ap=5.0, r_in=8.0, r_out=12.0, min_ann=10, max_src=None,
                 device="cuda", filter=0):
        L = load()
        self.L, self.W, self.H = L, W, H
        self.cfg = cfg or BgConfig()
        self.max_src = max_src if max_src is not None else max(4096, (W * H) // 256)
        dev = torch.device(device)
        self.out, self.stats, self.c_out = _alloc_catalog(W, H, self.cfg, self.max_src, dev)
        self.bp = self.cfg.c()
        self.dp = _abi.DetParams(k, thresh_abs, min_area, filter)
        self.cp = _abi.CenParams(fwhm_win, cen_iter, tol2, 0)
        self.pp = _abi.PhotParams(r_ap, r_in, r_out, min_ann)
        need = L.ipp_extract_workspace_size(W, H, self.bp)
        self.ws = torch.empty(need, dtype=torch.uint8, device=dev)

    def __call__(self, img, calib=None, stream=None):
        _need_cuda(img, "img")
        if tuple(img.shape) != (self.H, self.W):
            raise ValueError(f"frame shape {tuple(img.shape)} != {(self.H, self.W)}")
        dtype, cal = _frame(img, calib)
        s = stream.cuda_stream if stream is not None else _stream()
        _abi.check("ipp_extract", self.L.ipp_extract(
            _ptr(img), dtype, self.W, self.H, img.stride(0), cal, self.bp, self.dp, self.cp, self.pp,
            self.max_src, self.c_out, _ptr(self.ws), self.ws.numel(), s))
        return self.out


class Batch:
    """The catalog path over a fixed list of frames of mixed sizes (ipp_batch_*):
    outputs preallocated per frame (self.outs, per-label statistics in
    self.stats).  mode="table": one launch per stage for all frames, from a
    device table of the frames' jobs (ipp_batch_table_*); mode="streams": the
    frames spread over `lanes` CUDA streams.  run() enqueues the batch;
    capture() records it as one CUDA graph that launch() replays (update the
    frames' contents in place between launches)."""

    def __init__(self, frames, lanes=4, cfg: BgConfig | None = None, k=1.5, thresh_abs=0.0, min_area=5,
                 fwhm_win=3.0, cen_iter=16, tol2=1e-8, r_ap=5.0, r_in=8.0, r_out=12.0, min_ann=10,
                 max_src=None, calib=None, mode="streams"):
        if mode not in ("streams", "table"):
            raise ValueError("mode is 'streams' or 'table'")
        self.mode = mode
        L = load()
        self.L = L
        self.cfg = cfg or BgConfig()
        self.frames = list(frames)
        if not self.frames:
            raise ValueError("empty batch")
        dev = self.frames[0].device
        self.outs, self.stats, descs = [], [], []
        self._keep = []
        for img in self.frames:
            _need_cuda(img, "frame")
            H, W = img.shape
            n = max_src if max_src is not None else max(4096, (W * H) // 256)
            o, st, c_out = _alloc_catalog(W, H, self.cfg, n, dev)
            self.stats.append(st)
            dtype, cal = _frame(img, calib)
            cal_p = C.pointer(cal) if cal is not None else None
            self._keep.append((cal, cal_p))
            self.outs.append(o)
            self._nmax = min(getattr(self, "_nmax", n), n)
            descs.append(_abi.FrameDesc(_ptr(img), dtype, 0, W, H, img.stride(0), cal_p, c_out))
        self.max_src = self._nmax
        self.descs = (_abi.FrameDesc * len(descs))(*descs)
        self.n = len(descs)
        self.bp = self.cfg.c()
        self.dp = _abi.DetParams(k, thresh_abs, min_area, 0)
        self.cp = _abi.CenParams(fwhm_win, cen_iter, tol2, 0)
        self.pp = _abi.PhotParams(r_ap, r_in, r_out, min_ann)
        mw = max(f.shape[1] for f in self.frames)
        mh = max(f.shape[0] for f in self.frames)
        if mode == "table":
            need = L.ipp_batch_table_workspace_size(self.descs, self.n, self.bp)
            if need == 0:
                raise ValueError("bad batch for the table form")
        else:
            need = L.ipp_batch_workspace_size(mw, mh, self.bp, _abi.IPP_BATCH_MAX_LANES)
        self.ws = torch.empty(need, dtype=torch.uint8, device=dev)
        self.h = C.c_void_p()
        self.lanes = lanes
        _abi.check("ipp_batch_create", L.ipp_batch_create(lanes, C.byref(self.h)))

    def _args(self):
        return (self.descs, self.n, self.bp, self.dp, self.cp, self.pp, self.max_src, _ptr(self.ws), self.ws.numel())

    def run(self, stream=None):
        s = stream.cuda_stream if stream is not None else _stream()
        if self.mode == "table":
            _abi.check("ipp_batch_table_extract", self.L.ipp_batch_table_extract(self.h, *self._args(), s))
        else:
            _abi.check("ipp_batch_extract", self.L.ipp_batch_extract(self.h, *self._args(), s))
        return self.outs

    def capture(self, stream):
        """Record the batch as a CUDA graph (stream: a torch.cuda.Stream, not the default)."""
        if self.mode == "table":
            _abi.check("ipp_batch_table_capture",
                       self.L.ipp_batch_table_capture(self.h, *self._args(), stream.cuda_stream))
        else:
            _abi.check("ipp_batch_capture", self.L.ipp_batch_capture(self.h, *self._args(), stream.cuda_stream))

    def launch(self, stream=None):
        s = stream.cuda_stream if stream is not None else _stream()
        _abi.check("ipp_batch_launch", self.L.ipp_batch_launch(self.h, s))
        return self.outs

    def autotune(self):
        """Time 1, 2, 4, 8 lanes on this batch (synchronises); returns (best, ms per lane count)."""
        best = C.c_int32(0)
        ms = (C.c_float * 4)()
        _abi.check("ipp_batch_autotune", self.L.ipp_batch_autotune(*self._args(), _stream(), C.byref(best), ms))
        return best.value, list(ms)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.ipp_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_BG_KEYS = ("mesh", "mesh_h", "filter_size", "maxiters", "min_valid", "nsigma", "estimator",
            "median_factor", "mean_factor", "interp")


def extract(img, cfg: BgConfig | None = None, calib=None, **kw):
    """The whole catalog path of one frame (ipp_extract); returns a dict of tensors.
    Background keywords (mesh, filter_size, ...) build the BgConfig; the others
    go to Extractor."""
    H, W = img.shape
    bgkw = {k: kw.pop(k) for k in list(kw) if k in _BG_KEYS}
    if cfg is None:
        cfg = BgConfig(**bgkw)
    ex = Extractor(W, H, cfg, device=img.device, **kw)
    out = dict(ex(img, calib))
    out["stats"] = ex.stats
    return out


def psf_fit(stamps, init=None, weights=None, model=PSF_MOFFAT, beta=2.5, max_iter=50, lambda0=1e-3,
            n_src=None, out=None):
    """Batched Levenberg-Marquardt PSF fit (ipp_psf_fit).  With n_src (an int32
    device tensor) only the first min(n_src, len(stamps)) stamps are fitted and
    the count stays on the device (ipp_psf_fit_dev).  `out` reuses output
    tensors of a previous call."""
    L = load()
    _need_cuda(stamps, "stamps", torch.float32)
    N, S = stamps.shape[0], stamps.shape[-1]
    dev = stamps.device
    if out is None:
        out = dict(params=torch.empty((N, 7), dtype=torch.float32, device=dev),
                   chi2=torch.empty(N, dtype=torch.float32, device=dev),
                   iters=torch.empty(N, dtype=torch.int32, device=dev),
                   flags=torch.empty(N, dtype=torch.int32, device=dev))
    fp = _abi.FitParams(model, beta, max_iter, lambda0)
    w = _ptr(None if weights is None else weights.contiguous())
    ini = _ptr(None if init is None else init.contiguous())
    outs = (_ptr(out["params"]), _ptr(out["chi2"]), _ptr(out["iters"]), _ptr(out["flags"]), _stream())
    if n_src is None:
        _abi.check("ipp_psf_fit", L.ipp_psf_fit(_ptr(stamps.contiguous()), N, S, w, ini, fp, *outs))
    else:
        _need_cuda(n_src, "n_src", torch.int32)
        _abi.check("ipp_psf_fit_dev", L.ipp_psf_fit_dev(_ptr(stamps.contiguous()), _ptr(n_src), N, S, w, ini, fp,
                                                          *outs))
    return out


def _psf_fwd(params, S, model, beta):
    L = load()
    N = params.shape[0]
    m = torch.empty((N, S, S), dtype=torch.float32, device=params.device)
    _abi.check("ipp_psf_model_fwd", L.ipp_psf_model_fwd(
        _ptr(params.contiguous()), N, S, _abi.FitParams(model, beta, 0, 0.0), _ptr(m), _stream()))
    return m


def _psf_adj(params, grad, S, model, beta):
    L = load()
    N = params.shape[0]
    g = torch.empty((N, 7), dtype=torch.float32, device=params.device)
    _abi.check("ipp_psf_model_adj", L.ipp_psf_model_adj(
        _ptr(params.contiguous()), N, S, _abi.FitParams(model, beta, 0, 0.0), _ptr(grad.contiguous()),
        _ptr(g), _stream()))
    return g


class PSFModel(torch.autograd.Function):
    """Differentiable PSF images m[N, S, S] of params[N, 7]: forward and the
    hand-written adjoint (vector-Jacobian product) are CUDA kernels."""

    @staticmethod
    def forward(ctx, params, S=15, model=PSF_MOFFAT, beta=2.5):
        params = params.detach().to(torch.float32).contiguous()
        ctx.save_for_backward(params)
        ctx.cfg = (S, model, beta)
        return _psf_fwd(params, S, model, beta)

    @staticmethod
    def backward(ctx, grad):
        (params,) = ctx.saved_tensors
        S, model, beta = ctx.cfg
        return _psf_adj(params, grad.to(torch.float32), S, model, beta), None, None, None


def psf_model(params, S=15, model=PSF_MOFFAT, beta=2.5):
    return PSFModel.apply(params, S, model, beta)
