"""FP64 CPU oracle of the catalog path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and it
shares no code with the CUDA library.  The arithmetic lives in ``ipp_oracle.c``
(plain C, FP64, one function per step of the paper); this module only builds
it with gcc and marshals numpy arrays.

Parity status per function is recorded at the top of ``ipp_oracle.c`` and in
the design notes: every function here is pinned by a ``-m "not gpu"`` test.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ipp_oracle.c")
_HDR = os.path.join(_HERE, "ipp_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_EDGE = 1
FLAG_WIN_NOT_CONVERGED = 2
FLAG_ANN_FEW = 4
FLAG_FIT_MAXITER = 8
FLAG_FIT_SINGULAR = 16
FLAG_FIT_BAD_SIGMA = 32
FLAG_KRON_BAD = 64

EST_SIGMA, EST_MEDIAN, EST_MEAN, EST_FACTORS = 0, 1, 2, 3
PSF_MOFFAT, PSF_GAUSS = 0, 1


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile liboracle.so with gcc (no fused multiply-add).  openmp=True
    builds liboracle_omp.so from the same source with -fopenmp: independent
    meshes, pixel rows, sources and stamps spread over threads, CCL serial, the
    arithmetic of each item unchanged (the all-cores CPU timing)."""
    lib_path = _LIB_OMP if openmp else _LIB
    stale = (not os.path.exists(lib_path)) or any(
        os.path.getmtime(f) > os.path.getmtime(lib_path) for f in (_SRC, _HDR))
    if force or stale:
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
               *(["-fopenmp"] if openmp else []), _SRC, "-o", lib_path + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(lib_path + ".tmp", lib_path)
    return lib_path


def use_openmp(threads: int) -> None:
    """Switch this process to the OpenMP build on `threads` threads (call before
    the first oracle function; for the CPU timing only)."""
    global _lib, _LIB
    os.environ["OMP_NUM_THREADS"] = str(int(threads))
    build(openmp=True)
    with _lock:
        _lib = None
        _LIB = _LIB_OMP


class Wcs(C.Structure):
    _fields_ = [("crpix", C.c_double * 2), ("crval", C.c_double * 2), ("cd", C.c_double * 4),
                ("a_order", C.c_int32), ("b_order", C.c_int32),
                ("a", C.c_double * 36), ("b", C.c_double * 36)]


def _wcs(w):
    """dict(crpix, crval, cd (2x2), a, b (6x6 arrays, a[p][q] of u^p v^q), a_order,
    b_order) -> the oracle's struct"""
    s = Wcs()
    s.crpix[:] = [float(v) for v in w["crpix"]]
    s.crval[:] = [float(v) for v in w["crval"]]
    s.cd[:] = [float(v) for v in np.asarray(w["cd"], np.float64).ravel()]
    for key in ("a", "b"):
        c = np.zeros((6, 6)) if w.get(key) is None else np.asarray(w[key], np.float64)
        getattr(s, key)[:] = [float(v) for v in c.ravel()]
        setattr(s, key + "_order", int(w.get(key + "_order", 0)))
    return s


class BgParams(C.Structure):
    _fields_ = [("mesh_w", C.c_int32), ("mesh_h", C.c_int32),
                ("filter_w", C.c_int32), ("filter_h", C.c_int32),
                ("maxiters", C.c_int32), ("min_valid", C.c_int32),
                ("estimator", C.c_int32), ("pad_", C.c_int32),
                ("nsigma", C.c_double), ("median_factor", C.c_double),
                ("mean_factor", C.c_double)]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build(openmp=_LIB == _LIB_OMP)
            L = C.CDLL(_LIB)
            vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            L.orc_calibrate.argtypes = [vp, i64, i64, i64, vp, d, vp, vp]
            L.orc_mesh_stats.argtypes = [vp, i64, i64, i64, vp, C.POINTER(BgParams), vp, vp, vp, vp, vp]
            L.orc_mesh_fill_filter.argtypes = [vp, vp, vp, i64, i64, i32, i32, vp, vp]
            L.orc_keys_weight.argtypes = [d]
            L.orc_keys_weight.restype = d
            L.orc_interp_map.argtypes = [vp, i64, i64, i32, i32, i64, i64, vp]
            L.orc_spline_map.argtypes = [vp, i64, i64, i32, i32, i64, i64, vp]
            L.orc_spline_nodes.argtypes = [vp, i64, i64, vp, vp, vp]
            L.orc_bg_subtract.argtypes = [vp, i64, i64, i64, vp, i64, i64, i32, i32, vp, vp]
            L.orc_threshold.argtypes = [vp, i64, i64, vp, i64, i64, i32, i32, d, d, vp]
            L.orc_threshold_filtered.argtypes = [vp, i64, i64, vp, i64, i64, i32, i32, d, d, vp]
            L.orc_label.argtypes = [vp, vp, i64, i64, i32, vp, i64] + [vp] * 10
            L.orc_label.restype = i64
            L.orc_centroid.argtypes = [vp, i64, i64, i64, vp, vp, d, i32, d, vp, vp, vp, vp]
            L.orc_overlap.argtypes = [d] * 7
            L.orc_overlap.restype = d
            L.orc_aperture.argtypes = [vp, i64, i64, i64, vp, vp, d, d, d, i32, vp, vp, vp, vp, vp]
            L.orc_stamp_cut.argtypes = [vp, i64, i64, i64, vp, vp, i32, vp, vp, vp, vp]
            L.orc_auto_phot.argtypes = [vp, vp, i64, i64, i64] + [vp] * 6 + [d, d, d] + [vp] * 7
            L.orc_deblend.argtypes = [vp, vp, i64, i64, i64, i32, d, vp]
            L.orc_gray_transform.argtypes = [vp, i64, i64, i32, d, d, d, vp]
            L.orc_hist_equalize.argtypes = [vp, i64, i64, i32, vp]
            L.orc_wcs_pix2world.argtypes = [C.POINTER(Wcs), vp, vp, i64, vp, vp]
            L.orc_wcs_world2pix.argtypes = [C.POINTER(Wcs), vp, vp, i64, vp, vp]
            L.orc_wcs_map.argtypes = [C.POINTER(Wcs), C.POINTER(Wcs), i64, i64, i32, vp, vp]
            L.orc_affine_fit.argtypes = [vp, vp, vp, vp, i64, vp, vp]
            L.orc_reproject_affine.argtypes = [vp, i64, i64, vp, i64, i64, d, vp]
            L.orc_zscale.argtypes = [vp, i64, i64, i32, d, d, i32, vp, vp]
            L.orc_chol_solve.argtypes = [vp, vp, i32]
            L.orc_clean.argtypes = [vp, vp, i64, i64, i64, vp, d, vp]
            L.orc_clean.restype = i64
            L.orc_clean_stats.argtypes = [vp, vp, i64, i64, i64] + [vp] * 7
            L.orc_sub_basis.argtypes = [i32, vp, vp, i32, vp]
            L.orc_sub_stamps.argtypes = [vp, vp, i64, i64, i32, i32, i32, i32, d, vp, vp]
            L.orc_sub_fit.argtypes = [vp, vp, i64, i64, vp, vp, i32, i32, i32, vp, vp, i32, i32, i32, vp]
            L.orc_sub_normal.argtypes = [vp, vp, i64, i64, vp, vp, i32, i32, i32, vp, vp, i32, i32, i32, vp, vp]
            L.orc_sub_apply.argtypes = [vp, vp, i64, i64, i32, vp, vp, i32, i32, i32, vp, i32, vp]
            L.orc_deblend.restype = i64
            L.orc_psf_model.argtypes = [vp, i32, i32, d, vp, vp]
            L.orc_psf_fit.argtypes = [vp, i64, i32, vp, vp, i32, d, i32, d, vp, vp, vp, vp]
            L.orc_psf_init.argtypes = [vp, i32, vp]
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ------------------------------------------------------------------ c0
def calibrate(raw, flat, bias=500.0, bias_map=None):
    raw = np.ascontiguousarray(raw, dtype=np.uint16)
    H, W = raw.shape
    out = np.empty((H, W), np.float32)
    bm = None if bias_map is None else _f32(bias_map)
    rc = lib().orc_calibrate(_p(raw), W, H, W, _p(bm), float(bias), _p(_f32(flat)), _p(out))
    assert rc == 0
    return out


# ------------------------------------------------------------- c1-c3
def bg_params(mesh=64, mesh_h=None, filter_size=3, maxiters=10, min_valid=100,
              nsigma=3.0, estimator=EST_SIGMA, median_factor=2.5, mean_factor=1.5):
    return BgParams(mesh, mesh_h or mesh, filter_size, filter_size, maxiters, min_valid,
                    estimator, 0, nsigma, median_factor, mean_factor)


def mesh_stats(img, mask=None, **kw):
    img = _f32(img)
    H, W = img.shape
    p = bg_params(**kw)
    nx, ny = -(-W // p.mesh_w), -(-H // p.mesh_h)
    rb, rr = np.zeros((ny, nx)), np.zeros((ny, nx))
    valid, niter = np.zeros((ny, nx), np.int32), np.zeros((ny, nx), np.int32)
    margin = np.zeros((ny, nx))
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    rc = lib().orc_mesh_stats(_p(img), W, H, W, _p(m), C.byref(p), _p(rb), _p(rr),
                              _p(valid), _p(niter), _p(margin))
    assert rc == 0
    return dict(raw_bkg=rb, raw_rms=rr, valid=valid, niter=niter, margin=margin)


def fill_filter(raw_bkg, raw_rms, valid, filter_size=3):
    ny, nx = raw_bkg.shape
    b, r = np.zeros((ny, nx)), np.zeros((ny, nx))
    rc = lib().orc_mesh_fill_filter(_p(np.ascontiguousarray(raw_bkg, np.float64)),
                                    _p(np.ascontiguousarray(raw_rms, np.float64)),
                                    _p(np.ascontiguousarray(valid, np.int32)),
                                    nx, ny, filter_size, filter_size, _p(b), _p(r))
    if rc != 0:
        raise ValueError("no valid mesh")
    return b, r


def bg_estimate(img, mask=None, **kw):
    """Sec. 2.2.2 mesh background: returns filtered (bkg, rms) as float32 grids
    and the unfiltered statistics."""
    st = mesh_stats(img, mask, **kw)
    fs = kw.get("filter_size", 3)
    b, r = fill_filter(st["raw_bkg"], st["raw_rms"], st["valid"], fs)
    return b.astype(np.float32), r.astype(np.float32), st


def spline_map(mesh, mesh_w, W, H, mesh_h=None):
    """natural-spline background map of the node grid (W x H, FP64)"""
    mesh = _f32(mesh)
    ny, nx = mesh.shape
    out = np.zeros((H, W))
    assert lib().orc_spline_map(_p(mesh), nx, ny, mesh_w, mesh_h or mesh_w, W, H, _p(out)) == 0
    return out


def spline_nodes(mesh):
    """second derivatives of the natural tensor spline at the nodes: Mx, My, Mxy"""
    mesh = _f32(mesh)
    ny, nx = mesh.shape
    Mx, My, Mxy = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    assert lib().orc_spline_nodes(_p(mesh), nx, ny, _p(Mx), _p(My), _p(Mxy)) == 0
    return Mx, My, Mxy


def keys_weight(s):
    return lib().orc_keys_weight(float(s))


def interp_map(mesh, mesh_w, W, H, mesh_h=None):
    mesh = _f32(mesh)
    ny, nx = mesh.shape
    out = np.zeros((H, W))
    rc = lib().orc_interp_map(_p(mesh), nx, ny, mesh_w, mesh_h or mesh_w, W, H, _p(out))
    assert rc == 0
    return out


def bg_subtract(img, mesh_bkg, mesh_w, mesh_h=None):
    img, mesh_bkg = _f32(img), _f32(mesh_bkg)
    H, W = img.shape
    ny, nx = mesh_bkg.shape
    sub, bmap = np.empty((H, W), np.float32), np.empty((H, W), np.float32)
    rc = lib().orc_bg_subtract(_p(img), W, H, W, _p(mesh_bkg), nx, ny, mesh_w,
                               mesh_h or mesh_w, _p(sub), _p(bmap))
    assert rc == 0
    return sub, bmap


def threshold(sub, mesh_rms, mesh_w, k=1.5, thresh_abs=0.0, mesh_h=None, filtered=False):
    sub, mesh_rms = _f32(sub), _f32(mesh_rms)
    H, W = sub.shape
    ny, nx = mesh_rms.shape
    m = np.zeros((H, W), np.uint8)
    fn = lib().orc_threshold_filtered if filtered else lib().orc_threshold
    rc = fn(_p(sub), W, H, _p(mesh_rms), nx, ny, mesh_w, mesh_h or mesh_w, float(k), float(thresh_abs), _p(m))
    assert rc == 0
    return m


# ------------------------------------------------------------- c6-c7
def label(mask, sub, min_area=5, max_src=None):
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    sub = _f32(sub)
    H, W = mask.shape
    labels = np.zeros((H, W), np.int32)
    cap = max_src if max_src is not None else max(1, (H * W) // max(1, min_area) + 1)
    cap = int(min(cap, H * W + 1))
    st = dict(area=np.zeros(cap, np.int32), first=np.zeros(cap, np.int64),
              xmin=np.zeros(cap, np.int32), xmax=np.zeros(cap, np.int32),
              ymin=np.zeros(cap, np.int32), ymax=np.zeros(cap, np.int32),
              peak=np.zeros(cap), sum=np.zeros(cap), xbar=np.zeros(cap), ybar=np.zeros(cap))
    order = ["area", "first", "xmin", "xmax", "ymin", "ymax", "peak", "sum", "xbar", "ybar"]
    K = lib().orc_label(_p(mask), _p(sub), W, H, min_area, _p(labels), cap,
                        *[_p(st[k]) for k in order])
    n = min(K, cap)
    return labels, int(K), {k: v[:n] for k, v in st.items()}


# ---------------------------------------------------------------- c8
def centroid(sub, x0, y0, fwhm_win=3.0, max_iter=16, tol2=1e-8):
    sub = _f32(sub)
    H, W = sub.shape
    x0, y0 = _f32(x0), _f32(y0)
    n = len(x0)
    x, y = np.zeros(n), np.zeros(n)
    it, fl = np.zeros(n, np.int32), np.zeros(n, np.int32)
    lib().orc_centroid(_p(sub), W, H, n, _p(x0), _p(y0), float(fwhm_win), int(max_iter),
                       float(tol2), _p(x), _p(y), _p(it), _p(fl))
    return x, y, it, fl


# --------------------------------------------------------------- c9-c11
def overlap(cx, cy, r, x0, x1, y0, y1):
    return lib().orc_overlap(float(cx), float(cy), float(r), float(x0), float(x1),
                             float(y0), float(y1))


def aperture(sub, x, y, r_ap=5.0, r_in=8.0, r_out=12.0, min_ann=10):
    sub = _f32(sub)
    H, W = sub.shape
    x, y = _f32(x), _f32(y)
    n = len(x)
    out = dict(flux=np.zeros(n), sky=np.zeros(n), area=np.zeros(n),
               n_ann=np.zeros(n, np.int32), flags=np.zeros(n, np.int32))
    lib().orc_aperture(_p(sub), W, H, n, _p(x), _p(y), float(r_ap), float(r_in), float(r_out),
                       int(min_ann), _p(out["flux"]), _p(out["sky"]), _p(out["area"]),
                       _p(out["n_ann"]), _p(out["flags"]))
    return out


GRAY_LINEAR, GRAY_LOG, GRAY_POWER, GRAY_EXP = 0, 1, 2, 3


def gray_transform(img, kind, lo, hi, a=1000.0):
    img = _f32(img)
    H, W = img.shape
    out = np.zeros((H, W))
    assert lib().orc_gray_transform(_p(img), W, H, int(kind), float(lo), float(hi), float(a), _p(out)) == 0
    return out


def hist_equalize(img, nbins=4096):
    img = _f32(img)
    H, W = img.shape
    out = np.zeros((H, W))
    assert lib().orc_hist_equalize(_p(img), W, H, int(nbins), _p(out)) == 0
    return out


def deblend(sub, labels, K, nthresh=32, mincont=0.005):
    """Deblended label map (objects numbered in raster order) and its count."""
    sub = _f32(sub)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    H, W = sub.shape
    out = np.zeros((H, W), np.int32)
    n = lib().orc_deblend(_p(sub), _p(labels), W, H, int(K), int(nthresh), float(mincont), _p(out))
    assert n >= 0
    return out, int(n)


def auto_phot(sub, labels, stats, k_kron=2.5, r_min=3.5, r_kmax=6.0):
    """Auto (Kron) photometry of the labelled sources; `stats` holds xmin, xmax,
    ymin, ymax (int) and xbar, ybar (cast to float32, the precision the
    library's statistics carry)."""
    sub = _f32(sub)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    H, W = sub.shape
    n = len(stats["xbar"])
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    xb, yb = _f32(stats["xbar"]), _f32(stats["ybar"])
    bb = [i32(stats[k]) for k in ("xmin", "xmax", "ymin", "ymax")]
    out = dict(flux=np.zeros(n), area=np.zeros(n), kron=np.zeros(n), x2=np.zeros(n),
               y2=np.zeros(n), xy=np.zeros(n), flags=np.zeros(n, np.int32))
    lib().orc_auto_phot(_p(sub), _p(labels), W, H, n, *[_p(b) for b in bb], _p(xb), _p(yb),
                        float(k_kron), float(r_min), float(r_kmax), _p(out["flux"]),
                        _p(out["area"]), _p(out["kron"]), _p(out["x2"]), _p(out["y2"]),
                        _p(out["xy"]), _p(out["flags"]))
    return out


def stamp_cut(sub, x, y, S=15):
    sub = _f32(sub)
    H, W = sub.shape
    x, y = _f32(x), _f32(y)
    n = len(x)
    out = dict(stamps=np.zeros((n, S, S), np.float32), weights=np.zeros((n, S, S), np.float32),
               origin=np.zeros((n, 2), np.int32), flags=np.zeros(n, np.int32))
    rc = lib().orc_stamp_cut(_p(sub), W, H, n, _p(x), _p(y), int(S), _p(out["stamps"]), _p(out["weights"]),
                             _p(out["origin"]), _p(out["flags"]))
    if rc:
        raise ValueError(f"orc_stamp_cut: status {rc}")
    return out


# -------------------------------------------------------------- c12-c13
def psf_model(p7, S=15, model=PSF_MOFFAT, beta=2.5, jac=True):
    p7 = np.ascontiguousarray(p7, dtype=np.float64)
    m = np.zeros(S * S)
    J = np.zeros((S * S, 7)) if jac else None
    lib().orc_psf_model(_p(p7), S, model, float(beta), _p(m), _p(J))
    return (m.reshape(S, S), J) if jac else m.reshape(S, S)


def psf_init(stamp):
    st = _f32(stamp)
    S = st.shape[-1]
    p = np.zeros(7)
    lib().orc_psf_init(_p(st), S, _p(p))
    return p


def psf_fit(stamps, init=None, weights=None, model=PSF_MOFFAT, beta=2.5, max_iter=50,
            lambda0=1e-3):
    stamps = _f32(stamps)
    N, S = stamps.shape[0], stamps.shape[-1]
    ini = None if init is None else _f32(init)
    w = None if weights is None else _f32(weights)
    out = dict(params=np.zeros((N, 7)), chi2=np.zeros(N), iters=np.zeros(N, np.int32),
               flags=np.zeros(N, np.int32))
    lib().orc_psf_fit(_p(stamps), N, S, _p(w), _p(ini), model, float(beta), int(max_iter),
                      float(lambda0), _p(out["params"]), _p(out["chi2"]), _p(out["iters"]),
                      _p(out["flags"]))
    return out


# ----------------------------------------------------------- whole path
def catalog(img, mesh=64, filter_size=3, k=1.5, min_area=5, fwhm_win=3.0,
            r_ap=5.0, r_in=8.0, r_out=12.0, mask_in=None, interp="keys"):
    """The whole per-frame path a1..a6 on one float32 frame.  interp="spline"
    takes the natural-spline map (spline_map) for the background and for the
    rms of the threshold: sub = float32(img - B), detected where
    sub > k rms(x, y) -- the same definitions, the other interpolant."""
    bkg, rms, st = bg_estimate(img, mesh=mesh, filter_size=filter_size)
    if interp == "spline":
        H, W = img.shape
        B = spline_map(bkg, mesh, W, H)
        sub = (_f32(img).astype(np.float64) - B).astype(np.float32)
        R = spline_map(rms, mesh, W, H)
        m = (sub.astype(np.float64) > k * R).astype(np.uint8) if mask_in is None else mask_in
    else:
        sub, _ = bg_subtract(img, bkg, mesh)
        m = threshold(sub, rms, mesh, k) if mask_in is None else mask_in
    labels, K, stats = label(m, sub, min_area)
    x, y, it, cfl = centroid(sub, stats["xbar"].astype(np.float32),
                             stats["ybar"].astype(np.float32), fwhm_win)
    ph = aperture(sub, x.astype(np.float32), y.astype(np.float32), r_ap, r_in, r_out)
    return dict(bkg=bkg, rms=rms, mesh_stats=st, sub=sub, mask=m, labels=labels, K=K,
                stats=stats, x=x, y=y, cen_iter=it, cen_flags=cfl, interp=interp, **ph)


def wcs_pix2world(w, x, y):
    """0-based pixel positions -> (RA, Dec) in degrees (Eqs. 5-7)."""
    x = np.ascontiguousarray(x, np.float64).ravel()
    y = np.ascontiguousarray(y, np.float64).ravel()
    ra, de = np.zeros_like(x), np.zeros_like(x)
    s = _wcs(w)
    assert lib().orc_wcs_pix2world(C.byref(s), _p(x), _p(y), x.size, _p(ra), _p(de)) == 0
    return ra, de


def wcs_world2pix(w, ra, dec):
    """(RA, Dec) in degrees -> 0-based pixel positions (inverse chain)."""
    ra = np.ascontiguousarray(ra, np.float64).ravel()
    de = np.ascontiguousarray(dec, np.float64).ravel()
    x, y = np.zeros_like(ra), np.zeros_like(ra)
    s = _wcs(w)
    assert lib().orc_wcs_world2pix(C.byref(s), _p(ra), _p(de), ra.size, _p(x), _p(y)) == 0
    return x, y


def wcs_map(src, tgt, W, H, step=1):
    """target-frame positions of the source node grid (multiples of step)."""
    nx, ny = (W - 1) // step + 1, (H - 1) // step + 1
    xo, yo = np.zeros((ny, nx)), np.zeros((ny, nx))
    a, b = _wcs(src), _wcs(tgt)
    assert lib().orc_wcs_map(C.byref(a), C.byref(b), W, H, int(step), _p(xo), _p(yo)) == 0
    return xo, yo


def affine_fit(x, y, xt, yt):
    """partial affine least squares (x, y) -> (xt, yt): (M, Minv), 2x3 each."""
    x, y, xt, yt = (np.ascontiguousarray(v, np.float64).ravel() for v in (x, y, xt, yt))
    M, Mi = np.zeros(6), np.zeros(6)
    e = lib().orc_affine_fit(_p(x), _p(y), _p(xt), _p(yt), x.size, _p(M), _p(Mi))
    if e:
        raise ValueError("affine fit needs two distinct finite points")
    return M.reshape(2, 3), Mi.reshape(2, 3)


def reproject_affine(src, Minv, Wo, Ho, fill=0.0):
    """bilinear reprojection of src onto a Wo x Ho frame through Minv (output
    pixel -> source position)."""
    src = _f32(src)
    H, W = src.shape
    Mi = np.ascontiguousarray(Minv, np.float64).ravel()
    out = np.zeros((Ho, Wo))
    assert lib().orc_reproject_affine(_p(src), W, H, _p(Mi), Wo, Ho, float(fill), _p(out)) == 0
    return out


def zscale(img, n_samples=1000, contrast=0.25, krej=2.5, max_iter=5):
    """ZScale limits (z1, z2) and (samples, good samples)."""
    img = _f32(img)
    H, W = img.shape
    z, cnt = np.zeros(2), np.zeros(2, np.int32)
    e = lib().orc_zscale(_p(img), W, H, int(n_samples), float(contrast), float(krej), int(max_iter), _p(z),
                         _p(cnt))
    if e:
        raise ValueError("zscale: no finite sample or bad parameters")
    return float(z[0]), float(z[1]), (int(cnt[0]), int(cnt[1]))


# ---- image subtraction (Sec. 2.2.4) ------------------------------------------------
SUB_SIG = (0.7, 1.5, 3.0)   # Gaussian widths of the basis (a reading: HOTPANTS' usual set)
SUB_DEG = (6, 4, 2)         # their polynomial degrees


def _basis_args(sig, deg):
    sg = np.ascontiguousarray(sig, np.float64)
    dg = np.ascontiguousarray(deg, np.int32)
    return sg, dg


def sub_basis(hw=10, sig=SUB_SIG, deg=SUB_DEG):
    """the basis kernels K_n (Eq. 9): (nb, 2 hw + 1, 2 hw + 1), rows v, columns u"""
    sg, dg = _basis_args(sig, deg)
    nb = int(sum((k + 1) * (k + 2) // 2 for k in deg))
    S = 2 * hw + 1
    out = np.zeros((nb, S, S))
    assert lib().orc_sub_basis(hw, _p(sg), _p(dg), len(sg), _p(out)) == nb
    return out


def sub_stamps(img, tmpl, nsx=10, nsy=10, hw=10, fh=10, nsig=5.0):
    """candidate stamp centres (x, y): one per region at most"""
    img, tmpl = _f32(img), _f32(tmpl)
    H, W = img.shape
    cx = np.zeros(nsx * nsy, np.int32)
    cy = np.zeros(nsx * nsy, np.int32)
    n = lib().orc_sub_stamps(_p(img), _p(tmpl), W, H, nsx, nsy, hw, fh, float(nsig), _p(cx), _p(cy))
    assert n >= 0
    return cx[:n].copy(), cy[:n].copy()


def sub_fit(img, tmpl, cx, cy, hw=10, fh=10, sig=SUB_SIG, deg=SUB_DEG, sord=2, bord=1):
    """kernel coefficients c[n, s] (n basis, s spatial term) and background d[b]"""
    img, tmpl = _f32(img), _f32(tmpl)
    H, W = img.shape
    sg, dg = _basis_args(sig, deg)
    cx = np.ascontiguousarray(cx, np.int32)
    cy = np.ascontiguousarray(cy, np.int32)
    nb = int(sum((k + 1) * (k + 2) // 2 for k in deg))
    ns = (sord + 1) * (sord + 2) // 2
    ng = (bord + 1) * (bord + 2) // 2 if bord >= 0 else 0
    coef = np.zeros(nb * ns + ng)
    e = lib().orc_sub_fit(_p(img), _p(tmpl), W, H, _p(cx), _p(cy), len(cx), hw, fh, _p(sg), _p(dg), len(sg), sord,
                          bord, _p(coef))
    if e:
        raise ValueError("subtraction fit: no candidate or a singular normal matrix")
    return coef


def sub_normal(img, tmpl, cx, cy, hw=10, fh=10, sig=SUB_SIG, deg=SUB_DEG, sord=2, bord=1):
    """normal equations (AtA, Atb) of the fit, unknowns ordered as sub_fit's"""
    img, tmpl = _f32(img), _f32(tmpl)
    H, W = img.shape
    sg, dg = _basis_args(sig, deg)
    cx = np.ascontiguousarray(cx, np.int32)
    cy = np.ascontiguousarray(cy, np.int32)
    nb = int(sum((k + 1) * (k + 2) // 2 for k in deg))
    npar = nb * (sord + 1) * (sord + 2) // 2 + ((bord + 1) * (bord + 2) // 2 if bord >= 0 else 0)
    AtA, Atb = np.zeros((npar, npar)), np.zeros(npar)
    e = lib().orc_sub_normal(_p(img), _p(tmpl), W, H, _p(cx), _p(cy), len(cx), hw, fh, _p(sg), _p(dg), len(sg),
                             sord, bord, _p(AtA), _p(Atb))
    if e:
        raise ValueError("subtraction normal equations: bad arguments")
    return AtA, Atb


def sub_apply(img, tmpl, coef, hw=10, sig=SUB_SIG, deg=SUB_DEG, sord=2, bord=1, tile=21):
    """difference image D = I + B - R (x) K (Eq. 10), NaN where the kernel
    support leaves the frame"""
    img, tmpl = _f32(img), _f32(tmpl)
    H, W = img.shape
    sg, dg = _basis_args(sig, deg)
    c = np.ascontiguousarray(coef, np.float64)
    D = np.zeros((H, W))
    assert lib().orc_sub_apply(_p(img), _p(tmpl), W, H, hw, _p(sg), _p(dg), len(sg), sord, bord, _p(c), int(tile),
                               _p(D)) == 0
    return D


def clean(sub, labels, nobj, thr, beta=1.0):
    """cleaned label map and object count (SExtractor-style cleaning)"""
    sub = _f32(sub)
    labels = np.ascontiguousarray(labels, np.int32)
    H, W = sub.shape
    thr = np.ascontiguousarray(np.broadcast_to(np.asarray(thr, np.float32), (H, W)))
    out = np.zeros((H, W), np.int32)
    k = lib().orc_clean(_p(sub), _p(labels), W, H, int(nobj), _p(thr), float(beta), _p(out))
    assert k >= 0
    return out, int(k)


def clean_stats(sub, labels, nobj):
    """per-object peak, peak index, barycentre and moments of the cleaning test
    (arrays indexed by label, entry 0 unused)"""
    sub = _f32(sub)
    labels = np.ascontiguousarray(labels, np.int32)
    H, W = sub.shape
    n = int(nobj) + 1
    out = {k: np.zeros(n) for k in ("peak", "cx", "cy", "x2", "y2", "xy")}
    pidx = np.zeros(n, np.int64)
    assert lib().orc_clean_stats(_p(sub), _p(labels), W, H, int(nobj), _p(out["peak"]), _p(pidx), _p(out["cx"]),
                                 _p(out["cy"]), _p(out["x2"]), _p(out["y2"]), _p(out["xy"])) == 0
    out["peak_index"] = pidx
    return out


def chol_solve(A, b):
    """x with A x = b by the oracle's Cholesky (A symmetric positive definite);
    ValueError when a pivot is not positive"""
    A = np.array(A, np.float64, order="C", copy=True)
    x = np.array(b, np.float64, copy=True)
    if lib().orc_chol_solve(_p(A), _p(x), int(x.size)):
        raise ValueError("not positive definite")
    return x
