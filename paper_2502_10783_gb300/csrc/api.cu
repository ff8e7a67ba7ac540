// api.cu -- the C ABI of libipp: argument validation, workspace layout and the
// launch sequences of each call.  All calls are asynchronous on `stream`.
#include <stdarg.h>
#include <mutex>
#include <cmath>
#include <stdio.h>
#include <string.h>

#include "checks.cuh"

using namespace ipp;

// ---- error reporting --------------------------------------------------------
static thread_local char g_detail[512] = "";

int ipp_set_error(int status, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
    return status;
}

int ipp_check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return IPP_OK;
}

static std::mutex g_once_lock;
static uint16_t g_once_done[64];  // bit `slot` of entry `device`

int ipp_once_per_device_impl(int slot, cudaError_t (*fn)(void*), void* arg) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64 || slot < 0 || slot >= 16)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "device %d / slot %d out of range", dev, slot);
    std::lock_guard<std::mutex> guard(g_once_lock);
    if ((g_once_done[dev] >> slot) & 1) return IPP_OK;
    e = fn(arg);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "per-device set-up: %s", cudaGetErrorString(e));
    g_once_done[dev] |= (uint16_t)(1u << slot);
    return IPP_OK;
}

extern "C" const char* ipp_status_string(int status) {
    switch (status) {
        case IPP_OK: return "ok";
        case IPP_ERR_INVALID_ARG: return "invalid argument";
        case IPP_ERR_CUDA: return "CUDA error";
        case IPP_ERR_CAPACITY: return "capacity exceeded";
        case IPP_ERR_NO_VALID_MESH: return "no valid mesh";
        case IPP_ERR_TIMEOUT: return "device wait timed out";
        case IPP_ERR_NOT_SUPPORTED: return "not supported";
        case IPP_ERR_DEGENERATE: return "too few usable points";
        default: return "unknown status";
    }
}

extern "C" const char* ipp_last_error_detail(void) { return g_detail; }

extern "C" int ipp_version(int* major, int* minor, int* patch) {
    if (!major || !minor || !patch) return IPP_ERR_INVALID_ARG;
    *major = 0; *minor = 1; *patch = 0;
    return IPP_OK;
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static void grid_of(int64_t W, int64_t H, const ipp_bg_params* p, int* nx, int* ny) {
    *nx = (int)cdiv(W, p->mesh_w);
    *ny = (int)cdiv(H, p->mesh_h);
}

// ---- background ---------------------------------------------------------------
extern "C" size_t ipp_bg_estimate_workspace_size(int64_t W, int64_t H, const ipp_bg_params* p) {
    if (!p || p->mesh_w < 1 || p->mesh_h < 1 || W <= 0 || H <= 0) return 0;
    int nx, ny;
    grid_of(W, H, p, &nx, &ny);
    return 4 * a256((size_t)nx * ny * sizeof(float));
}

static int bg_estimate_impl(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                            const uint8_t* mask, const ipp_calib* cal, const ipp_bg_params* p,
                            float* mesh_bkg, float* mesh_rms, float* raw_bkg, float* raw_rms,
                            int32_t* status_dev, void* ws, size_t ws_bytes, cudaStream_t s) {
    int nx, ny;
    grid_of(W, H, p, &nx, &ny);
    size_t nb = a256((size_t)nx * ny * sizeof(float));
    unsigned char* w = (unsigned char*)ws;
    float* rb = raw_bkg ? raw_bkg : (float*)(w + 0 * nb);
    float* rr = raw_rms ? raw_rms : (float*)(w + 1 * nb);
    float* fb = (float*)(w + 2 * nb);
    float* fr = (float*)(w + 3 * nb);
    MeshJob J;
    J.img = img; J.dtype = dtype; J.W = W; J.H = H; J.pitch = pitch; J.mask = mask;
    J.bias_map = cal ? cal->bias_map : nullptr; J.bias = cal ? cal->bias : 0.f;
    J.inv_flat = cal ? cal->inv_flat : nullptr;
    J.mesh_w = p->mesh_w; J.mesh_h = p->mesh_h; J.nx = nx; J.ny = ny;
    J.maxiters = p->maxiters; J.min_valid = p->min_valid; J.estimator = p->estimator;
    J.nsigma = p->nsigma; J.mf = p->median_factor; J.mnf = p->mean_factor;
    J.raw_bkg = rb; J.raw_rms = rr;
    if (int e = ipp_launch_mesh_stats(J, s)) return e;
    return ipp_launch_mesh_filter(rb, rr, fb, fr, nx, ny, p->filter_w, p->filter_h, mesh_bkg, mesh_rms,
                                  status_dev, s);
}

extern "C" int ipp_bg_estimate(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                               const uint8_t* mask, const ipp_calib* cal, const ipp_bg_params* p,
                               float* mesh_bkg, float* mesh_rms, float* raw_bkg, float* raw_rms,
                               int32_t* status_dev, void* ws, size_t ws_bytes, void* stream) {
    if (int e = check_frame(img, dtype, W, H, pitch, cal)) return e;
    if (int e = check_bg(p)) return e;
    REQUIRE(mesh_bkg && mesh_rms, "mesh outputs NULL");
    size_t need = ipp_bg_estimate_workspace_size(W, H, p);
    REQUIRE(ws && ws_bytes >= need, "workspace of %zu bytes needed", need);
    return bg_estimate_impl(img, dtype, W, H, pitch, mask, cal, p, mesh_bkg, mesh_rms, raw_bkg, raw_rms,
                            status_dev, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" int ipp_bg_subtract(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                               const ipp_calib* cal, const float* mesh_bkg, const ipp_bg_params* p,
                               float* sub, int64_t sub_pitch, float* bkg_map, void* stream) {
    if (int e = check_frame(img, dtype, W, H, pitch, cal)) return e;
    if (int e = check_bg(p)) return e;
    if (int e = check_keys_only(p, "ipp_bg_subtract")) return e;
    REQUIRE(mesh_bkg && sub, "mesh_bkg / sub NULL");
    REQUIRE(sub_pitch >= W, "sub_pitch < W");
    int nx, ny;
    grid_of(W, H, p, &nx, &ny);
    SubJob J;
    J.img = img; J.dtype = dtype; J.W = W; J.H = H; J.pitch = pitch;
    J.bias_map = cal ? cal->bias_map : nullptr; J.bias = cal ? cal->bias : 0.f;
    J.inv_flat = cal ? cal->inv_flat : nullptr;
    J.mesh = mesh_bkg; J.nx = nx; J.ny = ny; J.mesh_w = p->mesh_w; J.mesh_h = p->mesh_h;
    J.sub = sub; J.sub_pitch = sub_pitch; J.bkg_map = bkg_map;
    return ipp_launch_bg_subtract(J, (cudaStream_t)stream);
}

extern "C" size_t ipp_bg_spline_workspace_size(int64_t W, int64_t H, const ipp_bg_params* p) {
    if (!p || p->mesh_w < 1 || p->mesh_h < 1 || W <= 0 || H <= 0) return 0;
    int nx, ny;
    grid_of(W, H, p, &nx, &ny);
    return ipp_spline_ws_bytes(nx, ny);
}

extern "C" int ipp_bg_subtract_spline(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                                      const ipp_calib* cal, const float* mesh_bkg, const ipp_bg_params* p,
                                      float* sub, int64_t sub_pitch, float* bkg_map, void* ws, size_t ws_bytes,
                                      void* stream) {
    if (int e = check_frame(img, dtype, W, H, pitch, cal)) return e;
    if (int e = check_bg(p)) return e;
    REQUIRE(mesh_bkg && sub, "mesh_bkg / sub NULL");
    REQUIRE(sub_pitch >= W, "sub_pitch < W");
    const size_t need = ipp_bg_spline_workspace_size(W, H, p);
    REQUIRE(ws && ws_bytes >= need && ((uintptr_t)ws & 255) == 0, "workspace of %zu bytes (256-byte aligned) needed",
            need);
    int nx, ny;
    grid_of(W, H, p, &nx, &ny);
    SubJob J;
    J.img = img; J.dtype = dtype; J.W = W; J.H = H; J.pitch = pitch;
    J.bias_map = cal ? cal->bias_map : nullptr; J.bias = cal ? cal->bias : 0.f;
    J.inv_flat = cal ? cal->inv_flat : nullptr;
    J.mesh = mesh_bkg; J.nx = nx; J.ny = ny; J.mesh_w = p->mesh_w; J.mesh_h = p->mesh_h;
    J.sub = sub; J.sub_pitch = sub_pitch; J.bkg_map = bkg_map;
    return ipp_launch_bg_subtract_spline(J, ws, (cudaStream_t)stream);
}

// ---- detection ------------------------------------------------------------------
static int check_stats(const ipp_src_stats* st) {
    REQUIRE(st && st->area && st->first && st->xmin && st->xmax && st->ymin && st->ymax && st->peak &&
                st->flux && st->xbar && st->ybar, "stats arrays NULL");
    return IPP_OK;
}

extern "C" size_t ipp_detect_label_workspace_size(int64_t W, int64_t H) {
    if (W <= 0 || H <= 0) return 0;
    return ipp_ccl_workspace_size(W, H);
}

extern "C" int ipp_detect_label(const float* sub, int64_t W, int64_t H, int64_t pitch,
                                const float* mesh_rms, const ipp_bg_params* bp, const ipp_det_params* dp,
                                const uint32_t* mask_in, int32_t* labels, int32_t* n_src_dev,
                                int32_t max_src, const ipp_src_stats* stats, void* ws, size_t ws_bytes,
                                void* stream) {
    if (int e = check_frame(sub, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(dp, "det params NULL");
    REQUIRE(dp->min_area >= 1, "min_area must be >= 1");
    REQUIRE(dp->filter == 0 || dp->filter == 1, "detection filter must be 0 or 1");
    if (!mask_in) {
        if (int e = check_bg(bp)) return e;
        if (int e = check_keys_only(bp, "ipp_detect_label")) return e;
        REQUIRE(mesh_rms, "mesh_rms NULL (needed without mask_in)");
        REQUIRE(dp->k >= 0.f, "k must be >= 0");
    }
    REQUIRE(labels && n_src_dev, "labels / n_src_dev NULL");
    REQUIRE(max_src >= 0, "max_src < 0");
    if (int e = check_stats(stats)) return e;
    size_t need = ipp_detect_label_workspace_size(W, H);
    REQUIRE(ws && ws_bytes >= need, "workspace of %zu bytes needed", need);
    DetectArgs A;
    memset(&A, 0, sizeof(A));
    A.mode = mask_in ? 1 : 0;
    A.W = W; A.H = H; A.dtype = IPP_F32;
    A.sub = const_cast<float*>(sub); A.sub_pitch = pitch;
    A.mesh_rms = mesh_rms;
    if (bp) {
        grid_of(W, H, bp, &A.nx, &A.ny);
        A.mesh_w = bp->mesh_w; A.mesh_h = bp->mesh_h;
    }
    A.k = dp->k; A.thresh_abs = dp->thresh_abs; A.min_area = dp->min_area; A.mask_in = mask_in;
    A.filter = dp->filter;
    A.labels = labels; A.n_src_dev = n_src_dev; A.max_src = max_src; A.stats = *stats; A.ws = ws;
    return ipp_launch_detect(A, (cudaStream_t)stream);
}

// ---- per source -------------------------------------------------------------------
extern "C" int ipp_centroid(const float* sub, int64_t W, int64_t H, int64_t pitch,
                            const int32_t* n_src_dev, int32_t max_src, const float* x0, const float* y0,
                            const ipp_cen_params* p, float* x, float* y, int32_t* niter, int32_t* flags,
                            void* stream) {
    if (int e = check_frame(sub, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(p && p->fwhm_win > 0.f && p->max_iter >= 1 && p->tol2 >= 0.f, "bad centroid params");
    REQUIRE(p->fwhm_win <= 16.f, "fwhm_win above 16 px not supported");
    REQUIRE(n_src_dev && x0 && y0 && x && y && flags, "NULL pointer");
    REQUIRE(max_src >= 0, "max_src < 0");
    CenJob J;
    J.sub = sub; J.W = W; J.H = H; J.pitch = pitch; J.n_src_dev = n_src_dev; J.max_src = max_src;
    J.x0 = x0; J.y0 = y0;
    J.sw = (float)(p->fwhm_win / 2.3548200450309493);
    J.rad = 4.0f * J.sw;
    J.tol2 = p->tol2; J.max_iter = p->max_iter;
    J.x = x; J.y = y; J.niter = niter; J.flags = flags;
    return ipp_launch_centroid(J, (cudaStream_t)stream);
}

extern "C" int ipp_aperture_phot(const float* sub, int64_t W, int64_t H, int64_t pitch,
                                 const int32_t* n_src_dev, int32_t max_src, const float* x, const float* y,
                                 const ipp_phot_params* p, float* flux, float* sky, float* area,
                                 int32_t* n_ann, int32_t* flags, void* stream) {
    if (int e = check_frame(sub, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(p && p->r_ap > 0.f && p->r_in >= 0.f && p->r_out > p->r_in, "bad aperture params");
    REQUIRE(p->r_ap <= 16.f, "r_ap above 16 px not supported");
    REQUIRE(n_src_dev && x && y && flux, "NULL pointer");
    REQUIRE(max_src >= 0, "max_src < 0");
    PhotJob J;
    J.sub = sub; J.W = W; J.H = H; J.pitch = pitch; J.n_src_dev = n_src_dev; J.max_src = max_src;
    J.x = x; J.y = y; J.r_ap = p->r_ap; J.r_in = p->r_in; J.r_out = p->r_out; J.min_ann = p->min_ann;
    J.flux = flux; J.sky = sky; J.area = area; J.n_ann = n_ann; J.flags = flags;
    return ipp_launch_aperture(J, (cudaStream_t)stream);
}

extern "C" int ipp_auto_phot(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t pitch,
                             const int32_t* n_src_dev, int32_t max_src, const ipp_src_stats* stats,
                             const ipp_auto_params* p, float* flux, float* area, float* kron, float* shape,
                             int32_t* flags, void* stream) {
    if (int e = check_frame(sub, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(p && p->k_kron > 0.f && p->r_min >= 0.f && p->r_kmax > 0.f, "bad auto photometry params");
    REQUIRE(labels && n_src_dev && stats && flux, "NULL pointer");
    REQUIRE(stats->xmin && stats->xmax && stats->ymin && stats->ymax && stats->xbar && stats->ybar,
            "stats arrays NULL");
    REQUIRE(max_src >= 0, "max_src < 0");
    REQUIRE((W + 2) * (H + 2) < (int64_t(1) << 31) && pitch * H < (int64_t(1) << 31),
            "auto photometry needs a frame below 2^31 pixels");
    AutoJob J;
    J.sub = sub; J.labels = labels; J.W = W; J.H = H; J.pitch = pitch;
    J.n_src_dev = n_src_dev; J.max_src = max_src;
    J.xmin = stats->xmin; J.xmax = stats->xmax; J.ymin = stats->ymin; J.ymax = stats->ymax;
    J.xbar = stats->xbar; J.ybar = stats->ybar;
    J.k_kron = p->k_kron; J.r_min = p->r_min; J.r_kmax = p->r_kmax;
    J.flux = flux; J.area = area; J.kron = kron; J.shape = shape; J.flags = flags;
    return ipp_launch_auto_phot(J, (cudaStream_t)stream);
}

extern "C" size_t ipp_deblend_workspace_size(int64_t W, int64_t H, int32_t max_src) {
    if (W <= 0 || H <= 0) return 0;
    return ipp_deblend_ws_carve(W, H, max_src, nullptr, nullptr);
}

extern "C" int ipp_deblend(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t pitch,
                           const int32_t* n_src_dev, int32_t max_src, const ipp_src_stats* stats,
                           const ipp_deblend_params* p, int32_t* out_labels, int32_t* n_out_dev, void* ws,
                           size_t ws_bytes, void* stream) {
    if (int e = check_frame(sub, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(p && p->nthresh >= 2 && p->nthresh <= 256 && p->mincont >= 0.f && p->mincont <= 1.f,
            "bad deblending params");
    REQUIRE(labels && n_src_dev && stats && out_labels && n_out_dev && ws, "NULL pointer");
    REQUIRE(stats->xmin && stats->xmax && stats->ymin && stats->ymax && stats->area, "stats arrays NULL");
    REQUIRE(max_src >= 0, "max_src < 0");
    REQUIRE(W * H < (int64_t(1) << 31), "deblending needs a frame below 2^31 pixels");
    REQUIRE(((uintptr_t)ws & 255) == 0, "workspace not 256-byte aligned");
    REQUIRE(ws_bytes >= ipp_deblend_ws_carve(W, H, max_src, nullptr, nullptr), "workspace too small");
    DeblendJob J;
    J.sub = sub; J.pitch = pitch; J.labels = labels; J.W = W; J.H = H;
    J.n_src_dev = n_src_dev; J.max_src = max_src;
    J.xmin = stats->xmin; J.xmax = stats->xmax; J.ymin = stats->ymin; J.ymax = stats->ymax; J.area = stats->area;
    J.nthresh = p->nthresh; J.mincont = (double)p->mincont;
    J.out = out_labels; J.n_out_dev = n_out_dev;
    ipp_deblend_ws_carve(W, H, max_src, ws, &J.ws);
    return ipp_launch_deblend(J, (cudaStream_t)stream);
}

// ---- cleaning -------------------------------------------------------------------------
extern "C" size_t ipp_clean_workspace_size(int32_t max_obj) {
    if (max_obj < 0 || max_obj > (1 << 24)) return 0;
    return ipp_clean_ws_bytes(max_obj);
}

extern "C" int ipp_clean(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t pitch,
                         const int32_t* n_obj_dev, int32_t max_obj, const float* thr_map, const float* mesh_rms,
                         const ipp_bg_params* bp, const ipp_det_params* dp, float beta, int32_t* out_labels,
                         int32_t* n_out_dev, void* ws, size_t ws_bytes, void* stream) {
    if (int e = check_frame(sub, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(labels && n_obj_dev && out_labels && n_out_dev && ws && dp, "NULL pointer");
    REQUIRE(beta > 0.f && std::isfinite(beta), "beta must be > 0");
    REQUIRE(max_obj >= 0 && max_obj <= (1 << 24), "max_obj outside 0..2^24");
    REQUIRE(W * H < (int64_t(1) << 31) && W < 65536, "cleaning needs a frame below 2^31 pixels, W < 65536");
    REQUIRE(((uintptr_t)ws & 255) == 0, "workspace not 256-byte aligned");
    REQUIRE(ws_bytes >= ipp_clean_ws_bytes(max_obj), "workspace too small");
    int nx = 0, ny = 0;
    float mw = 1.f, mh = 1.f;
    if (!thr_map && mesh_rms) {
        if (int e = check_bg(bp)) return e;
        if (int e = check_keys_only(bp, "ipp_clean (threshold from mesh_rms)")) return e;
        nx = (int)cdiv(W, bp->mesh_w);
        ny = (int)cdiv(H, bp->mesh_h);
        mw = (float)bp->mesh_w;
        mh = (float)bp->mesh_h;
    }
    return ipp_launch_clean(sub, pitch, labels, W, H, n_obj_dev, max_obj, thr_map, thr_map ? nullptr : mesh_rms,
                            nx, ny, mw, mh, dp->k, dp->thresh_abs, beta, out_labels, n_out_dev, ws,
                            (cudaStream_t)stream);
}

// ---- image subtraction -----------------------------------------------------------------
static int sub_nb(int32_t nk, const int32_t* deg) {
    int nb = 0;
    for (int k = 0; k < nk; k++) nb += (deg[k] + 1) * (deg[k] + 2) / 2;
    return nb;
}

extern "C" size_t ipp_sub_apply_workspace_size(int32_t hw, int32_t nk, const int32_t* deg) {
    if (hw < 1 || nk < 1 || nk > 8 || !deg) return 0;
    for (int k = 0; k < nk; k++)
        if (deg[k] < 0 || deg[k] > 8) return 0;
    return ipp_sub_ws_bytes(sub_nb(nk, deg), hw);
}

extern "C" int ipp_sub_apply(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int32_t hw,
                             int32_t nk, const float* sig, const int32_t* deg, const float* coef, int32_t sord,
                             int32_t bord, float* D, int64_t out_pitch, void* ws, size_t ws_bytes, void* stream) {
    if (int e = check_frame(I, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(R && coef && D && ws && sig && deg, "NULL pointer");
    REQUIRE(out_pitch >= W, "out_pitch < W");
    REQUIRE((const void*)D != (const void*)I && (const void*)D != (const void*)R, "D must not alias I or R");
    REQUIRE(nk >= 1 && nk <= 8, "nk must be 1..8");
    for (int k = 0; k < nk; k++)
        REQUIRE(deg[k] >= 0 && deg[k] <= 8 && sig[k] > 0.f && std::isfinite(sig[k]), "bad basis description");
    const int nb = sub_nb(nk, deg);
    REQUIRE(nb <= 64, "more than 64 basis functions");
    REQUIRE(sord >= 0 && sord <= 4 && bord >= -1 && bord <= 4, "spatial order 0..4, background order -1..4");
    REQUIRE(((W + 2 * hw) / (2 * hw + 1)) * ((H + 2 * hw) / (2 * hw + 1)) < (int64_t(1) << 31),
            "frame too large (tiles)");
    if (hw != 4 && hw != 6 && hw != 8 && hw != 10 && hw != 12)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "kernel half width %d (built: 4, 6, 8, 10, 12)", hw);
    REQUIRE(ws_bytes >= ipp_sub_ws_bytes(nb, hw) && ((uintptr_t)ws & 15) == 0, "workspace too small or misaligned");
    const int ns = (sord + 1) * (sord + 2) / 2;
    return ipp_launch_sub_apply(I, R, W, H, pitch, hw, nk, sig, deg, nb, coef, sord, coef + (size_t)nb * ns, bord,
                                D, out_pitch, ws, (cudaStream_t)stream);
}

// ---- subtraction fit --------------------------------------------------------------------
static int check_sub_fit_basis(int32_t hw, int32_t fh, int32_t nk, const double* sig, const int32_t* deg,
                               int32_t sord, int32_t bord) {
    REQUIRE(sig && deg, "NULL basis description");
    REQUIRE(hw >= 0 && fh >= 0, "hw, fh must be >= 0");
    REQUIRE(nk >= 1 && nk <= 8, "nk must be 1..8");
    for (int k = 0; k < nk; k++)
        REQUIRE(deg[k] >= 0 && deg[k] <= 8 && sig[k] > 0.0 && std::isfinite(sig[k]), "bad basis description");
    REQUIRE(sord >= 0 && sord <= 4 && bord >= -1 && bord <= 4, "spatial order 0..4, background order -1..4");
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (ipp_subfit_smem(hw, fh, nk, deg, sord, bord) > (size_t)optin)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "footprint and basis need %zu B of shared memory (> %d)",
                             ipp_subfit_smem(hw, fh, nk, deg, sord, bord), optin);
    return IPP_OK;
}

extern "C" size_t ipp_sub_fit_workspace_size(int32_t max_c, int32_t nreg, int32_t hw, int32_t fh, int32_t nk,
                                             const int32_t* deg, int32_t sord, int32_t bord) {
    if (max_c < 0 || nreg < 0 || hw < 0 || fh < 0 || nk < 1 || nk > 8 || !deg || sord < 0 || sord > 4 ||
        bord < -1 || bord > 4)
        return 0;
    for (int k = 0; k < nk; k++)
        if (deg[k] < 0 || deg[k] > 8) return 0;
    return ipp_subfit_ws_bytes(max_c, nreg, hw, fh, nk, deg, sord, bord);
}

extern "C" int ipp_sub_stamps(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int32_t nsx,
                              int32_t nsy, int32_t hw, int32_t fh, double nsig, int32_t* cx, int32_t* cy,
                              int32_t* n_dev, void* ws, size_t ws_bytes, void* stream) {
    if (int e = check_frame(I, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(R && cx && cy && n_dev && ws, "NULL pointer");
    REQUIRE(W * H < (int64_t(1) << 31), "frame of 2^31 pixels or more");
    REQUIRE(nsx >= 1 && nsy >= 1 && (int64_t)nsx * nsy <= 65536, "regions: 1..65536");
    REQUIRE(hw >= 0 && fh >= 0 && std::isfinite(nsig), "bad hw, fh or nsig");
    REQUIRE(((uintptr_t)ws & 255) == 0 && ws_bytes >= (size_t)nsx * nsy * 8, "workspace too small or misaligned");
    return ipp_launch_sub_stamps(I, R, W, H, pitch, nsx, nsy, hw, fh, nsig, cx, cy, n_dev, ws, (cudaStream_t)stream);
}

extern "C" int ipp_sub_normal(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, const int32_t* cx,
                              const int32_t* cy, const int32_t* n_dev, int32_t max_c, int32_t hw, int32_t fh,
                              int32_t nk, const double* sig, const int32_t* deg, int32_t sord, int32_t bord,
                              double* AtA, double* Atb, void* ws, size_t ws_bytes, void* stream) {
    if (int e = check_frame(I, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(R && cx && cy && n_dev && AtA && Atb && ws, "NULL pointer");
    REQUIRE(max_c >= 0 && max_c <= 65536, "max_c must be 0..65536");
    if (int e = check_sub_fit_basis(hw, fh, nk, sig, deg, sord, bord)) return e;
    REQUIRE(((uintptr_t)ws & 255) == 0 && ws_bytes >= ipp_subfit_ws_bytes(max_c, 0, hw, fh, nk, deg, sord, bord),
            "workspace too small or misaligned");
    return ipp_launch_sub_normal(I, R, W, H, pitch, cx, cy, n_dev, max_c, 0, hw, fh, nk, sig, deg, sord, bord, AtA,
                                 Atb, ws, (cudaStream_t)stream);
}

extern "C" int ipp_sub_solve(double* AtA, double* Atb, int32_t np, double* coef64, float* coef, int32_t* status_dev,
                             void* stream) {
    REQUIRE(AtA && Atb && status_dev, "NULL pointer");
    REQUIRE(np >= 1 && np <= 8192, "np must be 1..8192");
    return ipp_launch_sub_solve(AtA, Atb, np, coef64, coef, status_dev, (cudaStream_t)stream);
}

extern "C" int ipp_sub_fit(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int32_t nsx,
                           int32_t nsy, double nsig, int32_t hw, int32_t fh, int32_t nk, const double* sig,
                           const int32_t* deg, int32_t sord, int32_t bord, double* coef64, float* coef, int32_t* cx,
                           int32_t* cy, int32_t* n_dev, int32_t* status_dev, void* ws, size_t ws_bytes,
                           void* stream) {
    if (int e = check_frame(I, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(R && status_dev && ws && (coef64 || coef), "NULL pointer");
    REQUIRE(W * H < (int64_t(1) << 31), "frame of 2^31 pixels or more");
    REQUIRE(nsx >= 1 && nsy >= 1 && (int64_t)nsx * nsy <= 65536, "regions: 1..65536");
    REQUIRE(std::isfinite(nsig), "nsig not finite");
    if (int e = check_sub_fit_basis(hw, fh, nk, sig, deg, sord, bord)) return e;
    const int nreg = nsx * nsy;
    REQUIRE(((uintptr_t)ws & 255) == 0 &&
                ws_bytes >= ipp_subfit_ws_bytes(nreg, nreg, hw, fh, nk, deg, sord, bord),
            "workspace too small or misaligned");
    return ipp_launch_sub_fit(I, R, W, H, pitch, nsx, nsy, nsig, hw, fh, nk, sig, deg, sord, bord, coef64, coef, cx,
                              cy, n_dev, status_dev, ws, (cudaStream_t)stream);
}

// ---- image alignment -------------------------------------------------------------------
static int check_wcs(const ipp_wcs* w, bool need_inverse) {
    REQUIRE(w, "wcs NULL");
    REQUIRE(w->a_order >= 0 && w->a_order <= 5 && w->b_order >= 0 && w->b_order <= 5, "SIP order must be 0..5");
    for (int k = 0; k < 2; k++) REQUIRE(std::isfinite(w->crpix[k]) && std::isfinite(w->crval[k]), "non-finite WCS");
    for (int k = 0; k < 4; k++) REQUIRE(std::isfinite(w->cd[k]), "non-finite CD");
    for (int k = 0; k < 36; k++) REQUIRE(std::isfinite(w->a[k]) && std::isfinite(w->b[k]), "non-finite SIP term");
    if (need_inverse) REQUIRE(w->cd[0] * w->cd[3] - w->cd[1] * w->cd[2] != 0.0, "singular target CD");
    return IPP_OK;
}

extern "C" int ipp_wcs_map(const ipp_wcs* src, const ipp_wcs* tgt, int64_t W, int64_t H, int32_t step,
                           double* x_out, double* y_out, void* stream) {
    if (int e = check_wcs(src, false)) return e;
    if (int e = check_wcs(tgt, true)) return e;
    REQUIRE(W >= 1 && H >= 1 && step >= 1, "W, H and step must be >= 1");
    REQUIRE(x_out && y_out, "NULL output");
    return ipp_launch_wcs_map(*src, *tgt, (W - 1) / step + 1, (H - 1) / step + 1, step, x_out, y_out,
                              (cudaStream_t)stream);
}

extern "C" size_t ipp_affine_fit_workspace_size(void) { return ipp_affine_ws_bytes(); }

extern "C" int ipp_affine_fit(const double* x, const double* y, const double* xt, const double* yt, int64_t n,
                              int64_t grid_nx, int32_t grid_step, double* M_out, int32_t* status_dev, void* ws,
                              size_t ws_bytes, void* stream) {
    REQUIRE(xt && yt && M_out && ws, "NULL pointer");
    REQUIRE((x == nullptr) == (y == nullptr), "x and y must both be given or both be NULL");
    REQUIRE(n >= 0, "n < 0");
    if (!x) REQUIRE(grid_nx >= 1 && grid_step >= 1, "grid_nx and grid_step must be >= 1");
    REQUIRE(((uintptr_t)ws & 7) == 0 && ws_bytes >= ipp_affine_ws_bytes(), "workspace misaligned or too small");
    return ipp_launch_affine_fit(x, y, xt, yt, n, grid_nx, grid_step, M_out, status_dev, ws, (cudaStream_t)stream);
}

extern "C" int ipp_reproject_affine(const float* src, int64_t W, int64_t H, int64_t pitch, const double* Minv_dev,
                                    int64_t Wo, int64_t Ho, float fill, float* out, int64_t out_pitch,
                                    void* stream) {
    if (int e = check_frame(src, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(Minv_dev && out, "NULL pointer");
    REQUIRE(Wo >= 1 && Ho >= 1 && Wo < (1ll << 24) && Ho < (1ll << 24) && out_pitch >= Wo, "bad output size");
    REQUIRE((const void*)out != (const void*)src, "out must not alias src");
    return ipp_launch_reproject(src, W, H, pitch, Minv_dev, Wo, Ho, fill, out, out_pitch, (cudaStream_t)stream);
}

// ---- gray-scale maps ------------------------------------------------------------------
extern "C" int ipp_gray_transform(const float* img, int64_t W, int64_t H, int64_t pitch, int32_t kind, float lo,
                                  float hi, float a, float* out, int64_t out_pitch, void* stream) {
    if (int e = check_frame(img, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(out && out_pitch >= W, "out NULL or out_pitch < W");
    REQUIRE((const void*)out != (const void*)img, "out must not alias img");
    REQUIRE(kind >= IPP_GRAY_LINEAR && kind <= IPP_GRAY_EXP, "unknown gray function %d", kind);
    REQUIRE(std::isfinite(lo) && std::isfinite(hi) && lo < hi, "need finite lo < hi");
    if (kind != IPP_GRAY_LINEAR) REQUIRE(a > 0.f && std::isfinite(a), "need finite a > 0");
    if (kind == IPP_GRAY_EXP) REQUIRE(a != 1.f, "exponential map needs a != 1");
    return ipp_launch_gray(img, W, H, pitch, kind, lo, hi, a, out, out_pitch, (cudaStream_t)stream);
}

extern "C" int ipp_zscale(const float* img, int64_t W, int64_t H, int64_t pitch, const ipp_zscale_params* p,
                          double* z_out, int32_t* counts_out, void* stream) {
    if (int e = check_frame(img, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(p && p->n_samples >= 1 && p->n_samples <= 4096, "n_samples must be 1..4096");
    REQUIRE(p->contrast > 0.f && std::isfinite(p->contrast) && p->krej > 0.f && std::isfinite(p->krej),
            "contrast and krej must be finite and > 0");
    REQUIRE(p->max_iter >= 0 && p->max_iter <= 100, "max_iter must be 0..100");
    REQUIRE(z_out, "z_out NULL");
    return ipp_launch_zscale(img, W, H, pitch, p->n_samples, (double)p->contrast, (double)p->krej, p->max_iter,
                             z_out, counts_out, (cudaStream_t)stream);
}

extern "C" size_t ipp_hist_equalize_workspace_size(int32_t nbins) {
    if (nbins < 2 || nbins > 16384) return 0;
    return ipp_equalize_ws_bytes(nbins);
}

extern "C" int ipp_hist_equalize(const float* img, int64_t W, int64_t H, int64_t pitch, int32_t nbins, float* out,
                                 int64_t out_pitch, void* ws, size_t ws_bytes, void* stream) {
    if (int e = check_frame(img, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(nbins >= 2 && nbins <= 16384, "nbins must be 2..16384 (got %d)", nbins);
    REQUIRE(out && out_pitch >= W, "out NULL or out_pitch < W");
    REQUIRE((const void*)out != (const void*)img, "out must not alias img");
    REQUIRE(ws && ((uintptr_t)ws & 255) == 0, "workspace NULL or not 256-byte aligned");
    REQUIRE(ws_bytes >= ipp_equalize_ws_bytes(nbins), "workspace too small");
    return ipp_launch_equalize(img, W, H, pitch, nbins, out, out_pitch, ws, (cudaStream_t)stream);
}

extern "C" int ipp_stamp_cut(const float* sub, int64_t W, int64_t H, int64_t pitch, const int32_t* n_src_dev,
                             int32_t max_src, const float* x, const float* y, int32_t S, float* stamps,
                             float* weights, int32_t* origin, int32_t* flags, void* stream) {
    if (int e = check_frame(sub, IPP_F32, W, H, pitch, nullptr)) return e;
    REQUIRE(S >= 3 && S <= 63 && (S & 1), "stamp size S must be odd, 3..63");
    REQUIRE(n_src_dev && x && y && stamps, "NULL pointer");
    REQUIRE(max_src >= 0, "max_src < 0");
    return ipp_launch_stamp_cut(sub, W, H, pitch, n_src_dev, max_src, x, y, S, stamps, weights, origin, flags,
                                (cudaStream_t)stream);
}

// ---- fused frame ---------------------------------------------------------------------
// ipp_extract's workspace: the mesh statistics' scratch, the labeling's, then
// the spline node tables of the mesh bkg and rms (used with interp = spline)
static size_t extract_spline_off(int64_t W, int64_t H, const ipp_bg_params* bp) {
    return a256(ipp_bg_estimate_workspace_size(W, H, bp)) + a256(ipp_ccl_workspace_size(W, H));
}

extern "C" size_t ipp_extract_workspace_size(int64_t W, int64_t H, const ipp_bg_params* bp) {
    if (!bp || bp->mesh_w < 1 || bp->mesh_h < 1) return 0;
    int nx, ny;
    grid_of(W, H, bp, &nx, &ny);
    return extract_spline_off(W, H, bp) + 2 * a256(ipp_spline_ws_bytes(nx, ny));
}

// The jobs of ipp_extract for one frame, after its argument checks: the mesh
// statistics and filter, the fused subtraction / detection, the centroid and
// the aperture photometry.  Shared by ipp_extract and the batched form, so the
// two run the same arithmetic on the same workspace layout.
int ipp_extract_jobs(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch, const ipp_calib* cal,
                     const ipp_bg_params* bp, const ipp_det_params* dp, const ipp_cen_params* cp,
                     const ipp_phot_params* pp, int32_t max_src, const ipp_catalog_out* out, void* ws,
                     size_t ws_bytes, MeshJob* M, MeshFilterJob* F, DetectArgs* A, CenJob* C, PhotJob* P) {
    if (int e = check_frame(img, dtype, W, H, pitch, cal)) return e;
    if (int e = check_bg(bp)) return e;
    REQUIRE(dp && cp && pp && out, "NULL parameter struct");
    REQUIRE(out->mesh_bkg && out->mesh_rms && out->sub && out->labels && out->n_src_dev, "NULL output");
    REQUIRE(out->x && out->y && out->cen_flags && out->flux, "NULL per-source output");
    if (int e = check_stats(&out->stats)) return e;
    REQUIRE(dp->min_area >= 1 && dp->k >= 0.f, "bad detection params");
    REQUIRE(dp->filter == 0 || dp->filter == 1, "detection filter must be 0 or 1");
    REQUIRE(cp->fwhm_win > 0.f && cp->fwhm_win <= 16.f && cp->max_iter >= 1 && cp->tol2 >= 0.f,
            "bad centroid params");
    REQUIRE(pp->r_ap > 0.f && pp->r_ap <= 16.f && pp->r_out > pp->r_in && pp->r_in >= 0.f, "bad aperture params");
    REQUIRE(pp->r_out <= 16.f, "r_out above 16 px not supported");
    REQUIRE(max_src >= 0, "max_src < 0");
    size_t need = ipp_extract_workspace_size(W, H, bp);
    REQUIRE(ws && ws_bytes >= need, "workspace of %zu bytes needed", need);
    unsigned char* w = (unsigned char*)ws;
    const size_t bgws = a256(ipp_bg_estimate_workspace_size(W, H, bp));
    int nx, ny;
    grid_of(W, H, bp, &nx, &ny);
    const size_t nb = a256((size_t)nx * ny * sizeof(float));
    float* rb = (float*)(w + 0 * nb);
    float* rr = (float*)(w + 1 * nb);
    // mesh statistics (as ipp_bg_estimate)
    memset(M, 0, sizeof(*M));
    M->img = img; M->dtype = dtype; M->W = W; M->H = H; M->pitch = pitch; M->mask = nullptr;
    M->bias_map = cal ? cal->bias_map : nullptr; M->bias = cal ? cal->bias : 0.f;
    M->inv_flat = cal ? cal->inv_flat : nullptr;
    M->mesh_w = bp->mesh_w; M->mesh_h = bp->mesh_h; M->nx = nx; M->ny = ny;
    M->maxiters = bp->maxiters; M->min_valid = bp->min_valid; M->estimator = bp->estimator;
    M->nsigma = bp->nsigma; M->mf = bp->median_factor; M->mnf = bp->mean_factor;
    M->raw_bkg = rb; M->raw_rms = rr;
    F->raw_bkg = rb; F->raw_rms = rr;
    F->fill_bkg = (float*)(w + 2 * nb); F->fill_rms = (float*)(w + 3 * nb);
    F->nx = nx; F->ny = ny; F->fw = bp->filter_w; F->fh = bp->filter_h;
    F->out_bkg = out->mesh_bkg; F->out_rms = out->mesh_rms; F->status_dev = out->status_dev;
    // fused subtraction, threshold and labeling
    memset(A, 0, sizeof(*A));
    A->mode = 2;
    A->W = W; A->H = H; A->img = img; A->dtype = dtype; A->pitch = pitch;
    A->bias_map = cal ? cal->bias_map : nullptr; A->bias = cal ? cal->bias : 0.f;
    A->inv_flat = cal ? cal->inv_flat : nullptr;
    A->mesh_bkg = out->mesh_bkg; A->sub = out->sub; A->sub_pitch = W; A->mesh_rms = out->mesh_rms;
    A->nx = nx; A->ny = ny;
    A->mesh_w = bp->mesh_w; A->mesh_h = bp->mesh_h;
    A->k = dp->k; A->thresh_abs = dp->thresh_abs; A->min_area = dp->min_area; A->mask_in = nullptr;
    A->filter = dp->filter;
    A->labels = out->labels; A->n_src_dev = out->n_src_dev; A->max_src = max_src; A->stats = out->stats;
    A->ws = w + bgws;
    A->interp = bp->interp;
    if (bp->interp == IPP_INTERP_SPLINE) {
        if (dp->filter) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "detection filter with the spline reading");
        const size_t so = extract_spline_off(W, H, bp);
        A->bnodes = reinterpret_cast<const float4*>(w + so);
        A->rnodes = reinterpret_cast<const float4*>(w + so + a256(ipp_spline_ws_bytes(nx, ny)));
    }
    // centroid (as ipp_centroid) and aperture photometry (as ipp_aperture_phot)
    memset(C, 0, sizeof(*C));
    C->sub = out->sub; C->W = W; C->H = H; C->pitch = W; C->n_src_dev = out->n_src_dev; C->max_src = max_src;
    C->x0 = out->stats.xbar; C->y0 = out->stats.ybar;
    C->sw = (float)(cp->fwhm_win / 2.3548200450309493);
    C->rad = 4.0f * C->sw;
    C->tol2 = cp->tol2; C->max_iter = cp->max_iter;
    C->x = out->x; C->y = out->y; C->niter = nullptr; C->flags = out->cen_flags;
    memset(P, 0, sizeof(*P));
    P->sub = out->sub; P->W = W; P->H = H; P->pitch = W; P->n_src_dev = out->n_src_dev; P->max_src = max_src;
    P->x = out->x; P->y = out->y; P->r_ap = pp->r_ap; P->r_in = pp->r_in; P->r_out = pp->r_out;
    P->min_ann = pp->min_ann;
    P->flux = out->flux; P->sky = out->sky; P->area = out->area; P->n_ann = out->n_ann; P->flags = out->phot_flags;
    return IPP_OK;
}

extern "C" int ipp_extract(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                           const ipp_calib* cal, const ipp_bg_params* bp, const ipp_det_params* dp,
                           const ipp_cen_params* cp, const ipp_phot_params* pp, int32_t max_src,
                           const ipp_catalog_out* out, void* ws, size_t ws_bytes, void* stream) {
    MeshJob M;
    MeshFilterJob F;
    DetectArgs A;
    CenJob C;
    PhotJob P;
    if (int e = ipp_extract_jobs(img, dtype, W, H, pitch, cal, bp, dp, cp, pp, max_src, out, ws, ws_bytes, &M, &F,
                                 &A, &C, &P))
        return e;
    cudaStream_t s = (cudaStream_t)stream;
    if (int e = ipp_launch_mesh_stats(M, s)) return e;
    if (int e = ipp_launch_mesh_filter(F.raw_bkg, F.raw_rms, F.fill_bkg, F.fill_rms, F.nx, F.ny, F.fw, F.fh,
                                       F.out_bkg, F.out_rms, F.status_dev, s))
        return e;
    if (A.interp == IPP_INTERP_SPLINE) {   // node tables of the filtered grids
        if (int e = ipp_launch_spline_nodes(F.out_bkg, F.nx, F.ny, (void*)A.bnodes, s)) return e;
        if (int e = ipp_launch_spline_nodes(F.out_rms, F.nx, F.ny, (void*)A.rnodes, s)) return e;
    }
    if (int e = ipp_launch_detect(A, s)) return e;
    if (int e = ipp_launch_centroid(C, s)) return e;
    return ipp_launch_aperture(P, s);
}

// ---- PSF fit and differentiable model --------------------------------------------
static int check_fit(const ipp_fit_params* p, int32_t S) {
    REQUIRE(p, "fit params NULL");
    REQUIRE(p->model == IPP_PSF_MOFFAT || p->model == IPP_PSF_GAUSS, "unknown PSF model %d", p->model);
    REQUIRE(p->model != IPP_PSF_MOFFAT || p->beta > 1.0f, "Moffat beta must be > 1");
    REQUIRE(S >= 3 && S <= 32, "stamp size %d outside 3..32", S);
    return IPP_OK;
}

extern "C" int ipp_psf_fit(const float* stamps, int64_t N, int32_t S, const float* weights,
                           const float* init, const ipp_fit_params* p, float* params, float* chi2,
                           int32_t* iters, int32_t* flags, void* stream) {
    if (int e = check_fit(p, S)) return e;
    REQUIRE(N >= 0, "N < 0");
    if (N == 0) return IPP_OK;
    REQUIRE(stamps && params && chi2, "NULL pointer");
    REQUIRE(p->max_iter >= 1 && p->lambda0 > 0.f, "bad LM params");
    FitJob J;
    J.stamps = stamps; J.N = N; J.n_dev = nullptr; J.S = S; J.weights = weights; J.init = init;
    J.model = p->model; J.beta = p->beta; J.max_iter = p->max_iter; J.lambda0 = p->lambda0;
    J.params = params; J.chi2 = chi2; J.iters = iters; J.flags = flags;
    return ipp_launch_psf_fit(J, (cudaStream_t)stream);
}

extern "C" int ipp_psf_fit_dev(const float* stamps, const int32_t* n_dev, int64_t n_max, int32_t S,
                               const float* weights, const float* init, const ipp_fit_params* p, float* params,
                               float* chi2, int32_t* iters, int32_t* flags, void* stream) {
    if (int e = check_fit(p, S)) return e;
    REQUIRE(n_max >= 0, "n_max < 0");
    REQUIRE(n_dev, "n_dev NULL");
    if (n_max == 0) return IPP_OK;
    REQUIRE(stamps && params && chi2, "NULL pointer");
    REQUIRE(p->max_iter >= 1 && p->lambda0 > 0.f, "bad LM params");
    FitJob J;
    J.stamps = stamps; J.N = n_max; J.n_dev = n_dev; J.S = S; J.weights = weights; J.init = init;
    J.model = p->model; J.beta = p->beta; J.max_iter = p->max_iter; J.lambda0 = p->lambda0;
    J.params = params; J.chi2 = chi2; J.iters = iters; J.flags = flags;
    return ipp_launch_psf_fit(J, (cudaStream_t)stream);
}

extern "C" int ipp_psf_model_fwd(const float* params, int64_t N, int32_t S, const ipp_fit_params* p,
                                 float* model, void* stream) {
    if (int e = check_fit(p, S)) return e;
    REQUIRE(N >= 0, "N < 0");
    if (N == 0) return IPP_OK;
    REQUIRE(params && model, "NULL pointer");
    return ipp_launch_psf_fwd(params, N, S, p->model, p->beta, model, (cudaStream_t)stream);
}

extern "C" int ipp_psf_model_adj(const float* params, int64_t N, int32_t S, const ipp_fit_params* p,
                                 const float* grad_model, float* grad_params, void* stream) {
    if (int e = check_fit(p, S)) return e;
    REQUIRE(N >= 0, "N < 0");
    if (N == 0) return IPP_OK;
    REQUIRE(params && grad_model && grad_params, "NULL pointer");
    return ipp_launch_psf_adj(params, N, S, p->model, p->beta, grad_model, grad_params, (cudaStream_t)stream);
}
