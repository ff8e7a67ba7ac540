/*
 * ipp.h -- C ABI of the GB300 (sm_103a) catalog path.
 *
 * The library implements the per-frame hot path of the GPU image
 * pre-processing method of Cao, Jia et al., "Image Pre-Processing Framework for
 * Time-Domain Astronomy in the Artificial Intelligence Era" (arXiv 2502.10783):
 *
 *   ipp_bg_estimate   mesh background: iterative sigma clip per mesh, the
 *                     2.5 median - 1.5 mean estimator, median filter on the
 *                     mesh grid                               (Sec. 2.2.2, Eqs. 1-4)
 *   ipp_bg_subtract   interpolation of the mesh back to full resolution and
 *                     subtraction                             (Sec. 2.2.2)
 *   ipp_detect_label  pixel detection above k x local rms, 8-connected
 *                     labeling, per-candidate peak / flux     (Sec. 2.2.5)
 *   ipp_centroid      windowed centroid of each candidate     (positions, Sec. 2.2.5)
 *   ipp_aperture_phot circular aperture photometry with a local sky annulus
 *                                                             (Sec. 2.2.5)
 *   ipp_deblend       multi-threshold deblending of the candidates (Sec. 2.2.5)
 *   ipp_clean         cleaning of the deblended objects (Sec. 2.2.5)
 *   ipp_auto_phot     auto (Kron) photometry in an elliptical aperture (Sec. 2.2.5)
 *   ipp_stamp_cut     S x S stamps at the measured positions (input of the fit)
 *   ipp_psf_fit       batched Levenberg-Marquardt PSF fit of stamps
 *   ipp_extract       all catalog steps of one frame, fused where the data allow
 *
 * and, beside that path:
 *
 *   ipp_wcs_map, ipp_affine_fit, ipp_reproject_affine
 *                     image alignment through both frames' WCS   (Sec. 2.2.3, Eqs. 5-7)
 *   ipp_sub_apply     convolution and difference of image subtraction
 *                                                             (Sec. 2.2.4, Eqs. 8-10)
 *   ipp_gray_transform, ipp_hist_equalize, ipp_zscale
 *                     gray-scale maps and display limits       (Sec. 2.2.6)
 *
 * Conventions for every call
 *   - Pixel (row i, col j) has its centre at (x = j, y = i).  Frames are row-major
 *     with `pitch` elements between rows (pitch >= W).
 *   - Every pointer argument is a DEVICE pointer unless stated otherwise; the
 *     caller owns all buffers.  Parameter structs are host pointers, read during
 *     the call only.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *   - Calls enqueue work on `stream` and return without synchronising.  Counts
 *     that depend on the data (number of sources) stay in device memory.
 *   - The return value is an IPP_* status.  IPP_ERR_INVALID_ARG and
 *     IPP_ERR_NOT_SUPPORTED are detected on the host before anything is enqueued;
 *     IPP_ERR_CUDA reports a launch failure (ipp_last_error_detail() has the
 *     text).  Errors that arise on the device are reported through the device
 *     status words documented per call, never by trapping.
 *   - Workspaces (`ws`) are device buffers of at least the size returned by the
 *     matching *_workspace_size() query, 256-byte aligned.  The library allocates
 *     no device memory inside a call.
 */
#ifndef IPP_H
#define IPP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define IPP_OK 0
#define IPP_ERR_INVALID_ARG 1   /* null pointer, bad size, pitch < W, misalignment, bad parameter */
#define IPP_ERR_CUDA 2          /* CUDA launch/runtime error; detail in ipp_last_error_detail() */
#define IPP_ERR_CAPACITY 3      /* device status: more sources than max_src (see ipp_detect_label) */
#define IPP_ERR_NO_VALID_MESH 4 /* device status: no mesh had enough usable pixels */
#define IPP_ERR_TIMEOUT 5       /* device status: a bounded device-side wait ran out */
#define IPP_ERR_NOT_SUPPORTED 6 /* valid request outside what this build implements */
#define IPP_ERR_DEGENERATE 7    /* device status: too few usable points (ipp_affine_fit) */

/* image element types */
#define IPP_F32 0
#define IPP_U16 1

/* per-source flag bits */
#define IPP_FLAG_EDGE 1              /* window / aperture / annulus crosses the frame edge */
#define IPP_FLAG_WIN_NOT_CONVERGED 2 /* windowed centroid did not converge (seed kept if sum <= 0) */
#define IPP_FLAG_ANN_FEW 4           /* fewer than min_ann annulus pixels: sky = 0 */
#define IPP_FLAG_FIT_MAXITER 8       /* PSF fit stopped at max_iter */
#define IPP_FLAG_FIT_SINGULAR 16     /* PSF fit normal matrix not positive definite */
#define IPP_FLAG_FIT_BAD_SIGMA 32    /* PSF fit width at or below 0.05 px */
#define IPP_FLAG_KRON_BAD 64         /* auto photometry: no usable Kron radius (minimum aperture used) */

/* background estimators (Sec. 2.2.2) */
#define IPP_EST_SIGMA 0   /* Eq. 3: 2.5 median - 1.5 mean (default) */
#define IPP_EST_MEDIAN 1  /* Eq. 1 */
#define IPP_EST_MEAN 2    /* Eq. 2 */
#define IPP_EST_FACTORS 3 /* Eq. 4, read as median_factor * median - mean_factor * mean */

/* PSF models */
/* World coordinate system of a frame (Sec. 2.2.3, Eqs. 5-7): SIP distortion,
 * CD matrix and gnomonic (TAN) projection. */
typedef struct {
    double crpix[2];     /* reference pixel, FITS 1-based (0-based pixel j is FITS j + 1) */
    double crval[2];     /* RA, Dec of the reference pixel, degrees */
    double cd[4];        /* CD1_1, CD1_2, CD2_1, CD2_2, degrees per pixel */
    int32_t a_order;     /* SIP orders 0..5 (0: no distortion) */
    int32_t b_order;
    double a[36];        /* a[p*6 + q]: coefficient of u^p v^q in xi, p + q <= a_order */
    double b[36];        /* likewise in eta */
} ipp_wcs;

/* ZScale parameters (Sec. 2.2.6; defaults of the published IRAF algorithm). */
typedef struct {
    int32_t n_samples;  /* pixels sampled at a flat stride, 1..4096 [1000] */
    float contrast;     /* slope divisor, > 0 [0.25] */
    float krej;         /* rejection threshold in sigma of the residuals, > 0 [2.5] */
    int32_t max_iter;   /* fit-and-reject passes, 0..100 [5] */
} ipp_zscale_params;

/* Gray-scale functions of ipp_gray_transform (Sec. 2.2.6). */
#define IPP_GRAY_LINEAR 0
#define IPP_GRAY_LOG 1
#define IPP_GRAY_POWER 2
#define IPP_GRAY_EXP 3

#define IPP_INTERP_KEYS 0
#define IPP_INTERP_SPLINE 1

#define IPP_PSF_MOFFAT 0
#define IPP_PSF_GAUSS 1

/* Mesh background parameters (Sec. 2.2.2).  Defaults in brackets. */
typedef struct {
    int32_t mesh_w, mesh_h;     /* mesh size in px [64, 64]; 4 <= size, mesh_w*mesh_h <= 16384 */
    int32_t filter_w, filter_h; /* median-filter window on the mesh grid, odd, <= 7 [3, 3] */
    int32_t maxiters;           /* clip passes [10] */
    int32_t min_valid;          /* usable pixels for a valid mesh [100] */
    int32_t estimator;          /* IPP_EST_* [IPP_EST_SIGMA] */
    int32_t interp;             /* IPP_INTERP_KEYS [default]: Keys cubic convolution of the nodes;
                                   IPP_INTERP_SPLINE: the natural tensor-product spline (the map of
                                   ipp_bg_subtract_spline), used by ipp_extract for both the
                                   background and the rms of the threshold; calls that interpolate
                                   without a spline workspace (ipp_bg_subtract, ipp_detect_label,
                                   ipp_clean from mesh_rms, the table form of the batch) return
                                   IPP_ERR_NOT_SUPPORTED for it */
    double nsigma;              /* clip half-width in sigma [3] */
    double median_factor;       /* Eq. 4 [2.5] */
    double mean_factor;         /* Eq. 4 [1.5] */
} ipp_bg_params;

/* Detection parameters (Sec. 2.2.5). */
typedef struct {
    float k;            /* threshold in units of the interpolated mesh rms [1.5] */
    float thresh_abs;   /* absolute floor of the threshold, ADU [0] */
    int32_t min_area;   /* smallest kept candidate, px [5] */
    int32_t filter;     /* 0: threshold sub itself [0]; 1: threshold sub smoothed by the
                           3 x 3 pyramid [1 2 1; 2 4 2; 1 2 1] / 16, weights renormalised over
                           the taps inside the frame (detection filter; statistics still
                           from the unsmoothed sub) */
} ipp_det_params;

/* Windowed-centroid parameters (paper-silent reading). */
typedef struct {
    float fwhm_win;     /* window FWHM, px: sigma_w = fwhm / 2.35482, radius 4 sigma_w [3] */
    int32_t max_iter;   /* [16] */
    float tol2;         /* stop when the squared step is below this, px^2 [1e-8] */
    int32_t reserved;
} ipp_cen_params;

/* Aperture photometry parameters. */
typedef struct {
    float r_ap;         /* aperture radius, px [5] */
    float r_in, r_out;  /* sky annulus: pixel centres with r_in <= d < r_out [8, 12]; r_out <= 32 */
    int32_t min_ann;    /* fewest annulus pixels for a sky value [10] */
} ipp_phot_params;

/* Deblending parameters (Sec. 2.2.5; values are readings). */
typedef struct {
    int32_t nthresh;    /* number of levels N between a candidate's lowest and highest pixel [32] */
    float mincont;      /* a branch splits off when it holds this fraction of the candidate's flux [0.005] */
} ipp_deblend_params;

/* Auto (Kron) photometry parameters (paper-silent reading). */
typedef struct {
    float k_kron;       /* aperture = k_kron x Kron radius, in moment units [2.5] */
    float r_min;        /* smallest aperture, moment units [3.5] */
    float r_kmax;       /* Kron radius measured out to this moment radius [6] */
    int32_t reserved;
} ipp_auto_params;

/* PSF fit parameters (paper-silent reading). */
typedef struct {
    int32_t model;      /* IPP_PSF_MOFFAT or IPP_PSF_GAUSS */
    float beta;         /* Moffat exponent [2.5] */
    int32_t max_iter;   /* LM trials [50] */
    float lambda0;      /* initial damping [1e-3] */
} ipp_fit_params;

/* Per-source statistics of ipp_detect_label: device arrays of max_src entries
 * (structure of arrays).  Entry k describes label k+1. */
typedef struct {
    int32_t* area;      /* pixels */
    int64_t* first;     /* raster index i*W + j of the first pixel */
    int32_t* xmin;
    int32_t* xmax;
    int32_t* ymin;
    int32_t* ymax;
    float* peak;        /* largest value */
    float* flux;        /* isophotal flux: sum of values */
    float* xbar;        /* flux-weighted barycentre */
    float* ybar;
} ipp_src_stats;

/* Bias/flat calibration for IPP_U16 frames: f = (raw - bias) * inv_flat. */
typedef struct {
    const float* bias_map;  /* nullable device map (pitch = W); else `bias` */
    float bias;
    int32_t reserved;
    const float* inv_flat;  /* device map of 1/flat, pitch = W (required) */
} ipp_calib;

/* ------------------------------------------------------------ queries */
const char* ipp_status_string(int status);
/* Text of the last IPP_ERR_CUDA / argument error seen by this host thread. */
const char* ipp_last_error_detail(void);
/* 0 on success; fills the library version triple. */
int ipp_version(int* major, int* minor, int* patch);

/* ---------------------------------------------------------- background */
/*
 * ipp_bg_estimate -- mesh statistics and mesh filter (Sec. 2.2.2, Eqs. 1-4).
 * The frame is cut into mesh_w x mesh_h regions (nx = ceil(W / mesh_w),
 * ny = ceil(H / mesh_h); partial last meshes keep their real pixels).  Per mesh,
 * over the unmasked finite pixels: repeat up to maxiters times -- median (Eq. 1),
 * mean (Eq. 2) and population sigma of the current set, drop values outside
 * [median - nsigma sigma, median + nsigma sigma] (bounds inclusive) -- until no
 * value is dropped; the background is the chosen estimator of the final set
 * (Eq. 3 by default) and the rms its sigma.  Meshes with fewer than min_valid
 * usable pixels take the median of the valid meshes in the nearest
 * (2k+1)^2 neighbourhood that holds any.  Both grids are then median filtered
 * with a filter_w x filter_h window that shrinks at the grid edges.
 *   img       device frame, dtype IPP_F32 (or IPP_U16 with `cal`), pitch elements
 *   mask      nullable device uint8 map (pitch = W); nonzero excludes the pixel
 *   cal       calibration for IPP_U16 input (nullable for IPP_F32)
 *   mesh_bkg, mesh_rms   device float[ny * nx] outputs (filtered)
 *   raw_bkg, raw_rms     nullable device float[ny * nx]: values before fill/filter
 *                        (invalid meshes hold -1 in raw_rms)
 *   ws, ws_bytes         workspace of ipp_bg_estimate_workspace_size() bytes
 *   status_dev           nullable device int32: set to IPP_ERR_NO_VALID_MESH when
 *                        no mesh is valid (outputs then hold 0), else IPP_OK
 */
size_t ipp_bg_estimate_workspace_size(int64_t W, int64_t H, const ipp_bg_params* p);
int ipp_bg_estimate(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                    const uint8_t* mask, const ipp_calib* cal, const ipp_bg_params* p,
                    float* mesh_bkg, float* mesh_rms, float* raw_bkg, float* raw_rms,
                    int32_t* status_dev, void* ws, size_t ws_bytes, void* stream);

/*
 * ipp_bg_estimate_noalloc -- ipp_bg_estimate for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is an interface choice.
 * Some callers must not call cudaMalloc once they run -- real-time pipelines
 * with a device-memory budget fixed at start-up, or code called back from
 * another framework, where an allocation may synchronise the device or break
 * that framework's memory accounting.  This variant takes no workspace: its
 * scratch is a device array inside the library of IPP_BG_NOALLOC_MAX_MESHES
 * nodes x 4 floats (256 KiB), which every GPU that loads the library keeps until
 * the process exits.  The caller still passes the frame and the output grids.
 *   - Same arguments and results as ipp_bg_estimate, minus raw_* and ws.
 *   - A mesh grid larger than IPP_BG_NOALLOC_MAX_MESHES nodes is rejected with
 *     IPP_ERR_NOT_SUPPORTED (nothing is enqueued).
 *   - The first call on a device looks up the scratch address on that device;
 *     make that first call before any stream capture.
 *   - All calls on a device share the one scratch array: calls whose work can
 *     overlap on the GPU (different streams without ordering) race and give
 *     wrong results.  Calls ordered on one stream are fine.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define IPP_BG_NOALLOC_MAX_MESHES 16384
int ipp_bg_estimate_noalloc(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                            const uint8_t* mask, const ipp_calib* cal, const ipp_bg_params* p,
                            float* mesh_bkg, float* mesh_rms, int32_t* status_dev, void* stream);

/*
 * ipp_bg_subtract -- interpolation back to full resolution and subtraction
 * (Sec. 2.2.2).  Node (p, q) of the filtered mesh sits at
 * ((q + 1/2) mesh_w - 1/2, (p + 1/2) mesh_h - 1/2); the background at each pixel
 * is the separable Keys (1981) cubic convolution (a = -1/2) of the 4 x 4 nearest
 * nodes, indices clamped to the grid.  sub = f - B.
 *   sub        device float output, sub_pitch elements per row (may alias img
 *              only when dtype is IPP_F32 and pitches match)
 *   bkg_map    nullable device float output of B (pitch = sub_pitch)
 */
int ipp_bg_subtract(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                    const ipp_calib* cal, const float* mesh_bkg, const ipp_bg_params* p,
                    float* sub, int64_t sub_pitch, float* bkg_map, void* stream);

/*
 * ipp_bg_subtract_spline -- the natural-spline reading of Sec. 2.2.2's spline
 * interpolation back to full resolution (the default reading is the Keys cubic
 * of ipp_bg_subtract): B is the tensor product of 1-D natural cubic splines
 * through the filtered mesh nodes (node positions as in ipp_bg_subtract, zero
 * second derivative at the end nodes, beyond them the line with the end slope);
 * sub = f - B.  Arguments as ipp_bg_subtract, plus a workspace of
 * ipp_bg_spline_workspace_size() bytes, 256-byte aligned (the nodes' values
 * and second derivatives).  FP32.
 */
size_t ipp_bg_spline_workspace_size(int64_t W, int64_t H, const ipp_bg_params* p);
int ipp_bg_subtract_spline(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                           const ipp_calib* cal, const float* mesh_bkg, const ipp_bg_params* p,
                           float* sub, int64_t sub_pitch, float* bkg_map, void* ws, size_t ws_bytes,
                           void* stream);

/* --------------------------------------------------------------- detection */
/*
 * ipp_detect_label -- pixel detection and connection into candidates, with the
 * per-candidate pre-analysis of Sec. 2.2.5.  A pixel is detected when
 * sub > max(k * rms(x, y), thresh_abs), rms(x, y) being the Keys interpolation of
 * mesh_rms; detected pixels are joined into 8-connected components; components
 * smaller than min_area pixels are dropped and the rest numbered 1..K in raster
 * order of their first pixel (the numbering does not depend on tiling).
 *   mask_in    nullable device bit mask that replaces the threshold: row i holds
 *              ceil(W/32) uint32 words, pixel (i, j) is bit (j % 32) of word j / 32
 *   labels     device int32 map, pitch = W (0 = background)
 *   n_src_dev  device int32: K, the number of candidates (all of them, even above
 *              max_src)
 *   stats      host struct of device arrays of max_src entries; entries for labels
 *              above max_src are not written (K > max_src is the capacity case)
 *   ws         workspace of ipp_detect_label_workspace_size() bytes
 */
size_t ipp_detect_label_workspace_size(int64_t W, int64_t H);
int ipp_detect_label(const float* sub, int64_t W, int64_t H, int64_t pitch,
                     const float* mesh_rms, const ipp_bg_params* bp, const ipp_det_params* dp,
                     const uint32_t* mask_in, int32_t* labels, int32_t* n_src_dev,
                     int32_t max_src, const ipp_src_stats* stats, void* ws, size_t ws_bytes,
                     void* stream);

/* -------------------------------------------------------------- per source */
/*
 * ipp_centroid -- windowed centroid (paper-silent reading of the positions of
 * Sec. 2.2.5): Gaussian window sigma_w = fwhm_win / 2.35482 over the pixels with
 * centres within 4 sigma_w of the current position and inside the frame;
 * x += 2 sum(w f (x_i - x)) / sum(w f) (same for y) until the squared step is
 * below tol2 or max_iter updates; a non-positive weighted sum returns the seed.
 * Processes min(*n_src_dev, max_src) sources.
 *   x0, y0     seeds (e.g. the barycentres of ipp_detect_label)
 *   x, y, niter, flags   device outputs per source (niter nullable)
 */
int ipp_centroid(const float* sub, int64_t W, int64_t H, int64_t pitch,
                 const int32_t* n_src_dev, int32_t max_src, const float* x0, const float* y0,
                 const ipp_cen_params* p, float* x, float* y, int32_t* niter, int32_t* flags,
                 void* stream);

/*
 * ipp_aperture_phot -- aperture photometry (Sec. 2.2.5) with a local sky
 * annulus (paper-silent reading): weights are the exact areas of the pixel /
 * disk overlaps, sky is the median (Eq. 1) of the pixels whose centres satisfy
 * r_in <= d < r_out, flux = sum(w f) - sky sum(w), area = sum(w).
 *   flux, sky, area, n_ann, flags   device outputs per source (nullable except flux)
 */
int ipp_aperture_phot(const float* sub, int64_t W, int64_t H, int64_t pitch,
                      const int32_t* n_src_dev, int32_t max_src, const float* x, const float* y,
                      const ipp_phot_params* p, float* flux, float* sky, float* area,
                      int32_t* n_ann, int32_t* flags, void* stream);

/*
 * ipp_deblend -- deblending of the candidates of ipp_detect_label (Sec. 2.2.5:
 * multi-level thresholds between each candidate's threshold and its peak, a
 * tree of the sub-components found at each level, traversed bottom-up and
 * pruned on intensity).  Reading:
 *   levels  L_i = T (P/T)^(i/N), i = 1..N-1 (FP64), T and P the candidate's
 *           lowest and highest pixel; T <= 0 or P <= T keeps it whole;
 *   tree    nodes of level i are the 8-connected components of the candidate's
 *           pixels above L_i; level 0 is the candidate;
 *   objects from the top level down: a node with two or more children holding
 *           at least mincont of the candidate's flux passes on their objects,
 *           with one such child it passes on that child's objects when there
 *           are two or more, otherwise it is one object whose core is its pixels;
 *   pixels  outside every core go to the object whose elliptical Gaussian (core
 *           flux, barycentre and second moments; 1/12 added to x2 and y2 when
 *           x2 y2 - xy^2 < 1/144) is largest there, ties to the earlier core;
 *   numbers objects of candidate 1 first, then of candidate 2, ...; within a
 *           candidate by the raster order of the object's first pixel.
 * Processes min(*n_src_dev, max_src) candidates.
 *   labels      device int32 label map of ipp_detect_label (pitch W)
 *   stats       host struct of device arrays (xmin, xmax, ymin, ymax, area read)
 *   out_labels  device int32[W*H] (pitch W): the deblended map, 0 = background
 *   n_out_dev   device int32[1]: the number of objects
 *   ws          device workspace of ipp_deblend_workspace_size(W, H, max_src)
 *               bytes (112 B per frame pixel), 256-byte aligned
 * Errors: INVALID_ARG for NULL inputs, nthresh outside 2..256, mincont outside
 * 0..1, a small workspace or a frame of 2^31 pixels or more.
 */
size_t ipp_deblend_workspace_size(int64_t W, int64_t H, int32_t max_src);
int ipp_deblend(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t pitch,
                const int32_t* n_src_dev, int32_t max_src, const ipp_src_stats* stats,
                const ipp_deblend_params* p, int32_t* out_labels, int32_t* n_out_dev, void* ws,
                size_t ws_bytes, void* stream);

/*
 * ipp_clean -- cleaning of the deblended objects (Sec. 2.2.5: an object that
 * does not stand out from its neighbours is merged into them).  Reading, after
 * SExtractor's cleaning:
 *   per object, from its pixels of sub: the peak (largest value, first in
 *     raster order on ties); the barycentre and second moments weighted by the
 *     positive values (1/12 added to x2 and y2 when x2 y2 - xy^2 < 1/144; no
 *     positive pixel: the unweighted centre, x2 = y2 = 1/12, xy = 0);
 *   model of object j: peak_j (1 + r^2 / a^2)^-beta about its barycentre,
 *     r^2 = (y2 dx^2 - 2 xy dx dy + x2 dy^2) / (x2 y2 - xy^2),
 *     a^2 = 2 ln 2 / (2^(1/beta) - 1);
 *   object i merges when its peak less the sum of the models of every brighter
 *     object (larger peak; equal peaks: smaller label) at its peak pixel is
 *     below the detection threshold there; the target is
 *     the brighter object whose model is largest there (ties: smaller label),
 *     merges followed to a kept object; kept objects are renumbered 1.. in label
 *     order (a label with no pixel is no object and takes no number).
 * The sums over pixels are exact (integer accumulators), so the result does not
 * depend on the order of the atomics; the models are FP32, summed with a
 * compensated (two-sum) accumulator in a fixed order (brightest first), so the
 * result is the same from run to run.
 * Processes labels 1..min(*n_obj_dev, max_obj); other labels map to 0.
 *   labels      device int32 map (pitch W), e.g. the output of ipp_deblend
 *   thr_map     nullable device float threshold map (pitch W); when NULL the
 *               threshold is max(dp->k rms(x, y), dp->thresh_abs), rms the Keys
 *               interpolation of mesh_rms on the grid of bp (the detection
 *               threshold of ipp_detect_label), or dp->thresh_abs when mesh_rms
 *               is NULL too
 *   beta        Moffat index of the model, > 0 [1]
 *   out_labels  device int32[W*H] (pitch W): the cleaned map, 0 = background
 *   n_out_dev   device int32[1]: the number of kept objects
 *   ws          device workspace of ipp_clean_workspace_size(max_obj) bytes
 *               (about 200 + 16 P / 4096 B per object, P the power of two at
 *               or above max(max_obj, 2048)), 256-byte aligned
 * Sizes: frames below 2^31 pixels, narrower than 65536 pixels, objects below
 * 2^24 pixels (range of the exact sums).
 * Errors: INVALID_ARG for NULL inputs, beta <= 0, max_obj above 2^24, a small
 * or misaligned workspace, or sizes out of range.
 */
size_t ipp_clean_workspace_size(int32_t max_obj);
int ipp_clean(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t pitch,
              const int32_t* n_obj_dev, int32_t max_obj, const float* thr_map, const float* mesh_rms,
              const ipp_bg_params* bp, const ipp_det_params* dp, float beta, int32_t* out_labels,
              int32_t* n_out_dev, void* ws, size_t ws_bytes, void* stream);

/*
 * ipp_auto_phot -- auto (Kron) photometry; Sec. 2.2.5 lists auto photometry
 * beside aperture and isophotal photometry without defining it (reading after
 * Kron's first-moment radius and SExtractor's automatic aperture):
 *   1. second moments of sub over the source's isophotal footprint (pixels with
 *      labels == k+1 inside its bounding box) about (xbar, ybar):
 *      x2 = sum f dx^2 / sum f, y2, xy likewise; 1/12 is added to x2 and y2
 *      when x2 y2 - xy^2 < 1/144; a footprint with sum f <= 0 takes
 *      x2 = y2 = 1/12, xy = 0 and KRON_BAD;
 *   2. elliptical radius r^2 = (y2 dx^2 - 2 xy dx dy + x2 dy^2) / (x2 y2 - xy^2);
 *      Kron radius r1 = sum r f / sum f over in-frame pixels with r <= r_kmax
 *      (neighbours not masked); sums not positive give r1 = 0 and KRON_BAD;
 *   3. flux = sum f over in-frame pixel centres with r <= max(k_kron r1, r_min),
 *      area = their number; EDGE when such a pixel centre lies in the one-pixel
 *      border around the frame.
 * Frames must hold fewer than 2^31 pixels (32-bit box coordinates).
 * Processes min(*n_src_dev, max_src) sources; the isophotal flux is
 * stats->flux of ipp_detect_label.
 *   labels     device int32 label map of ipp_detect_label (pitch W)
 *   stats      host struct of device arrays (xmin, xmax, ymin, ymax, xbar, ybar read)
 *   flux       device float[max_src] (required); area, kron (r1) nullable;
 *   shape      nullable device float[3*max_src]: x2, y2, xy per source;
 *   flags      nullable device int32[max_src]: EDGE, KRON_BAD
 * Errors: INVALID_ARG for NULL inputs, k_kron <= 0, r_min < 0 or r_kmax <= 0.
 */
int ipp_auto_phot(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t pitch,
                  const int32_t* n_src_dev, int32_t max_src, const ipp_src_stats* stats,
                  const ipp_auto_params* p, float* flux, float* area, float* kron, float* shape,
                  int32_t* flags, void* stream);

/*
 * ipp_gray_transform -- value-to-gray map of Sec. 2.2.6 (the display functions
 * it lists: linear, logarithmic, power, exponential).  With
 * xn = clip((x - lo) / (hi - lo), 0, 1) per pixel:
 *   IPP_GRAY_LINEAR  xn
 *   IPP_GRAY_LOG     log10(a xn + 1) / log10(a + 1)      (a > 0)
 *   IPP_GRAY_POWER   xn^a                                (a > 0)
 *   IPP_GRAY_EXP     (a^xn - 1) / (a - 1)                (a > 0, a != 1)
 * Non-finite pixels map to 0.  Arithmetic is FP32 (xn from (x - lo) times the
 * rounded 1 / (hi - lo)); the result is within a few 1e-7 of the FP64 value.
 *   img     device float, rows of `pitch` elements
 *   out     device float, rows of `out_pitch` (>= W); must not alias img
 *   lo, hi  finite, lo < hi
 * Errors: INVALID_ARG for NULL pointers, bad sizes or pitches, an unknown kind,
 * lo >= hi or an `a` outside the ranges above, or out == img.
 */
int ipp_gray_transform(const float* img, int64_t W, int64_t H, int64_t pitch, int32_t kind, float lo, float hi,
                       float a, float* out, int64_t out_pitch, void* stream);

/*
 * ipp_hist_equalize -- histogram equalisation of Sec. 2.2.6.  Over the finite
 * pixels, min and max give nbins bins of width (max - min) / nbins; pixel x falls
 * in bin floor((x - min) s), s = nbins / (max - min) (FP32, clamped to
 * [0, nbins - 1]); C(b) is the fraction of finite pixels in bins 0..b.  The gray
 * value is C interpolated linearly between bin centres at t = (x - min) s - 1/2:
 * C(0) for t <= 0, C(nbins - 1) for t >= nbins - 1.  Non-finite pixels, and every
 * pixel of a frame with no finite value or max == min, map to 0.
 *   nbins   2 <= nbins <= 16384
 *   out     device float, rows of `out_pitch` (>= W); must not alias img
 *   ws      device workspace of ipp_hist_equalize_workspace_size(nbins) bytes,
 *           256-byte aligned; after the call it holds (from byte 256) the counts
 *           uint32[nbins] and, at the next 256-byte boundary, C as float[nbins]
 *           (followed by the pairs (C(b), C(b + 1) - C(b)) the apply pass reads)
 * Four launches (min/max, histogram, cumulative sum, apply) and one memset on
 * `stream`; no host synchronisation.
 * Errors: INVALID_ARG for NULL pointers, bad sizes or pitches, nbins out of range,
 * a misaligned or short workspace, or out == img.
 */
size_t ipp_hist_equalize_workspace_size(int32_t nbins);
int ipp_hist_equalize(const float* img, int64_t W, int64_t H, int64_t pitch, int32_t nbins, float* out,
                      int64_t out_pitch, void* ws, size_t ws_bytes, void* stream);

/*
 * ipp_wcs_map -- coordinate mapping of Sec. 2.2.3: source pixel -> sky -> target
 * pixel, through Eq. 5 (SIP, on the offsets u = x - CRPIX1, v = y - CRPIX2 of
 * the FITS pixel position), Eq. 6 (CD) and Eq. 7 (gnomonic deprojection about
 * the source's CRVAL), then the inverse chain of the target: gnomonic projection
 * about its CRVAL, CD^-1, and the inverse of its SIP polynomial by Newton's
 * method (at most 50 steps, until the step is below 1e-12 px).  FP64.
 * Node (j, i) of the grid is source pixel (j step, i step), 0 <= j < nx =
 * (W - 1) / step + 1, 0 <= i < ny = (H - 1) / step + 1; step 1 maps every pixel
 * (the paper's thread per pixel; FP64-bound, about 300 FP64 operations a node).
 *   x_out, y_out  device double[ny * nx], row-major: the 0-based target pixel
 *                 position of each node; NaN where the sky point is 90 degrees or
 *                 more from the target's tangent point or Newton does not converge
 * Errors: INVALID_ARG for NULL pointers, W, H or step < 1, a SIP order outside
 * 0..5, non-finite WCS values or a singular target CD.
 */
int ipp_wcs_map(const ipp_wcs* src, const ipp_wcs* tgt, int64_t W, int64_t H, int32_t step, double* x_out,
                double* y_out, void* stream);

/*
 * ipp_affine_fit -- the partial affine estimate of Sec. 2.2.3 (rotation, one
 * scale and a translation, the model of OpenCV's estimateAffinePartial2D that
 * the paper uses), as the least-squares similarity of point pairs
 * (x, y) -> (xt, yt) in closed form about the centroids: a = s cos t and
 * b = s sin t are the centred cross sums over the centred source norm.  No
 * outlier rejection (pairs from a WCS mapping have no outliers); pairs with a
 * non-finite member are skipped.  FP64, deterministic (fixed reduction order).
 *   x, y      device double[n], or both NULL: then pair k's source point is the
 *             grid node ((k % grid_nx) grid_step, (k / grid_nx) grid_step) of
 *             ipp_wcs_map
 *   xt, yt    device double[n]
 *   M_out     device double[12]: M = [a -b tx; b a ty] (source -> target), then
 *             its inverse (target -> source), each 2 x 3 row-major
 *   status_dev nullable device int32: IPP_OK, or IPP_ERR_DEGENERATE (fewer than
 *             two distinct usable pairs; M_out is then NaN)
 *   ws        device workspace of ipp_affine_fit_workspace_size() bytes,
 *             8-byte aligned
 * Errors: INVALID_ARG for NULL pointers, n < 0, or grid_nx / grid_step < 1 when
 * x, y are NULL.
 */
size_t ipp_affine_fit_workspace_size(void);
int ipp_affine_fit(const double* x, const double* y, const double* xt, const double* yt, int64_t n,
                   int64_t grid_nx, int32_t grid_step, double* M_out, int32_t* status_dev, void* ws,
                   size_t ws_bytes, void* stream);

/*
 * ipp_reproject_affine -- image reprojection of Sec. 2.2.3: output pixel (j, i)
 * of a Wo x Ho frame is the source value at (x, y) = Minv (j, i, 1) by bilinear
 * interpolation between the four surrounding pixel centres.  Defined for
 * 0 <= x <= W - 1 and 0 <= y <= H - 1 (on the last column or row the pair
 * beyond has weight 0 and is not read); elsewhere, or when a neighbour with
 * non-zero weight is not finite, the output is `fill`.  The position is formed
 * in double-float arithmetic once per 128 output pixels and offset in FP32
 * (error near 1e-5 px); the interpolation is FP32.  Wo, Ho < 2^24.
 *   src       device float, rows of `pitch` elements
 *   Minv_dev  device double[6] (2 x 3 row-major), e.g. M_out + 6 of ipp_affine_fit,
 *             read by the kernel: no host synchronisation between fit and warp
 *   out       device float, rows of `out_pitch` (>= Wo); must not alias src
 * Errors: INVALID_ARG for NULL pointers, bad sizes or pitches, Wo or Ho >= 2^24,
 * or out == src.
 */
int ipp_reproject_affine(const float* src, int64_t W, int64_t H, int64_t pitch, const double* Minv_dev, int64_t Wo,
                         int64_t Ho, float fill, float* out, int64_t out_pitch, void* stream);

/*
 * ipp_zscale -- display limits of Sec. 2.2.6 (SAOimage's zscale; reading after
 * the published IRAF algorithm).  Samples: up to n_samples pixels at flat
 * (row-major) indices k stride, stride = max(1, W H / n_samples), non-finite
 * ones dropped, sorted: s_0 <= ... <= s_{npix-1}; c = (npix - 1) / 2; median =
 * s_c (npix odd) or (s_c + s_{c+1}) / 2.  Up to max_iter passes, stopping when
 * the good count stops falling or drops below minpix = max(5, npix / 2): the
 * least-squares line of s_k against k - c over the good samples; residuals of
 * every sample; rejection where |residual| > krej x their population standard
 * deviation over the good samples; a sample is good when no rejected sample
 * lies within h = max(1, npix / 100) / 2 of it.  Limits: with at least minpix
 * good samples z1 = max(s_0, median - (c - 1) slope / contrast), z2 =
 * min(s_{npix-1}, median + (npix - c) slope / contrast), else (s_0, s_{npix-1}).
 * FP64 fit; one block of 1024 threads (the samples sorted in shared memory).
 *   z_out       device double[2]: z1, z2 (NaN when no sample is finite)
 *   counts_out  nullable device int32[2]: samples used, good samples at the end
 * Errors: INVALID_ARG for NULL pointers, bad sizes or pitches, or parameters
 * outside the ranges above.
 */
int ipp_zscale(const float* img, int64_t W, int64_t H, int64_t pitch, const ipp_zscale_params* p, double* z_out,
               int32_t* counts_out, void* stream);

/*
 * ipp_sub_apply -- the convolution and difference of image subtraction
 * (Sec. 2.2.4, HOTPANTS-style; Eqs. 8-10), the paper's dominant cost.  Given the
 * fitted coefficients, the kernel of each (2 hw + 1)^2 output tile is
 *   K(u, v) = sum_n a_n(xc, yc) K_n(u, v),  a_n = sum_s c[n * ns + s] P_s (Eq. 8),
 *   K_n(u, v) = exp(-(u^2 + v^2) / (2 sig_k^2)) u^i v^j  (Eq. 9; Gaussian k outer,
 *   then i, then j, i + j <= deg_k; u and v the offsets in x and y),
 * at the tile's centre (xc, yc); P_s are xs^p ys^q (p outer, p + q <= sord) of
 * xs = 2x / (W - 1) - 1, ys = 2y / (H - 1) - 1.  The difference (the residual of
 * Eq. 10, read as I + B = R (x) K) is
 *   D(x, y) = I(x, y) + B(x, y) - sum_{u,v} K(u, v) R(x - u, y - v),
 *   B = sum_b c[nb * ns + b] P_b(x, y) (order bord; none when bord = -1),
 * NaN where the kernel's support leaves the frame.  FP32 arithmetic.
 *   I, R      device float, W x H, rows of `pitch` elements (the same for both)
 *   coef      device float[nb * ns + nb_bg]: kernel coefficients, then background
 *   sig, deg  host arrays of nk (1..8) Gaussian widths (> 0) and degrees (0..8);
 *             nb = sum (deg_k + 1)(deg_k + 2) / 2 <= 64
 *   hw        kernel half width: 4, 6, 8, 10 or 12 (NOT_SUPPORTED otherwise)
 *   D         device float, rows of `out_pitch` (>= W); must not alias I or R
 *   ws        device workspace of ipp_sub_apply_workspace_size() bytes (the basis)
 * Errors: INVALID_ARG for NULL pointers, bad sizes, orders (sord 0..4, bord
 * -1..4) or basis descriptions; NOT_SUPPORTED for another hw.
 */
size_t ipp_sub_apply_workspace_size(int32_t hw, int32_t nk, const int32_t* deg);
int ipp_sub_apply(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int32_t hw, int32_t nk,
                  const float* sig, const int32_t* deg, const float* coef, int32_t sord, int32_t bord, float* D,
                  int64_t out_pitch, void* ws, size_t ws_bytes, void* stream);

/*
 * The fit of image subtraction (Sec. 2.2.4, Eqs. 8-10, HOTPANTS-style readings;
 * the model and basis as ipp_sub_apply's, sig in FP64 here):
 *   ipp_sub_stamps  candidate stamps: the frame is cut into nsx x nsy regions
 *     (region (sx, sy) spans x in [sx W / nsx, (sx + 1) W / nsx), likewise y); in
 *     each, med and MAD are the median (Eq. 1's mean of the middle pair for an
 *     even count) of the template's finite pixels and of their FP64 |R - med|;
 *     the candidate is the brightest template pixel (first in raster order among
 *     equals) whose footprint (2 fh + 1)^2 in I and support (2 (fh + hw) + 1)^2
 *     in R lie inside the frame and are finite, kept when R > med + nsig 1.4826
 *     MAD (FP64).  Exact: the same candidates as a sequential evaluation.
 *     cx, cy: device int32[nsx * nsy], the candidates in region order (row-major
 *     over the regions); n_dev: device int32[1], their count.
 *   ipp_sub_normal  the normal equations of the unweighted least-squares fit over
 *     every footprint pixel of candidates 0 .. min(*n_dev, max_c) - 1: unknowns
 *     c[n * ns + s] (kernel) then d[b] (background), design row of a pixel
 *     [C_n P_s(candidate centre)] then [-P_b(pixel)], C_n = R (x) K_n, target I.
 *     FP64 throughout (the scaled normal matrix has condition numbers ~1e11, so
 *     FP32 entries would move the fitted model by percents); the convolutions
 *     use the basis' separability.  A candidate whose support leaves the frame
 *     contributes nothing.  AtA: device double[np * np] (full, symmetric), Atb:
 *     device double[np], np = nb * ns + nb_bg.
 *   ipp_sub_solve   Cholesky solve of AtA x = Atb in FP64, in place (AtA takes
 *     L, Atb the solution); coef64 (double) and coef (float, the input of
 *     ipp_sub_apply) receive the solution when not NULL; *status_dev = 0, or 1
 *     when a pivot is not positive (no solution written).
 *   ipp_sub_fit     the three in sequence on the frame's own candidates;
 *     cx, cy, n_dev nullable (else the candidates are reported there).
 * Workspace: ipp_sub_fit_workspace_size(max_c, nreg, ...) bytes, 256-byte
 * aligned: max_c candidates (nsx * nsy for ipp_sub_fit, 0 for ipp_sub_stamps),
 * nreg regions (nsx * nsy for ipp_sub_stamps and ipp_sub_fit, 0 for
 * ipp_sub_normal).  Limits: nk 1..8, deg 0..8, sord 0..4, bord -1..4, frames
 * below 2^31 pixels, at most 65536 regions; NOT_SUPPORTED when a footprint and
 * basis need more shared memory than one block has (fh = hw = 10 with the
 * 49-function basis takes 187 KB).  Errors: INVALID_ARG for NULL pointers, a
 * basis or orders out of range, non-finite sig or nsig, or a small or
 * misaligned workspace, all before anything is enqueued; the workspace query
 * returns 0 for arguments out of range.  A singular normal matrix is not an
 * error of the call: it is *status_dev = 1 on the device.
 */
size_t ipp_sub_fit_workspace_size(int32_t max_c, int32_t nreg, int32_t hw, int32_t fh, int32_t nk, const int32_t* deg,
                                  int32_t sord, int32_t bord);
int ipp_sub_stamps(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int32_t nsx, int32_t nsy,
                   int32_t hw, int32_t fh, double nsig, int32_t* cx, int32_t* cy, int32_t* n_dev, void* ws,
                   size_t ws_bytes, void* stream);
int ipp_sub_normal(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, const int32_t* cx,
                   const int32_t* cy, const int32_t* n_dev, int32_t max_c, int32_t hw, int32_t fh, int32_t nk,
                   const double* sig, const int32_t* deg, int32_t sord, int32_t bord, double* AtA, double* Atb,
                   void* ws, size_t ws_bytes, void* stream);
int ipp_sub_solve(double* AtA, double* Atb, int32_t np, double* coef64, float* coef, int32_t* status_dev,
                  void* stream);
int ipp_sub_fit(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int32_t nsx, int32_t nsy,
                double nsig, int32_t hw, int32_t fh, int32_t nk, const double* sig, const int32_t* deg, int32_t sord,
                int32_t bord, double* coef64, float* coef, int32_t* cx, int32_t* cy, int32_t* n_dev,
                int32_t* status_dev, void* ws, size_t ws_bytes, void* stream);

/*
 * ipp_stamp_cut -- S x S stamps of the subtracted frame around each source, the
 * input of the PSF fit (the paper fits no PSF; this cut is part of that
 * paper-silent reading of Sec. 2.2.5's photometry).  For source s < min(*n_src_dev,
 * max_src) the stamp origin is ox = floor(x[s] + 1/2) - S/2, oy = floor(y[s] + 1/2)
 * - S/2 (round half up, S odd, integer division), and stamp pixel (r, c) is frame
 * pixel (row oy + r, column ox + c).  Stamp pixels outside the frame are 0 with
 * weight 0 and the source gets IPP_FLAG_EDGE; inside pixels have weight 1.  A
 * position that is not finite or lies more than 2^30 px outside the frame gives a
 * stamp of zeros with weight 0, origin (0, 0) and IPP_FLAG_EDGE.
 *   S        odd, 3 <= S <= 63
 *   stamps   device float[max_src * S * S], source-major, rows of S (only the first
 *            n stamps are written)
 *   weights  nullable device float[max_src * S * S]
 *   origin   nullable device int32[max_src * 2]: (ox, oy) per source
 *   flags    nullable device int32[max_src]: written (0 or IPP_FLAG_EDGE), not or-ed
 */
int ipp_stamp_cut(const float* sub, int64_t W, int64_t H, int64_t pitch,
                  const int32_t* n_src_dev, int32_t max_src, const float* x, const float* y,
                  int32_t S, float* stamps, float* weights, int32_t* origin, int32_t* flags,
                  void* stream);

/* ------------------------------------------------------------- fused frame */
/*
 * ipp_extract -- the catalog path of one frame in one call: bg_estimate,
 * bg_subtract fused with the threshold and the per-tile labeling, label merge,
 * centroid and aperture photometry.  Outputs as in the individual calls; the
 * positions used for photometry are the windowed centroids.
 */
typedef struct {
    float* mesh_bkg; float* mesh_rms;     /* [ny*nx] */
    float* sub;                           /* [H*W] background-subtracted frame, pitch W */
    int32_t* labels;                      /* [H*W] */
    int32_t* n_src_dev;                   /* [1] */
    ipp_src_stats stats;                  /* [max_src] */
    float* x; float* y; int32_t* cen_flags;              /* [max_src] */
    float* flux; float* sky; float* area; int32_t* n_ann; int32_t* phot_flags; /* [max_src] */
    int32_t* status_dev;                  /* [1] nullable */
} ipp_catalog_out;

size_t ipp_extract_workspace_size(int64_t W, int64_t H, const ipp_bg_params* bp);
int ipp_extract(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                const ipp_calib* cal, const ipp_bg_params* bp, const ipp_det_params* dp,
                const ipp_cen_params* cp, const ipp_phot_params* pp, int32_t max_src,
                const ipp_catalog_out* out, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- batches */
/*
 * The catalog path over a batch of independent frames of mixed sizes (the
 * batched form of ipp_extract; the paper runs every frame through the same
 * steps, Sec. 2.1).  A runner spreads the frames over `lanes` CUDA streams of
 * its own, forked from the caller's stream and joined back to it, assigning
 * each frame to the least-loaded lane by pixel count (largest frames first),
 * so that the small kernels of one frame overlap the large ones of another.
 * ipp_batch_capture records a whole batch as one CUDA graph; ipp_batch_launch
 * replays it with a single call (inputs are read from, and outputs written to,
 * the pointers given at capture).
 *
 *   ipp_frame_desc   one frame: device image, type, size, pitch, optional
 *                    calibration (host struct, read during the call) and the
 *                    frame's catalog outputs (as for ipp_extract; sub has pitch W)
 *   lanes            1..IPP_BATCH_MAX_LANES streams
 *   ws               device workspace of ipp_batch_workspace_size() bytes for the
 *                    largest frame of the batch; lanes do not share scratch
 * Errors: IPP_ERR_INVALID_ARG for a bad frame (index in ipp_last_error_detail())
 * before anything is enqueued; otherwise as ipp_extract.  The runner holds CUDA
 * streams, events and at most one graph; ipp_batch_destroy releases them.
 */
#define IPP_BATCH_MAX_LANES 8

typedef struct {
    const void* img;
    int32_t dtype;
    int32_t reserved;
    int64_t W, H, pitch;
    const ipp_calib* cal;       /* host pointer, nullable */
    ipp_catalog_out out;
} ipp_frame_desc;

typedef struct ipp_batch_s* ipp_batch;

size_t ipp_batch_workspace_size(int64_t max_W, int64_t max_H, const ipp_bg_params* bp, int32_t lanes);
int ipp_batch_create(int32_t lanes, ipp_batch* out);
int ipp_batch_destroy(ipp_batch b);
int ipp_batch_extract(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                      const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                      int32_t max_src, void* ws, size_t ws_bytes, void* stream);
int ipp_batch_capture(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                      const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                      int32_t max_src, void* ws, size_t ws_bytes, void* stream);
int ipp_batch_launch(ipp_batch b, void* stream);

/*
 * The table form of the batch: one launch per stage for all frames.  The jobs
 * of every frame (the same as ipp_extract's) are packed into a device table at
 * the head of ws; each stage is a single launch over the frames' blocks, a block
 * finding its frame by binary search over the frames' first blocks, and runs the
 * per-frame kernel body -- so the outputs equal ipp_extract's bit for bit.  The
 * frames are split into one group per lane of the runner (largest first, to the
 * least-loaded lane); each group is a table of its own whose ~17 launches go to
 * the lane's stream, so the stages of different groups overlap (a memory-bound
 * stage of one group beside a compute-bound one of another).  Frames keep
 * separate scratch (ws holds them one after another).
 *   ipp_batch_table_workspace_size  bytes of ws for these frames (the table plus
 *                                   each frame's ipp_extract workspace)
 *   ipp_batch_table_extract         enqueues the batch on `stream`; the table is
 *                                   uploaded from the runner's pinned staging
 *                                   buffer unless it equals the one uploaded to
 *                                   this ws last (same frames and parameters)
 *   ipp_batch_table_capture         uploads the table, then records the stages as
 *                                   the runner's graph (ipp_batch_launch replays
 *                                   it; the graph reads the table in ws, so ws is
 *                                   not to be reused for another batch meanwhile)
 * Limits: 1..1024 frames; the windowed centroid's box at most 15 px (fwhm_win
 * up to ~3.5 px), the Keys reading (interp = IPP_INTERP_KEYS) -- NOT_SUPPORTED
 * otherwise, where the stream form applies.
 * Errors: INVALID_ARG for a bad frame (its index in ipp_last_error_detail()), a
 * NULL or misaligned workspace or one too small for these frames, before
 * anything is enqueued; otherwise as ipp_extract.  The workspace query returns
 * 0 for a bad frame list.
 */
size_t ipp_batch_table_workspace_size(const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp);
int ipp_batch_table_extract(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                            const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                            int32_t max_src, void* ws, size_t ws_bytes, void* stream);
int ipp_batch_table_capture(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                            const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                            int32_t max_src, void* ws, size_t ws_bytes, void* stream);

/*
 * ipp_batch_autotune -- times ipp_batch_extract on this batch for 1, 2, 4 and 8
 * lanes (two runs each after a warm-up, CUDA events on `stream`), and returns
 * the fastest lane count in *best_lanes and the times in ms_per_lanes[4]
 * (nullable).  Synchronises `stream`.  ws must be sized for 8 lanes.
 */
int ipp_batch_autotune(const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                       const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                       int32_t max_src, void* ws, size_t ws_bytes, void* stream, int32_t* best_lanes,
                       float* ms_per_lanes);

/* ---------------------------------------------------------------- PSF fit */
/*
 * ipp_psf_fit -- batched Levenberg-Marquardt fit of an elliptical Moffat or
 * Gaussian PSF (paper-silent) to N stamps of S x S pixels.  Parameters per stamp:
 * (x0, y0, F, sky, sx, sy, theta); model point-sampled at pixel centres
 * (0..S-1):  u = cos(t) dx + sin(t) dy, v = -sin(t) dx + cos(t) dy,
 * q = u^2/sx^2 + v^2/sy^2, Moffat F (beta-1)/(pi sx sy) (1+q)^-beta + sky,
 * Gaussian F/(2 pi sx sy) exp(-q/2) + sky.  Model, Jacobian and J'WJ in FP32;
 * the 7x7 damped normal equations solved in FP64 (LDL' factorisation).  One trial per
 * iteration: accepted when chi^2 drops (lambda /= 10), else lambda *= 10; widths
 * must stay above 0.05.  Converged, before a trial, when the Gauss-Newton
 * decrease g'(J'WJ)^-1 g (g = J'W r) is at most 1e-10 chi^2 + 1e-12 sum w
 * (m - sky)^2 -- each parameter then lies within ~1.5e-4 standard errors of the
 * optimum, and the second term covers what FP32 rounding of the model can
 * fake -- or when lambda exceeds 1e10 (no step lowers chi^2).  Otherwise
 * FIT_MAXITER after max_iter trials.  Result canonicalised to
 * sx >= sy and theta in [-pi/2, pi/2).
 *   stamps   device float[N*S*S]; weights nullable (same shape)
 *   init     nullable device float[N*7]; NULL = stamp centre, border-median sky,
 *            sum above sky, sx = 1.6, sy = 1.4, theta = 0
 *   params   device float[N*7]; chi2 float[N]; iters, flags int32[N] (nullable)
 */
int ipp_psf_fit(const float* stamps, int64_t N, int32_t S, const float* weights,
                const float* init, const ipp_fit_params* p, float* params, float* chi2,
                int32_t* iters, int32_t* flags, void* stream);

/*
 * ipp_psf_fit_dev -- ipp_psf_fit with the stamp count in device memory:
 * min(*n_dev, n_max) stamps are fitted (n_dev typically the detection count
 * that ipp_stamp_cut filled), so no host copy of the count is needed between
 * detection and the fit.  Grid and lanes per stamp are sized for n_max;
 * outputs beyond the count are not written.  Errors as ipp_psf_fit; n_dev must
 * not be NULL.
 */
int ipp_psf_fit_dev(const float* stamps, const int32_t* n_dev, int64_t n_max, int32_t S, const float* weights,
                    const float* init, const ipp_fit_params* p, float* params, float* chi2, int32_t* iters,
                    int32_t* flags, void* stream);

/* Model images m[N*S*S] of params[N*7] (forward of the differentiable model). */
int ipp_psf_model_fwd(const float* params, int64_t N, int32_t S, const ipp_fit_params* p,
                      float* model, void* stream);

/* Adjoint: grad_params[n][k] = sum_pixels grad_model[n][pix] * dm/dparam_k. */
int ipp_psf_model_adj(const float* params, int64_t N, int32_t S, const ipp_fit_params* p,
                      const float* grad_model, float* grad_params, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IPP_H */
