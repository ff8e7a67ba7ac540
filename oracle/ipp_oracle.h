/*
 * ipp_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU oracle of the per-frame catalog path of
 * "Image Pre-Processing Framework for Time-Domain Astronomy in the Artificial
 * Intelligence Era" (Cao, Jia et al., arXiv 2502.10783).  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the CUDA
 * library never does, and this file shares nothing with it.
 *
 * Every function follows one step of the paper (section / equation named at the
 * definition) or, where the paper is silent, the stated reading.  Arithmetic is
 * FP64 throughout; inputs are the same float32 arrays the GPU path consumes.
 * Build: gcc -O2 -std=c11 -ffp-contract=off (no fused multiply-add, so that
 * the distance tests below are the exact IEEE expressions documented here).
 */
#ifndef IPP_ORACLE_H
#define IPP_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_INVALID_ARG 1
#define ORC_NO_VALID_MESH 4

/* per-source flag bits (same meaning as the library's; values restated here) */
#define ORC_FLAG_EDGE 1
#define ORC_FLAG_WIN_NOT_CONVERGED 2
#define ORC_FLAG_ANN_FEW 4
#define ORC_FLAG_FIT_MAXITER 8
#define ORC_FLAG_FIT_SINGULAR 16
#define ORC_FLAG_FIT_BAD_SIGMA 32
#define ORC_FLAG_KRON_BAD 64

/* background estimators, Sec. 2.2.2 Eqs. 1-4 */
#define ORC_EST_SIGMA 0   /* Eq. 3: 2.5 median - 1.5 mean (default) */
#define ORC_EST_MEDIAN 1  /* Eq. 1 */
#define ORC_EST_MEAN 2    /* Eq. 2 */
#define ORC_EST_FACTORS 3 /* Eq. 4 read as median_factor*median - mean_factor*mean */

typedef struct {
    int32_t mesh_w, mesh_h;     /* mesh (sub-region) size, Sec. 2.2.2: default 64 x 64 */
    int32_t filter_w, filter_h; /* median-filter window on the mesh grid (odd) */
    int32_t maxiters;           /* clip iterations (reading: 10) */
    int32_t min_valid;          /* at least 100 pixels per mesh, Sec. 2.2.2 */
    int32_t estimator;          /* ORC_EST_* */
    int32_t pad_;
    double nsigma;              /* clip half-width in sigma (3) */
    double median_factor, mean_factor; /* Eq. 4 weights */
} orc_bg_params;

int orc_calibrate(const uint16_t* raw, int64_t W, int64_t H, int64_t pitch,
                  const float* bias_map, double bias, const float* flat, float* out);

int orc_mesh_stats(const float* img, int64_t W, int64_t H, int64_t pitch,
                   const uint8_t* mask, const orc_bg_params* p,
                   double* raw_bkg, double* raw_rms, int32_t* valid,
                   int32_t* niter, double* margin);

int orc_mesh_fill_filter(const double* raw_bkg, const double* raw_rms,
                         const int32_t* valid, int64_t nx, int64_t ny,
                         int32_t fw, int32_t fh, double* bkg, double* rms);

double orc_keys_weight(double s);

int orc_interp_map(const float* mesh, int64_t nx, int64_t ny, int32_t mesh_w,
                   int32_t mesh_h, int64_t W, int64_t H, double* out);
/* natural-spline variant of the background map (tensor-product natural cubic
 * spline through the mesh nodes, linear beyond the end nodes) */
int orc_spline_map(const float* mesh, int64_t nx, int64_t ny, int32_t mesh_w, int32_t mesh_h, int64_t W, int64_t H,
                   double* out);
int orc_spline_nodes(const float* mesh, int64_t nx, int64_t ny, double* Mx, double* My, double* Mxy);

int orc_bg_subtract(const float* img, int64_t W, int64_t H, int64_t pitch,
                    const float* mesh_bkg, int64_t nx, int64_t ny,
                    int32_t mesh_w, int32_t mesh_h, float* sub, float* bkg_map);

int orc_threshold(const float* sub, int64_t W, int64_t H, const float* mesh_rms,
                  int64_t nx, int64_t ny, int32_t mesh_w, int32_t mesh_h,
                  double k, double thresh_abs, uint8_t* mask);

/* Detection on the frame smoothed by the normalised 3 x 3 pyramid (reading). */
int orc_threshold_filtered(const float* sub, int64_t W, int64_t H, const float* mesh_rms,
                           int64_t nx, int64_t ny, int32_t mesh_w, int32_t mesh_h,
                           double k, double thresh_abs, uint8_t* mask);

int64_t orc_label(const uint8_t* mask, const float* sub, int64_t W, int64_t H,
                  int32_t min_area, int32_t* labels, int64_t max_src,
                  int32_t* area, int64_t* first, int32_t* xmin, int32_t* xmax,
                  int32_t* ymin, int32_t* ymax, double* peak, double* sum,
                  double* xbar, double* ybar);

int orc_centroid(const float* sub, int64_t W, int64_t H, int64_t n,
                 const float* x0, const float* y0, double fwhm_win,
                 int32_t max_iter, double tol2, double* x, double* y,
                 int32_t* niter, int32_t* flags);

double orc_overlap(double cx, double cy, double r, double x0, double x1,
                   double y0, double y1);

int orc_aperture(const float* sub, int64_t W, int64_t H, int64_t n,
                 const float* x, const float* y, double r_ap, double r_in,
                 double r_out, int32_t min_ann, double* flux, double* sky,
                 double* area, int32_t* n_ann, int32_t* flags);

/* Gray-scale maps (Sec. 2.2.6): kind 0 linear, 1 log, 2 power, 3 exp of the
 * value clipped to [lo, hi]; histogram equalisation over nbins bins. */
int orc_gray_transform(const float* img, int64_t W, int64_t H, int32_t kind, double lo, double hi,
                       double a, double* out);
int orc_hist_equalize(const float* img, int64_t W, int64_t H, int32_t nbins, double* out);

/* Image alignment (Sec. 2.2.3, Eqs. 5-7).  SIP coefficient a[p*6+q] multiplies
 * u^p v^q, p + q <= order <= 5; crpix 1-based; crval and cd in degrees. */
typedef struct {
    double crpix[2];
    double crval[2];
    double cd[4];       /* CD1_1, CD1_2, CD2_1, CD2_2 */
    int32_t a_order, b_order;
    double a[36], b[36];
} orc_wcs;
int orc_wcs_pix2world(const orc_wcs* w, const double* x, const double* y, int64_t n, double* ra, double* dec);
int orc_wcs_world2pix(const orc_wcs* w, const double* ra, const double* dec, int64_t n, double* x, double* y);
int orc_wcs_map(const orc_wcs* src, const orc_wcs* tgt, int64_t W, int64_t H, int32_t step, double* xo,
                double* yo);
int orc_affine_fit(const double* x, const double* y, const double* xt, const double* yt, int64_t n, double* M,
                   double* Minv);
int orc_reproject_affine(const float* src, int64_t W, int64_t H, const double* Minv, int64_t Wo, int64_t Ho,
                         double fill, double* out);

/* ZScale display limits (Sec. 2.2.6; reading after the published IRAF
 * algorithm): z[0], z[1] = z1, z2; counts = (samples, good samples). */
int orc_zscale(const float* img, int64_t W, int64_t H, int32_t n_samples, double contrast, double krej,
               int32_t max_iter, double* z, int32_t* counts);

/* Cleaning of deblended objects (Sec. 2.2.5; SExtractor-style reading):
 * returns the number of kept objects, out = cleaned label map. */
int64_t orc_clean(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t nobj, const float* thr,
                  double beta, int32_t* out);
int orc_clean_stats(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t nobj, double* pk,
                    int64_t* pidx, double* cx, double* cy, double* x2, double* y2, double* xy);

/* Image subtraction (Sec. 2.2.4, Eqs. 8-10): basis, stamps, fit, apply. */
int orc_sub_basis(int32_t hw, const double* sig, const int32_t* deg, int32_t nk, double* out);
int orc_sub_stamps(const float* I, const float* R, int64_t W, int64_t H, int32_t nsx, int32_t nsy, int32_t hw,
                   int32_t fh, double nsig, int32_t* cx, int32_t* cy);
int orc_sub_normal(const float* I, const float* R, int64_t W, int64_t H, const int32_t* cx, const int32_t* cy,
                   int32_t nc, int32_t hw, int32_t fh, const double* sig, const int32_t* deg, int32_t nk,
                   int32_t sord, int32_t bord, double* AtA, double* Atb);
int orc_sub_fit(const float* I, const float* R, int64_t W, int64_t H, const int32_t* cx, const int32_t* cy,
                int32_t nc, int32_t hw, int32_t fh, const double* sig, const int32_t* deg, int32_t nk, int32_t sord,
                int32_t bord, double* coef);
int orc_sub_apply(const float* I, const float* R, int64_t W, int64_t H, int32_t hw, const double* sig,
                  const int32_t* deg, int32_t nk, int32_t sord, int32_t bord, const double* coef, int32_t tile,
                  double* D);

/* Deblending (Sec. 2.2.5): multi-level thresholds, sub-component tree, pruning
 * on intensity (mincont), remaining pixels to the likeliest object; objects
 * numbered candidate by candidate, within one in raster order of their first
 * pixel.  Returns K'. */
int64_t orc_deblend(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t K,
                    int32_t nthresh, double mincont, int32_t* out);

/* Auto (Kron) photometry (Sec. 2.2.5; method paper-silent): moments over the
 * footprint labels == k+1, Kron radius within elliptical radius r_kmax,
 * flux within max(k_kron r1, r_min); see the definition for the steps. */
int orc_auto_phot(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t n,
                  const int32_t* xmin, const int32_t* xmax, const int32_t* ymin,
                  const int32_t* ymax, const float* xbar, const float* ybar,
                  double k_kron, double r_min, double r_kmax, double* flux, double* area,
                  double* kron, double* x2, double* y2, double* xy, int32_t* flags);

/* Stamp cut (paper-silent; input of the PSF fit): S x S stamp whose centre pixel
 * is (floor(x + 1/2), floor(y + 1/2)); out-of-frame pixels 0 with weight 0. */
int orc_stamp_cut(const float* sub, int64_t W, int64_t H, int64_t n,
                  const float* x, const float* y, int32_t S, float* stamps,
                  float* weights, int32_t* origin, int32_t* flags);

/* PSF model (paper-silent reading): params = x0, y0, F, sky, sx, sy, theta */
#define ORC_PSF_MOFFAT 0
#define ORC_PSF_GAUSS 1
int orc_psf_model(const double* prm, int32_t S, int32_t model, double beta,
                  double* m, double* jac /* nullable, [S*S][7] */);

int orc_psf_fit(const float* stamps, int64_t N, int32_t S, const float* weights,
                const float* init, int32_t model, double beta, int32_t max_iter,
                double lambda0, double* params, double* chi2, int32_t* iters,
                int32_t* flags);

int orc_psf_init(const float* stamp, int32_t S, double* p7);

#endif
