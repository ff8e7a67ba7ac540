/*
 * ipp_oracle.c -- TEST INFRASTRUCTURE ONLY (see ipp_oracle.h).
 *
 * Plain FP64 restatement of the catalog path of arXiv 2502.10783:
 *   Sec. 2.2.2 (Eqs. 1-4): mesh background by iterative sigma clipping,
 *                          median filter on the mesh grid, interpolation back
 *                          to full resolution, subtraction;
 *   Sec. 2.2.5           : pixel detection above a threshold, connection of the
 *                          detected pixels into candidates, per-candidate peak and
 *                          total flux, aperture photometry, positions;
 * plus the readings used where the paper is silent (windowed centroid, sky
 * annulus, exact pixel/circle overlap, PSF model and Levenberg-Marquardt fit).
 * No blocking, fusion or reordering beyond the definitions: slow on purpose.
 */
#include "ipp_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Eq. 1 (Sec. 2.2.2): median of N values -- the middle order statistic for odd
 * N, the mean of the two middle ones for even N.  Sorts a copy. */
static double median_of(const double* v, int64_t n) {
    double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(t, v, sizeof(double) * (size_t)n);
    qsort(t, (size_t)n, sizeof(double), cmp_double);
    double m = (n & 1) ? t[(n - 1) / 2] : 0.5 * (t[n / 2 - 1] + t[n / 2]);
    free(t);
    return m;
}

/* ---------------------------------------------------------------- c0 ---- */
/* Bias/flat correction (paper-silent): f = (raw - bias) / flat, cast to float32. */
int orc_calibrate(const uint16_t* raw, int64_t W, int64_t H, int64_t pitch,
                  const float* bias_map, double bias, const float* flat, float* out) {
    if (!raw || !flat || !out || W <= 0 || H <= 0 || pitch < W) return ORC_INVALID_ARG;
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            double b = bias_map ? (double)bias_map[i * W + j] : bias;
            out[i * W + j] = (float)(((double)raw[i * pitch + j] - b) / (double)flat[i * W + j]);
        }
    return ORC_OK;
}

/* ---------------------------------------------------------- c1 / c2 ---- */
/* mean (Eq. 2) and population standard deviation, two-pass, FP64 */
static void mean_sd(const double* v, int64_t n, double* mean, double* sd) {
    double s = 0.0;
    for (int64_t k = 0; k < n; k++) s += v[k];
    double mu = s / (double)n;
    double q = 0.0;
    for (int64_t k = 0; k < n; k++) q += (v[k] - mu) * (v[k] - mu);
    *mean = mu;
    *sd = sqrt(q / (double)n);
}

/*
 * Mesh statistics, Sec. 2.2.2: the frame is cut into mesh_w x mesh_h regions
 * (the last row/column of meshes keeps only its real pixels).  In each mesh the
 * unmasked finite pixels are clipped iteratively: the centre (median, Eq. 1),
 * mean (Eq. 2) and standard deviation are computed, values outside
 * [median - n sigma, median + n sigma] are dropped, and this repeats until no
 * value is dropped or maxiters passes were made.  The background of the mesh is
 * then the chosen estimator of the final set (Eq. 3 by default:
 * 2.5 median - 1.5 mean) and the rms is its standard deviation.  A mesh with
 * fewer than min_valid (100) usable pixels is invalid.
 *
 * margin (diagnostic, nullable): the smallest distance, over all passes, of a
 * value of the set to a clip bound, in units of that pass's sigma.  A tiny
 * margin marks a mesh whose kept set is decided by the last bits of sigma.
 */
int orc_mesh_stats(const float* img, int64_t W, int64_t H, int64_t pitch,
                   const uint8_t* mask, const orc_bg_params* p,
                   double* raw_bkg, double* raw_rms, int32_t* valid,
                   int32_t* niter, double* margin) {
    if (!img || !p || W <= 0 || H <= 0 || pitch < W || p->mesh_w < 1 || p->mesh_h < 1)
        return ORC_INVALID_ARG;
    int64_t nx = (W + p->mesh_w - 1) / p->mesh_w, ny = (H + p->mesh_h - 1) / p->mesh_h;
    /* meshes are independent: with -fopenmp (the all-cores timing build) each
     * thread takes whole meshes with its own scratch; the arithmetic of a mesh
     * is the same either way */
#pragma omp parallel
    {
    double* a = (double*)malloc(sizeof(double) * (size_t)p->mesh_w * (size_t)p->mesh_h);
    double* b = (double*)malloc(sizeof(double) * (size_t)p->mesh_w * (size_t)p->mesh_h);
#pragma omp for schedule(dynamic)
    for (int64_t id = 0; id < nx * ny; id++) {
            const int64_t my = id / nx, mx = id % nx;
            int64_t n = 0;
            for (int64_t i = my * p->mesh_h; i < (my + 1) * p->mesh_h && i < H; i++)
                for (int64_t j = mx * p->mesh_w; j < (mx + 1) * p->mesh_w && j < W; j++) {
                    float v = img[i * pitch + j];
                    if (mask && mask[i * W + j]) continue;
                    if (!isfinite(v)) continue;
                    a[n++] = (double)v;
                }
            double mg = INFINITY;
            if (n < p->min_valid || n == 0) {
                raw_bkg[id] = 0.0; raw_rms[id] = 0.0; valid[id] = 0;
                if (niter) niter[id] = 0;
                if (margin) margin[id] = mg;
                continue;
            }
            double med = 0, mu = 0, sd = 0;
            int it, done = 0;
            for (it = 0; it < p->maxiters; it++) {
                med = median_of(a, n);
                mean_sd(a, n, &mu, &sd);
                double lo = med - p->nsigma * sd, hi = med + p->nsigma * sd;
                int64_t m = 0;
                for (int64_t k = 0; k < n; k++) {
                    if (sd > 0) {
                        double d = fmin(fabs(a[k] - lo), fabs(a[k] - hi)) / sd;
                        if (d < mg) mg = d;
                    }
                    if (a[k] >= lo && a[k] <= hi) b[m++] = a[k];
                }
                if (m == n) { done = 1; it++; break; }
                memcpy(a, b, sizeof(double) * (size_t)m);
                n = m;
            }
            if (!done) { /* set changed on the last allowed pass: statistics of the final set */
                med = median_of(a, n);
                mean_sd(a, n, &mu, &sd);
            }
            double bk;
            switch (p->estimator) {
                case ORC_EST_MEDIAN: bk = med; break;
                case ORC_EST_MEAN: bk = mu; break;
                case ORC_EST_FACTORS: bk = p->median_factor * med - p->mean_factor * mu; break;
                default: bk = 2.5 * med - 1.5 * mu; break;
            }
            raw_bkg[id] = bk; raw_rms[id] = sd; valid[id] = 1;
            if (niter) niter[id] = it;
            if (margin) margin[id] = mg;
        }
    free(a); free(b);
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- c3 ---- */
/*
 * Invalid-mesh fill (paper-silent reading) then the median filter on the mesh
 * grid of Sec. 2.2.2.  An invalid mesh takes the median (Eq. 1) of the valid
 * meshes in the smallest (2k+1)^2 neighbourhood, k = 1, 2, ..., that holds any.
 * The filter replaces each node by the median of the in-bounds nodes of the
 * fw x fh window centred on it (the window shrinks at the grid edges).
 * bkg and rms are treated independently.
 */
int orc_mesh_fill_filter(const double* raw_bkg, const double* raw_rms,
                         const int32_t* valid, int64_t nx, int64_t ny,
                         int32_t fw, int32_t fh, double* bkg, double* rms) {
    int64_t nn = nx * ny, nvalid = 0;
    for (int64_t k = 0; k < nn; k++) nvalid += valid[k] != 0;
    if (nvalid == 0) return ORC_NO_VALID_MESH;
    double* fb = (double*)malloc(sizeof(double) * (size_t)nn);
    double* fr = (double*)malloc(sizeof(double) * (size_t)nn);
    double* tb = (double*)malloc(sizeof(double) * (size_t)nn);
    double* tr = (double*)malloc(sizeof(double) * (size_t)nn);
    for (int64_t p = 0; p < ny; p++)
        for (int64_t q = 0; q < nx; q++) {
            int64_t id = p * nx + q;
            if (valid[id]) { fb[id] = raw_bkg[id]; fr[id] = raw_rms[id]; continue; }
            for (int64_t k = 1;; k++) {
                int64_t c = 0;
                for (int64_t pp = p - k; pp <= p + k; pp++)
                    for (int64_t qq = q - k; qq <= q + k; qq++) {
                        if (pp < 0 || pp >= ny || qq < 0 || qq >= nx) continue;
                        if (!valid[pp * nx + qq]) continue;
                        tb[c] = raw_bkg[pp * nx + qq]; tr[c] = raw_rms[pp * nx + qq]; c++;
                    }
                if (c > 0) { fb[id] = median_of(tb, c); fr[id] = median_of(tr, c); break; }
            }
        }
    int32_t hw = fw / 2, hh = fh / 2;
    for (int64_t p = 0; p < ny; p++)
        for (int64_t q = 0; q < nx; q++) {
            int64_t c = 0;
            for (int64_t pp = p - hh; pp <= p + hh; pp++)
                for (int64_t qq = q - hw; qq <= q + hw; qq++) {
                    if (pp < 0 || pp >= ny || qq < 0 || qq >= nx) continue;
                    tb[c] = fb[pp * nx + qq]; tr[c] = fr[pp * nx + qq]; c++;
                }
            bkg[p * nx + q] = median_of(tb, c);
            rms[p * nx + q] = median_of(tr, c);
        }
    free(fb); free(fr); free(tb); free(tr);
    return ORC_OK;
}

/* ---------------------------------------------------------------- c4 ---- */
/* Keys (1981) cubic convolution kernel with a = -1/2. */
double orc_keys_weight(double s) {
    double t = fabs(s);
    if (t <= 1.0) return 1.5 * t * t * t - 2.5 * t * t + 1.0;
    if (t < 2.0) return -0.5 * t * t * t + 2.5 * t * t - 4.0 * t + 2.0;
    return 0.0;
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Interpolated value at pixel (i, j): mesh node (p, q) sits at
 * ((q + 1/2) mesh_w - 1/2, (p + 1/2) mesh_h - 1/2); separable Keys cubic over the
 * 4 x 4 nearest nodes with indices clamped to the grid, written as
 * v11 + sum w (v - v11) so that equal nodes reproduce exactly. */
static double interp_at(const float* mesh, int64_t nx, int64_t ny, int32_t mw,
                        int32_t mh, int64_t i, int64_t j) {
    double u = ((double)j + 0.5) / (double)mw - 0.5;
    double v = ((double)i + 0.5) / (double)mh - 0.5;
    double qf = floor(u), pf = floor(v);
    double s = u - qf, t = v - pf;
    int64_t q0 = (int64_t)qf, p0 = (int64_t)pf;
    double wx[4], wy[4];
    for (int k = 0; k < 4; k++) {
        wx[k] = orc_keys_weight(s - (double)(k - 1));
        wy[k] = orc_keys_weight(t - (double)(k - 1));
    }
    double v11 = (double)mesh[clampi(p0, 0, ny - 1) * nx + clampi(q0, 0, nx - 1)];
    double acc = 0.0;
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            int64_t pp = clampi(p0 - 1 + a, 0, ny - 1), qq = clampi(q0 - 1 + b, 0, nx - 1);
            acc += wy[a] * wx[b] * ((double)mesh[pp * nx + qq] - v11);
        }
    return v11 + acc;
}

int orc_interp_map(const float* mesh, int64_t nx, int64_t ny, int32_t mesh_w,
                   int32_t mesh_h, int64_t W, int64_t H, double* out) {
    if (!mesh || !out || nx < 1 || ny < 1) return ORC_INVALID_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++)
            out[i * W + j] = interp_at(mesh, nx, ny, mesh_w, mesh_h, i, j);
    return ORC_OK;
}

/* Sec. 2.2.2: interpolate the filtered mesh background back to full
 * resolution and subtract it: sub = f - B (returned as float32). */
int orc_bg_subtract(const float* img, int64_t W, int64_t H, int64_t pitch,
                    const float* mesh_bkg, int64_t nx, int64_t ny,
                    int32_t mesh_w, int32_t mesh_h, float* sub, float* bkg_map) {
    if (!img || !mesh_bkg || !sub || pitch < W) return ORC_INVALID_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            double B = interp_at(mesh_bkg, nx, ny, mesh_w, mesh_h, i, j);
            sub[i * W + j] = (float)((double)img[i * pitch + j] - B);
            if (bkg_map) bkg_map[i * W + j] = (float)B;
        }
    return ORC_OK;
}

/* ---------------------------------------------------------------- c5 ---- */
/* Sec. 2.2.5 pixel detection: a pixel is detected when its background-
 * subtracted value exceeds the threshold max(k * rms(x, y), thresh_abs), with
 * rms(x, y) interpolated from the filtered mesh rms like the background. */
int orc_threshold(const float* sub, int64_t W, int64_t H, const float* mesh_rms,
                  int64_t nx, int64_t ny, int32_t mesh_w, int32_t mesh_h,
                  double k, double thresh_abs, uint8_t* mask) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            double thr = k * interp_at(mesh_rms, nx, ny, mesh_w, mesh_h, i, j);
            if (thresh_abs > thr) thr = thresh_abs;
            mask[i * W + j] = (double)sub[i * W + j] > thr;
        }
    return ORC_OK;
}

/*
 * Detection on a smoothed frame (the detection filter of SExtractor-style
 * pipelines; paper-silent, reading): the subtracted frame is convolved with the
 * 3 x 3 pyramid [1 2 1; 2 4 2; 1 2 1] / 16, the weights renormalised over the
 * taps inside the frame (a constant frame stays constant at the edges), and the
 * convolved value is compared with the same threshold k rms(x, y) (floored at
 * thresh_abs) as unsmoothed detection.  The statistics of the candidates still
 * come from the unsmoothed frame.
 */
int orc_threshold_filtered(const float* sub, int64_t W, int64_t H, const float* mesh_rms,
                           int64_t nx, int64_t ny, int32_t mesh_w, int32_t mesh_h,
                           double k, double thresh_abs, uint8_t* mask) {
    static const double kw[3][3] = {{1, 2, 1}, {2, 4, 2}, {1, 2, 1}};
    for (int64_t i = 0; i < H; i++)
        for (int64_t j = 0; j < W; j++) {
            double num = 0.0, den = 0.0;
            for (int di = -1; di <= 1; di++)
                for (int dj = -1; dj <= 1; dj++) {
                    const int64_t a = i + di, b = j + dj;
                    if (a < 0 || a >= H || b < 0 || b >= W) continue;
                    num += kw[di + 1][dj + 1] * (double)sub[a * W + b];
                    den += kw[di + 1][dj + 1];
                }
            double thr = k * interp_at(mesh_rms, nx, ny, mesh_w, mesh_h, i, j);
            if (thresh_abs > thr) thr = thresh_abs;
            mask[i * W + j] = num / den > thr;
        }
    return ORC_OK;
}

/* ---------------------------------------------------------- c6 / c7 ---- */
/*
 * Sec. 2.2.5: detected pixels are connected into candidates (8-connectivity);
 * candidates smaller than min_area pixels are dropped; the survivors are numbered
 * 1..K in raster order of their first pixel.  Per candidate (the "pre-analysis"
 * of Sec. 2.2.5): area, peak value, total flux, flux-weighted barycentre,
 * bounding box, first-pixel raster index.  Breadth-first flood fill, raster scan.
 * Returns K (all survivors); stats are written for the first max_src of them.
 */
int64_t orc_label(const uint8_t* mask, const float* sub, int64_t W, int64_t H,
                  int32_t min_area, int32_t* labels, int64_t max_src,
                  int32_t* area, int64_t* first, int32_t* xmin, int32_t* xmax,
                  int32_t* ymin, int32_t* ymax, double* peak, double* sum,
                  double* xbar, double* ybar) {
    int64_t npx = W * H;
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npx > 0 ? npx : 1));
    uint8_t* seen = (uint8_t*)calloc((size_t)(npx > 0 ? npx : 1), 1);
    for (int64_t k = 0; k < npx; k++) labels[k] = 0;
    int64_t K = 0;
    for (int64_t s = 0; s < npx; s++) {
        if (!mask[s] || seen[s]) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = s;
        seen[s] = 1;
        while (head < tail) {
            int64_t c = queue[head++];
            int64_t ci = c / W, cj = c % W;
            for (int64_t di = -1; di <= 1; di++)
                for (int64_t dj = -1; dj <= 1; dj++) {
                    int64_t ni = ci + di, nj = cj + dj;
                    if (ni < 0 || ni >= H || nj < 0 || nj >= W) continue;
                    int64_t nk = ni * W + nj;
                    if (mask[nk] && !seen[nk]) { seen[nk] = 1; queue[tail++] = nk; }
                }
        }
        if (tail < min_area) continue;
        K++;
        for (int64_t t = 0; t < tail; t++) labels[queue[t]] = (int32_t)K;
        if (K > max_src) continue;
        int64_t o = K - 1;
        double sm = 0, sx = 0, sy = 0, pk = -INFINITY;
        int32_t x0 = INT32_MAX, x1 = -1, y0 = INT32_MAX, y1 = -1;
        for (int64_t t = 0; t < tail; t++) {
            int64_t c = queue[t], ci = c / W, cj = c % W;
            double f = (double)sub[c];
            sm += f; sx += f * (double)cj; sy += f * (double)ci;
            if (f > pk) pk = f;
            if (cj < x0) x0 = (int32_t)cj;
            if (cj > x1) x1 = (int32_t)cj;
            if (ci < y0) y0 = (int32_t)ci;
            if (ci > y1) y1 = (int32_t)ci;
        }
        area[o] = (int32_t)tail; first[o] = s;
        xmin[o] = x0; xmax[o] = x1; ymin[o] = y0; ymax[o] = y1;
        peak[o] = pk; sum[o] = sm;
        xbar[o] = sx / sm; ybar[o] = sy / sm;
    }
    free(queue); free(seen);
    return K;
}

/* ---------------------------------------------------------------- c8 ---- */
/*
 * Windowed centroid (paper-silent; positions are an output of Sec. 2.2.5).
 * Gaussian window of sigma_w = fwhm_win / (2 sqrt(2 ln 2)) over the pixels
 * whose centres lie within 4 sigma_w of the current position and inside the
 * frame; update x += 2 sum(w f (x_i - x)) / sum(w f), same for y, until the
 * squared step is below tol2 or max_iter updates were made.  A non-positive
 * weighted sum returns the seed with WIN_NOT_CONVERGED.  EDGE is set when the
 * window disk (radius 4 sigma_w) at the final position crosses the frame's outer
 * boundary.
 */
int orc_centroid(const float* sub, int64_t W, int64_t H, int64_t n,
                 const float* x0, const float* y0, double fwhm_win,
                 int32_t max_iter, double tol2, double* x, double* y,
                 int32_t* niter, int32_t* flags) {
    double sw = fwhm_win / (2.0 * sqrt(2.0 * log(2.0)));
    double rad = 4.0 * sw, rad2 = rad * rad;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = 0; s < n; s++) {
        double cx = (double)x0[s], cy = (double)y0[s];
        int32_t fl = ORC_FLAG_WIN_NOT_CONVERGED, it;
        for (it = 0; it < max_iter; it++) {
            double sw0 = 0, swx = 0, swy = 0;
            int64_t i0 = (int64_t)floor(cy - rad), i1 = (int64_t)ceil(cy + rad);
            int64_t j0 = (int64_t)floor(cx - rad), j1 = (int64_t)ceil(cx + rad);
            for (int64_t i = i0; i <= i1; i++)
                for (int64_t j = j0; j <= j1; j++) {
                    double dx = (double)j - cx, dy = (double)i - cy;
                    double d2 = dx * dx + dy * dy;
                    if (!(d2 < rad2)) continue;
                    if (i < 0 || i >= H || j < 0 || j >= W) continue;
                    double w = exp(-d2 / (2.0 * sw * sw)) * (double)sub[i * W + j];
                    sw0 += w; swx += w * dx; swy += w * dy;
                }
            if (!(sw0 > 0.0)) { cx = (double)x0[s]; cy = (double)y0[s]; it++; break; }
            double ddx = 2.0 * swx / sw0, ddy = 2.0 * swy / sw0;
            cx += ddx; cy += ddy;
            if (ddx * ddx + ddy * ddy < tol2) { fl = 0; it++; break; }
        }
        /* EDGE: the window disk at the final position crosses the frame's outer
         * boundary [-1/2, W-1/2] x [-1/2, H-1/2] */
        if (cx - rad < -0.5 || cx + rad > (double)W - 0.5 || cy - rad < -0.5 ||
            cy + rad > (double)H - 0.5)
            fl |= ORC_FLAG_EDGE;
        x[s] = cx; y[s] = cy;
        if (niter) niter[s] = it;
        flags[s] = fl;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- c9 ---- */
/* primitive of sqrt(r^2 - t^2), t relative to the centre:
 *   G(t) = (t sqrt(r^2 - t^2) + r^2 asin(t / r)) / 2,
 * evaluated with r^2 - t^2 = (r - t)(r + t) and asin(t/r) = atan2(t, sqrt(r^2 - t^2))
 * so that it stays accurate next to t = +-r. */
static double prim(double t, double r) {
    if (t >= r) return 0.25 * M_PI * r * r;
    if (t <= -r) return -0.25 * M_PI * r * r;
    double s = sqrt((r - t) * (r + t));
    return 0.5 * (t * s + r * r * atan2(t, s));
}

static double half_chord(double t, double r) {
    double a = fabs(t);
    return a >= r ? 0.0 : sqrt((r - a) * (r + a));
}

/*
 * Exact area of disk(cx, cy, r) intersected with the box [x0,x1] x [y0,y1]
 * (paper-silent reading of "aperture photometry"), in coordinates centred on
 * the disk: integral over x of the chord clipped to [y0, y1].  The x range is
 * split where the circle crosses y = y0 and y = y1, so that on each piece the
 * upper limit is either y1 or the circle and the lower limit either y0 or the
 * circle; the circle parts integrate through the primitive G above.
 */
double orc_overlap(double cx, double cy, double r, double x0, double x1,
                   double y0, double y1) {
    double X0 = x0 - cx, X1 = x1 - cx, Y0 = y0 - cy, Y1 = y1 - cy;
    double a = fmax(X0, -r), b = fmin(X1, r);
    if (!(a < b) || !(Y0 < Y1)) return 0.0;
    double pts[6];
    int np = 0;
    pts[np++] = a;
    double ys[2] = {Y0, Y1};
    for (int k = 0; k < 2; k++) {
        if (fabs(ys[k]) <= r) {  /* |y| = r: the circle touches the edge line at x = 0 */
            double h = half_chord(ys[k], r);
            if (-h > a && -h < b) pts[np++] = -h;
            if (h > a && h < b) pts[np++] = h;
        }
    }
    pts[np++] = b;
    qsort(pts, (size_t)np, sizeof(double), cmp_double);
    double area = 0.0;
    for (int k = 0; k + 1 < np; k++) {
        double p = pts[k], q = pts[k + 1];
        if (!(q > p)) continue;
        double hm = half_chord(0.5 * (p + q), r);
        double up = hm < Y1 ? hm : Y1;
        double lo = -hm > Y0 ? -hm : Y0;
        if (!(up > lo)) continue;
        double dG = prim(q, r) - prim(p, r);
        double iu = (hm < Y1) ? dG : Y1 * (q - p);
        double il = (-hm > Y0) ? -dG : Y0 * (q - p);
        area += iu - il;
    }
    return area;
}

/* --------------------------------------------------------- c10 / c11 ---- */
/*
 * Aperture photometry (Sec. 2.2.5) with a local sky annulus (paper-silent):
 *   w(i,j) = exact overlap of the aperture disk with pixel (i,j);
 *   sky    = median (Eq. 1) of the in-frame pixels whose centres satisfy
 *            r_in <= d < r_out (d^2 = (j-x)^2 + (i-y)^2 in FP64); fewer than
 *            min_ann of them -> sky = 0 and ANN_FEW;
 *   flux   = sum w f - sky sum w, area = sum w, over in-frame pixels;
 *   EDGE when the disk of radius max(r_ap, r_out) crosses the frame's outer
 *   boundary [-1/2, W-1/2] x [-1/2, H-1/2].
 */
int orc_aperture(const float* sub, int64_t W, int64_t H, int64_t n,
                 const float* x, const float* y, double r_ap, double r_in,
                 double r_out, int32_t min_ann, double* flux, double* sky,
                 double* area, int32_t* n_ann, int32_t* flags) {
    int64_t cap = (int64_t)((2 * ceil(r_out) + 3) * (2 * ceil(r_out) + 3));
    double rin2 = r_in * r_in, rout2 = r_out * r_out;
#pragma omp parallel
    {
    double* ann = (double*)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
    for (int64_t s = 0; s < n; s++) {
        double cx = (double)x[s], cy = (double)y[s];
        int32_t fl = 0;
        double sw = 0, swf = 0;
        int64_t i0 = (int64_t)floor(cy - r_ap) - 1, i1 = (int64_t)ceil(cy + r_ap) + 1;
        int64_t j0 = (int64_t)floor(cx - r_ap) - 1, j1 = (int64_t)ceil(cx + r_ap) + 1;
        for (int64_t i = i0; i <= i1; i++)
            for (int64_t j = j0; j <= j1; j++) {
                double w = orc_overlap(cx, cy, r_ap, (double)j - 0.5, (double)j + 0.5,
                                       (double)i - 0.5, (double)i + 0.5);
                if (!(w > 0.0)) continue;
                if (i < 0 || i >= H || j < 0 || j >= W) continue;
                sw += w; swf += w * (double)sub[i * W + j];
            }
        int64_t na = 0;
        i0 = (int64_t)floor(cy - r_out) - 1; i1 = (int64_t)ceil(cy + r_out) + 1;
        j0 = (int64_t)floor(cx - r_out) - 1; j1 = (int64_t)ceil(cx + r_out) + 1;
        for (int64_t i = i0; i <= i1; i++)
            for (int64_t j = j0; j <= j1; j++) {
                double dx = (double)j - cx, dy = (double)i - cy;
                double d2 = dx * dx + dy * dy;
                if (!(d2 >= rin2 && d2 < rout2)) continue;
                if (i < 0 || i >= H || j < 0 || j >= W) continue;
                ann[na++] = (double)sub[i * W + j];
            }
        {
            double R = r_ap > r_out ? r_ap : r_out;
            if (cx - R < -0.5 || cx + R > (double)W - 0.5 || cy - R < -0.5 ||
                cy + R > (double)H - 0.5)
                fl |= ORC_FLAG_EDGE;
        }
        double sk = 0.0;
        if (na < min_ann) fl |= ORC_FLAG_ANN_FEW;
        else sk = median_of(ann, na);
        flux[s] = swf - sk * sw;
        sky[s] = sk; area[s] = sw; n_ann[s] = (int32_t)na; flags[s] = fl;
    }
    free(ann);
    }
    return ORC_OK;
}

/* ----------------------------------------------------- gray-scale maps */
/*
 * Gray-scale transforms (Sec. 2.2.6: pixel values mapped to new gray values by
 * mathematical functions; the functions are readings after the usual display
 * scales).  xn = clip((x - lo) / (hi - lo), 0, 1); non-finite x gives 0.
 *   ORC_GRAY_LINEAR  y = xn
 *   ORC_GRAY_LOG     y = log10(a xn + 1) / log10(a + 1)
 *   ORC_GRAY_POWER   y = xn ^ a            (a > 0)
 *   ORC_GRAY_EXP     y = (a ^ xn - 1) / (a - 1)   (a > 0, a != 1)
 */
int orc_gray_transform(const float* img, int64_t W, int64_t H, int32_t kind, double lo, double hi,
                       double a, double* out) {
    if (!(hi > lo)) return ORC_INVALID_ARG;
    for (int64_t k = 0; k < W * H; k++) {
        const double x = (double)img[k];
        if (!isfinite(x)) { out[k] = 0.0; continue; }
        double xn = (x - lo) / (hi - lo);
        xn = xn < 0.0 ? 0.0 : (xn > 1.0 ? 1.0 : xn);
        double y;
        switch (kind) {
            case 1: y = log10(a * xn + 1.0) / log10(a + 1.0); break;
            case 2: y = pow(xn, a); break;
            case 3: y = (pow(a, xn) - 1.0) / (a - 1.0); break;
            default: y = xn;
        }
        out[k] = y;
    }
    return ORC_OK;
}

/*
 * Histogram equalisation (Sec. 2.2.6: a histogram of the gray values, its
 * cumulative distribution, and an interpolation that maps each value onto a
 * uniform distribution).  Over the finite pixels: mn, mx = min, max; nbins bins
 * of width (mx - mn) / nbins; the bin of x is floor((x - mn) s), s = nbins /
 * (mx - mn), clamped to the last bin -- taken in single precision, exactly as
 * written here, because it decides an integer; cdf_i = (count of bins <= i) / N;
 * y = the linear interpolation of cdf between the bin centres at
 * t = (x - mn) s - 1/2 (float), held at cdf_0 below the first centre and cdf_last
 * above the last.  mx == mn gives 0; non-finite pixels give 0.
 */
int orc_hist_equalize(const float* img, int64_t W, int64_t H, int32_t nbins, double* out) {
    if (nbins < 2) return ORC_INVALID_ARG;
    const int64_t n = W * H;
    float mn = INFINITY, mx = -INFINITY;
    int64_t nf = 0;
    for (int64_t k = 0; k < n; k++) {
        const float x = img[k];
        if (!isfinite(x)) continue;
        if (x < mn) mn = x;
        if (x > mx) mx = x;
        nf++;
    }
    if (nf == 0 || !(mx > mn)) {
        for (int64_t k = 0; k < n; k++) out[k] = 0.0;
        return ORC_OK;
    }
    const float sc = (float)nbins / (mx - mn);
    int64_t* cnt = (int64_t*)calloc((size_t)nbins, sizeof(int64_t));
    for (int64_t k = 0; k < n; k++) {
        const float x = img[k];
        if (!isfinite(x)) continue;
        int b = (int)floorf((x - mn) * sc);
        if (b > nbins - 1) b = nbins - 1;
        if (b < 0) b = 0;
        cnt[b]++;
    }
    double* cdf = (double*)malloc(sizeof(double) * (size_t)nbins);
    int64_t run = 0;
    for (int b = 0; b < nbins; b++) { run += cnt[b]; cdf[b] = (double)run / (double)nf; }
    for (int64_t k = 0; k < n; k++) {
        const float x = img[k];
        if (!isfinite(x)) { out[k] = 0.0; continue; }
        const float t = (x - mn) * sc - 0.5f;
        if (!(t > 0.0f)) { out[k] = cdf[0]; continue; }
        const int b = (int)floorf(t);
        if (b >= nbins - 1) { out[k] = cdf[nbins - 1]; continue; }
        const double fr = (double)(t - (float)b);
        out[k] = cdf[b] + fr * (cdf[b + 1] - cdf[b]);
    }
    free(cnt); free(cdf);
    return ORC_OK;
}

/* ------------------------------------------------------------ deblending */
/*
 * Deblending (Sec. 2.2.5, source detection: multi-level thresholds between each
 * candidate's threshold and its peak, a tree of the sub-components found at
 * each level, traversed bottom-up and pruned on intensity).  Reading:
 *  levels -- per candidate C (pixels labelled c): T = min sub over C,
 *    P = max sub over C, L_i = T (P/T)^(i/N) for i = 1 .. N-1 (N = nthresh),
 *    in FP64 (by square roots and products when N is a power of two, see
 *    level_of).  A candidate with T <= 0 or P <= T stays whole.
 *  tree -- the nodes of level i are the 8-connected components of
 *    {p in C : sub(p) > L_i}; level 0 is C itself.  The parent of a level-i
 *    node is the level-(i-1) node holding its pixels (level sets are nested).
 *    flux(node) = sum of sub over its pixels.
 *  objects, from the top level down -- a node without children is one object.
 *    Otherwise let S be its children whose flux is at least mincont x flux(C):
 *    |S| >= 2 gives the objects of every member of S; |S| = 1 gives the
 *    objects of that child when it has two or more, else the node itself;
 *    |S| = 0 gives the node itself.  C splits when its root yields two or
 *    more objects.
 *  pixels -- the pixels of an object's node are its core.  Every other pixel
 *    of C goes to the object whose elliptical Gaussian is largest there:
 *    F exp(-r^2/2) / sqrt(x2 y2 - xy^2), with F, barycentre and second moments
 *    (x2, y2, xy) of the core (weights sub; 1/12 added to x2 and y2 when
 *    x2 y2 - xy^2 < 1/144) and r the Mahalanobis distance, compared as
 *    log F - log(x2 y2 - xy^2)/2 - r^2/2 (far from every core the Gaussians
 *    themselves underflow to 0 and could not be told apart); ties go to the
 *    object whose core starts first in raster order.
 *  numbering -- the objects of candidate 1 first, then those of candidate 2,
 *    and so on; within a candidate, raster order of each object's first pixel.
 *    Numbers run 1..K'.
 * Returns K'.
 */
static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

/* Level lv of N between T and P: T (P/T)^(lv/N).  For N a power of two the
 * N-th root of P/T is taken by log2(N) square roots and the level is T r^lv
 * formed by lv successive products (basic IEEE operations only, so any
 * implementation following the same steps gets the same double); else pow. */
static double level_of(double T, double P, int lv, int N) {
    if ((N & (N - 1)) == 0) {
        double r = P / T;
        for (int m = N; m > 1; m >>= 1) r = sqrt(r);
        double L = T;
        for (int k = 0; k < lv; k++) L = L * r;
        return L;
    }
    return T * pow(P / T, (double)lv / (double)N);
}

int64_t orc_deblend(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t K,
                    int32_t nthresh, double mincont, int32_t* out) {
    if (!sub || !labels || !out || W <= 0 || H <= 0 || K < 0 || nthresh < 2) return -1;
    const int64_t npx = W * H;
    /* pixel lists of the candidates, raster order (CSR) */
    int64_t* start = (int64_t*)calloc((size_t)K + 2, sizeof(int64_t));
    for (int64_t q = 0; q < npx; q++)
        if (labels[q] > 0 && labels[q] <= K) start[labels[q] + 1]++;
    for (int64_t c = 0; c <= K; c++) start[c + 1] += start[c];
    int64_t* pix = (int64_t*)malloc(sizeof(int64_t) * (size_t)(start[K + 1] > 0 ? start[K + 1] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(K + 1));
    for (int64_t c = 0; c <= K; c++) fill[c] = start[c];
    for (int64_t q = 0; q < npx; q++) {
        out[q] = 0;
        if (labels[q] > 0 && labels[q] <= K) pix[fill[labels[q]]++] = q;
    }
    /* object id of every pixel (provisional numbering), and each object's first pixel */
    int64_t* obj_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)(npx > 0 ? npx : 1));
    int64_t cap_obj = K + 16, nobj = 0;
    int64_t* obj_first = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap_obj);
    int64_t* obj_cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap_obj);
    for (int64_t c = 1; c <= K; c++) {
        const int64_t n = start[c + 1] - start[c];
        const int64_t* P = pix + start[c];
        if (n == 0) continue;
        double T = INFINITY, Pk = -INFINITY, Fc = 0.0;
        int64_t i0 = INT64_MAX, i1 = -1, j0 = INT64_MAX, j1 = -1;
        for (int64_t t = 0; t < n; t++) {
            const double f = (double)sub[P[t]];
            if (f < T) T = f;
            if (f > Pk) Pk = f;
            Fc += f;
            const int64_t i = P[t] / W, j = P[t] % W;
            if (i < i0) i0 = i;
            if (i > i1) i1 = i;
            if (j < j0) j0 = j;
            if (j > j1) j1 = j;
        }
        /* local index map of the candidate's box */
        const int64_t bw = j1 - j0 + 1, bh = i1 - i0 + 1;
        int64_t* map = (int64_t*)malloc(sizeof(int64_t) * (size_t)(bw * bh));
        for (int64_t t = 0; t < bw * bh; t++) map[t] = -1;
        for (int64_t t = 0; t < n; t++) map[(P[t] / W - i0) * bw + (P[t] % W - j0)] = t;
        /* node of each pixel at each level (-1: below the level); level 0 = node 0 */
        const int N = nthresh;
        int64_t* node = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * N));
        int64_t* nnodes = (int64_t*)calloc((size_t)N, sizeof(int64_t));
        for (int64_t t = 0; t < n; t++) node[t] = 0;
        nnodes[0] = 1;
        const int split_ok = T > 0.0 && Pk > T;
        int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        for (int lv = 1; lv < N; lv++) {
            int64_t* nd = node + (int64_t)lv * n;
            for (int64_t t = 0; t < n; t++) nd[t] = -1;
            if (!split_ok) continue;
            const double L = level_of(T, Pk, lv, N);
            int64_t m = 0;
            for (int64_t s0 = 0; s0 < n; s0++) {
                if (nd[s0] >= 0 || !((double)sub[P[s0]] > L)) continue;
                int64_t head = 0, tail = 0;
                queue[tail++] = s0;
                nd[s0] = m;
                while (head < tail) {
                    const int64_t u = queue[head++];
                    const int64_t ui = P[u] / W - i0, uj = P[u] % W - j0;
                    for (int64_t di = -1; di <= 1; di++)
                        for (int64_t dj = -1; dj <= 1; dj++) {
                            const int64_t vi = ui + di, vj = uj + dj;
                            if (vi < 0 || vi >= bh || vj < 0 || vj >= bw) continue;
                            const int64_t v = map[vi * bw + vj];
                            if (v < 0 || nd[v] >= 0 || !((double)sub[P[v]] > L)) continue;
                            nd[v] = m;
                            queue[tail++] = v;
                        }
                }
                m++;
            }
            nnodes[lv] = m;
        }
        /* node offsets, fluxes, parents, first pixel (in the candidate's raster list) */
        int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
        off[0] = 0;
        for (int lv = 0; lv < N; lv++) off[lv + 1] = off[lv] + nnodes[lv];
        const int64_t tot = off[N];
        double* flux = (double*)calloc((size_t)tot, sizeof(double));
        int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)tot);
        int64_t* nfirst = (int64_t*)malloc(sizeof(int64_t) * (size_t)tot);
        for (int64_t g = 0; g < tot; g++) { parent[g] = -1; nfirst[g] = INT64_MAX; }
        for (int lv = 0; lv < N; lv++)
            for (int64_t t = 0; t < n; t++) {
                const int64_t a = node[(int64_t)lv * n + t];
                if (a < 0) continue;
                const int64_t g = off[lv] + a;
                flux[g] += (double)sub[P[t]];
                if (t < nfirst[g]) nfirst[g] = t;
                if (lv > 0) parent[g] = off[lv - 1] + node[(int64_t)(lv - 1) * n + t];
            }
        /* objects bottom-up: each node's list of object nodes (CSR built per node) */
        int64_t** objs = (int64_t**)calloc((size_t)tot, sizeof(int64_t*));
        int64_t* nob = (int64_t*)calloc((size_t)tot, sizeof(int64_t));
        for (int lv = N - 1; lv >= 0; lv--)
            for (int64_t a = 0; a < nnodes[lv]; a++) {
                const int64_t g = off[lv] + a;
                int64_t nsig = 0, sig = -1, total = 0;
                if (lv + 1 < N)
                    for (int64_t b = 0; b < nnodes[lv + 1]; b++) {
                        const int64_t h = off[lv + 1] + b;
                        if (parent[h] != g) continue;
                        if (flux[h] >= mincont * Fc) { nsig++; sig = h; total += nob[h]; }
                    }
                int64_t cnt = 0;
                if (nsig >= 2) cnt = total;
                else if (nsig == 1 && nob[sig] >= 2) cnt = nob[sig];
                else cnt = 1;
                objs[g] = (int64_t*)malloc(sizeof(int64_t) * (size_t)cnt);
                nob[g] = cnt;
                if (nsig >= 2) {
                    int64_t w = 0;
                    for (int64_t b = 0; b < nnodes[lv + 1]; b++) {
                        const int64_t h = off[lv + 1] + b;
                        if (parent[h] != g || !(flux[h] >= mincont * Fc)) continue;
                        for (int64_t e = 0; e < nob[h]; e++) objs[g][w++] = objs[h][e];
                    }
                } else if (nsig == 1 && nob[sig] >= 2) {
                    for (int64_t e = 0; e < nob[sig]; e++) objs[g][e] = objs[sig][e];
                } else {
                    objs[g][0] = g;
                }
            }
        const int64_t no = nob[0];
        /* order the objects by the first pixel of their cores */
        int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * no));
        for (int64_t e = 0; e < no; e++) { ord[2 * e] = nfirst[objs[0][e]]; ord[2 * e + 1] = objs[0][e]; }
        qsort(ord, (size_t)no, 2 * sizeof(int64_t), cmp_i64);
        /* level and node index of each object's core */
        int* olv = (int*)malloc(sizeof(int) * (size_t)no);
        int64_t* onode = (int64_t*)malloc(sizeof(int64_t) * (size_t)no);
        for (int64_t e = 0; e < no; e++) {
            const int64_t g = ord[2 * e + 1];
            int lv = 0;
            while (lv + 1 <= N && off[lv + 1] <= g) lv++;
            olv[e] = lv;
            onode[e] = g - off[lv];
        }
        int64_t* assign = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        for (int64_t t = 0; t < n; t++) assign[t] = -1;
        if (no == 1) {
            for (int64_t t = 0; t < n; t++) assign[t] = 0;
        } else {
            double* F = (double*)calloc((size_t)no, sizeof(double));
            double* mx = (double*)calloc((size_t)no, sizeof(double));
            double* my = (double*)calloc((size_t)no, sizeof(double));
            double* ca = (double*)calloc((size_t)no, sizeof(double));
            double* cb = (double*)calloc((size_t)no, sizeof(double));
            double* cc = (double*)calloc((size_t)no, sizeof(double));
            double* nrm = (double*)calloc((size_t)no, sizeof(double));
            for (int64_t e = 0; e < no; e++) {
                double s0 = 0, sx = 0, sy = 0;
                for (int64_t t = 0; t < n; t++) {
                    if (node[(int64_t)olv[e] * n + t] != onode[e]) continue;
                    assign[t] = e;
                    const double f = (double)sub[P[t]];
                    s0 += f; sx += f * (double)(P[t] % W); sy += f * (double)(P[t] / W);
                }
                F[e] = s0; mx[e] = sx / s0; my[e] = sy / s0;
                double sxx = 0, syy = 0, sxy = 0;
                for (int64_t t = 0; t < n; t++) {
                    if (node[(int64_t)olv[e] * n + t] != onode[e]) continue;
                    const double f = (double)sub[P[t]];
                    const double dx = (double)(P[t] % W) - mx[e], dy = (double)(P[t] / W) - my[e];
                    sxx += f * dx * dx; syy += f * dy * dy; sxy += f * dx * dy;
                }
                double x2 = sxx / s0, y2 = syy / s0, xy = sxy / s0;
                if (x2 * y2 - xy * xy < 1.0 / 144.0) { x2 += 1.0 / 12.0; y2 += 1.0 / 12.0; }
                const double det = x2 * y2 - xy * xy;
                ca[e] = y2 / det; cb[e] = -2.0 * xy / det; cc[e] = x2 / det;
                nrm[e] = log(F[e]) - 0.5 * log(det);  /* log of F / sqrt(det) */
            }
            for (int64_t t = 0; t < n; t++) {
                if (assign[t] >= 0) continue;
                const double x = (double)(P[t] % W), y = (double)(P[t] / W);
                int64_t best = 0;
                double bv = -INFINITY;
                for (int64_t e = 0; e < no; e++) {  /* largest log-likelihood */
                    const double dx = x - mx[e], dy = y - my[e];
                    const double r2 = ca[e] * dx * dx + cb[e] * dx * dy + cc[e] * dy * dy;
                    const double v = nrm[e] - 0.5 * r2;
                    if (v > bv) { bv = v; best = e; }
                }
                assign[t] = best;
            }
            free(F); free(mx); free(my); free(ca); free(cb); free(cc); free(nrm);
        }
        /* provisional object ids; the first pixel of each object */
        if (nobj + no > cap_obj) {
            while (nobj + no > cap_obj) cap_obj *= 2;
            obj_first = (int64_t*)realloc(obj_first, sizeof(int64_t) * (size_t)cap_obj);
            obj_cand = (int64_t*)realloc(obj_cand, sizeof(int64_t) * (size_t)cap_obj);
        }
        for (int64_t e = 0; e < no; e++) { obj_first[nobj + e] = INT64_MAX; obj_cand[nobj + e] = c; }
        for (int64_t t = 0; t < n; t++) {
            const int64_t id = nobj + assign[t];
            obj_of[P[t]] = id;
            if (P[t] < obj_first[id]) obj_first[id] = P[t];
        }
        nobj += no;
        for (int64_t g = 0; g < tot; g++) free(objs[g]);
        free(objs); free(nob); free(ord); free(olv); free(onode); free(assign);
        free(flux); free(parent); free(nfirst); free(off); free(node); free(nnodes); free(queue); free(map);
    }
    /* numbering: candidate by candidate (provisional ids are consecutive per
     * candidate), within one by the raster order of the objects' first pixels */
    int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nobj > 0 ? nobj : 1));
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * (nobj > 0 ? nobj : 1)));
    for (int64_t e0 = 0; e0 < nobj;) {
        int64_t e1 = e0 + 1;
        while (e1 < nobj && obj_cand[e1] == obj_cand[e0]) e1++;
        for (int64_t e = e0; e < e1; e++) { ord[2 * (e - e0)] = obj_first[e]; ord[2 * (e - e0) + 1] = e; }
        qsort(ord, (size_t)(e1 - e0), 2 * sizeof(int64_t), cmp_i64);
        for (int64_t e = e0; e < e1; e++) rank[ord[2 * (e - e0) + 1]] = e0 + (e - e0) + 1;
        e0 = e1;
    }
    for (int64_t c = 1; c <= K; c++)
        for (int64_t t = start[c]; t < start[c + 1]; t++) out[pix[t]] = (int32_t)rank[obj_of[pix[t]]];
    free(ord); free(rank); free(obj_first); free(obj_cand); free(obj_of); free(fill); free(pix); free(start);
    return nobj;
}

/* ------------------------------------------------------ auto photometry */
/*
 * Auto photometry (Sec. 2.2.5 lists it beside aperture and isophotal photometry;
 * the method is paper-silent: the reading follows Kron's first-moment radius
 * and SExtractor's automatic elliptical aperture).  Per source k (label k+1):
 *  1. shape -- second moments of sub over the isophotal footprint about the
 *     given barycentre:  x2 = sum f dx^2 / sum f, y2 = sum f dy^2 / sum f,
 *     xy = sum f dx dy / sum f, dx = x - xbar, dy = y - ybar.  A footprint
 *     thinner than a pixel (x2 y2 - xy^2 < 1/144) gets 1/12, the variance of a
 *     uniform pixel, added to x2 and y2.  A footprint whose sum f is not
 *     positive takes x2 = y2 = 1/12, xy = 0 and is flagged KRON_BAD.
 *  2. elliptical radius of a pixel centre:
 *     r^2 = (y2 dx^2 - 2 xy dx dy + x2 dy^2) / (x2 y2 - xy^2),
 *     the Mahalanobis distance under the moment covariance (r = 1 on its
 *     1-sigma ellipse).
 *  3. Kron radius r1 = sum r f / sum f over every in-frame pixel with
 *     r <= r_kmax (not only the footprint; neighbours are not masked).  If
 *     either sum is not positive, r1 = 0 and KRON_BAD.
 *  4. aperture R = max(k_kron r1, r_min); flux = sum f over in-frame pixels
 *     with r <= R, area = their number; EDGE when a pixel centre with r <= R
 *     lies in the one-pixel border around the frame (rows -1 and H, columns
 *     -1 and W).
 * Integer points examined: the box xbar -/+ (R sqrt(x2) + 1), likewise in y,
 * which holds the whole ellipse r <= R, cut to the frame and its border.
 */
static void ellipse_box(double c, double half, int64_t* lo, int64_t* hi) {
    *lo = (int64_t)floor(c - half) - 1;
    *hi = (int64_t)ceil(c + half) + 1;
}

int orc_auto_phot(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t n,
                  const int32_t* xmin, const int32_t* xmax, const int32_t* ymin,
                  const int32_t* ymax, const float* xbar, const float* ybar,
                  double k_kron, double r_min, double r_kmax, double* flux, double* area,
                  double* kron, double* x2o, double* y2o, double* xyo, int32_t* flags) {
    if (!sub || !labels || W <= 0 || H <= 0 || n < 0 || !(k_kron > 0) || !(r_min >= 0) ||
        !(r_kmax > 0))
        return ORC_INVALID_ARG;
    for (int64_t k = 0; k < n; k++) {
        const double xb = (double)xbar[k], yb = (double)ybar[k];
        int32_t fl = 0;
        /* 1. moments over the footprint */
        double s0 = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
        for (int64_t i = ymin[k]; i <= ymax[k]; i++)
            for (int64_t j = xmin[k]; j <= xmax[k]; j++) {
                if (labels[i * W + j] != (int32_t)(k + 1)) continue;
                const double f = (double)sub[i * W + j], dx = (double)j - xb, dy = (double)i - yb;
                s0 += f;
                sxx += f * dx * dx;
                syy += f * dy * dy;
                sxy += f * dx * dy;
            }
        double x2, y2, xy;
        if (s0 > 0.0) {
            x2 = sxx / s0; y2 = syy / s0; xy = sxy / s0;
            if (x2 * y2 - xy * xy < 1.0 / 144.0) { x2 += 1.0 / 12.0; y2 += 1.0 / 12.0; }
        } else {
            x2 = 1.0 / 12.0; y2 = 1.0 / 12.0; xy = 0.0;
            fl |= ORC_FLAG_KRON_BAD;
        }
        const double det = x2 * y2 - xy * xy;
        /* 3. Kron radius */
        double r1 = 0.0;
        if (!(fl & ORC_FLAG_KRON_BAD)) {
            int64_t x0, x1, y0, y1;
            ellipse_box(xb, r_kmax * sqrt(x2), &x0, &x1);
            ellipse_box(yb, r_kmax * sqrt(y2), &y0, &y1);
            double sr = 0.0, sf = 0.0;
            for (int64_t i = y0; i <= y1; i++)
                for (int64_t j = x0; j <= x1; j++) {
                    if (i < 0 || i >= H || j < 0 || j >= W) continue;
                    const double dx = (double)j - xb, dy = (double)i - yb;
                    const double r2 = (y2 * dx * dx - 2.0 * xy * dx * dy + x2 * dy * dy) / det;
                    if (r2 > r_kmax * r_kmax) continue;
                    const double f = (double)sub[i * W + j];
                    sr += sqrt(r2) * f;
                    sf += f;
                }
            if (sf > 0.0 && sr > 0.0) r1 = sr / sf;
            else fl |= ORC_FLAG_KRON_BAD;
        }
        /* 4. the automatic aperture */
        const double R = fmax(k_kron * r1, r_min);
        int64_t x0, x1, y0, y1;
        ellipse_box(xb, R * sqrt(x2), &x0, &x1);
        ellipse_box(yb, R * sqrt(y2), &y0, &y1);
        if (x0 < -1) x0 = -1;
        if (x1 > W) x1 = W;
        if (y0 < -1) y0 = -1;
        if (y1 > H) y1 = H;
        double fs = 0.0, na = 0.0;
        for (int64_t i = y0; i <= y1; i++)
            for (int64_t j = x0; j <= x1; j++) {
                const double dx = (double)j - xb, dy = (double)i - yb;
                const double r2 = (y2 * dx * dx - 2.0 * xy * dx * dy + x2 * dy * dy) / det;
                if (r2 > R * R) continue;
                if (i < 0 || i >= H || j < 0 || j >= W) { fl |= ORC_FLAG_EDGE; continue; }
                fs += (double)sub[i * W + j];
                na += 1.0;
            }
        flux[k] = fs; area[k] = na; kron[k] = r1;
        if (x2o) x2o[k] = x2;
        if (y2o) y2o[k] = y2;
        if (xyo) xyo[k] = xy;
        flags[k] = fl;
    }
    return ORC_OK;
}

/* ----------------------------------------------------------- stamps ---- */
/* The stamp of a source is the S x S block of the subtracted frame centred on
 * the pixel nearest to its position, ties rounded up: centre column
 * floor(x + 1/2), computed in FP64 where x + 1/2 is exact for every float x.
 * Pixels beyond the frame are 0 and get weight 0; a stamp that needs any of
 * them is flagged EDGE.  A non-finite position, or one more than 2^30 px
 * outside the frame, gives an all-zero stamp at origin (0, 0), flagged EDGE. */
int orc_stamp_cut(const float* sub, int64_t W, int64_t H, int64_t n,
                  const float* x, const float* y, int32_t S, float* stamps,
                  float* weights, int32_t* origin, int32_t* flags) {
    if (!sub || W <= 0 || H <= 0 || n < 0 || S < 3 || S % 2 == 0) return ORC_INVALID_ARG;
    int64_t half = S / 2;
    double lim = 1073741824.0 + (double)(W > H ? W : H);
    for (int64_t s = 0; s < n; s++) {
        double xs = x[s], ys = y[s];
        int ok = isfinite(xs) && isfinite(ys) && fabs(xs) < lim && fabs(ys) < lim;
        int64_t ox = 0, oy = 0;
        if (ok) {
            ox = (int64_t)floor(xs + 0.5) - half;
            oy = (int64_t)floor(ys + 0.5) - half;
        }
        int edge = !ok;
        for (int64_t r = 0; r < S; r++)
            for (int64_t c = 0; c < S; c++) {
                int64_t fy = oy + r, fx = ox + c, k = (s * S + r) * S + c;
                int in = ok && fy >= 0 && fy < H && fx >= 0 && fx < W;
                if (!in) edge = 1;
                stamps[k] = in ? sub[fy * W + fx] : 0.0f;
                if (weights) weights[k] = in ? 1.0f : 0.0f;
            }
        if (origin) { origin[2 * s] = (int32_t)ox; origin[2 * s + 1] = (int32_t)oy; }
        if (flags) flags[s] = edge ? ORC_FLAG_EDGE : 0;
    }
    return ORC_OK;
}

/* --------------------------------------------------------------- c12 ---- */
/*
 * PSF model (paper-silent), point-sampled at the pixel centres of an S x S
 * stamp, params (x0, y0, F, sky, sx, sy, theta):
 *   u = cos(t) dx + sin(t) dy,  v = -sin(t) dx + cos(t) dy,  dx = j - x0, dy = i - y0
 *   q = u^2/sx^2 + v^2/sy^2
 *   Moffat  : m = F (beta - 1) / (pi sx sy) (1 + q)^-beta + sky
 *   Gaussian: m = F / (2 pi sx sy) exp(-q / 2) + sky
 * Both profiles integrate to F over the plane.  jac (nullable) receives the
 * analytic derivatives dm/dparam, row-major [pixel][7].
 */
int orc_psf_model(const double* prm, int32_t S, int32_t model, double beta,
                  double* m, double* jac) {
    double x0 = prm[0], y0 = prm[1], F = prm[2], sky = prm[3];
    double sx = prm[4], sy = prm[5], th = prm[6];
    double c = cos(th), s = sin(th);
    for (int32_t i = 0; i < S; i++)
        for (int32_t j = 0; j < S; j++) {
            double dx = (double)j - x0, dy = (double)i - y0;
            double u = c * dx + s * dy, v = -s * dx + c * dy;
            double q = u * u / (sx * sx) + v * v / (sy * sy);
            double P, dPdq;
            if (model == ORC_PSF_GAUSS) {
                double A = F / (2.0 * M_PI * sx * sy);
                P = A * exp(-0.5 * q);
                dPdq = -0.5 * P;
            } else {
                double A = F * (beta - 1.0) / (M_PI * sx * sy);
                P = A * pow(1.0 + q, -beta);
                dPdq = -beta * P / (1.0 + q);
            }
            int64_t k = (int64_t)i * S + j;
            m[k] = P + sky;
            if (jac) {
                double* J = jac + 7 * k;
                double dqdu = 2.0 * u / (sx * sx), dqdv = 2.0 * v / (sy * sy);
                /* du/dx0 = -c, dv/dx0 = s ; du/dy0 = -s, dv/dy0 = -c */
                J[0] = dPdq * (dqdu * (-c) + dqdv * s);
                J[1] = dPdq * (dqdu * (-s) + dqdv * (-c));
                J[2] = (F != 0.0) ? P / F : 0.0;
                if (F == 0.0) {
                    double A1 = (model == ORC_PSF_GAUSS) ? 1.0 / (2.0 * M_PI * sx * sy)
                                                        : (beta - 1.0) / (M_PI * sx * sy);
                    J[2] = (model == ORC_PSF_GAUSS) ? A1 * exp(-0.5 * q) : A1 * pow(1.0 + q, -beta);
                }
                J[3] = 1.0;
                J[4] = -P / sx + dPdq * (-2.0 * u * u / (sx * sx * sx));
                J[5] = -P / sy + dPdq * (-2.0 * v * v / (sy * sy * sy));
                /* du/dtheta = v, dv/dtheta = -u */
                J[6] = dPdq * (dqdu * v + dqdv * (-u));
            }
        }
    return ORC_OK;
}

/* Default start (paper-silent reading): centre of the stamp, sky = median of
 * the border pixels, F = sum(stamp - sky), sx = 1.6, sy = 1.4, theta = 0.  The
 * widths start slightly unequal: with sx = sy the angle has zero gradient and a
 * source elongated at 45 degrees would never leave the circular saddle. */
int orc_psf_init(const float* st, int32_t S, double* p7) {
    double* b = (double*)calloc((size_t)S * (size_t)S + 1, sizeof(double));
    int32_t nb = 0;
    for (int32_t i = 0; i < S; i++)
        for (int32_t j = 0; j < S; j++)
            if (i == 0 || j == 0 || i == S - 1 || j == S - 1) b[nb++] = (double)st[i * S + j];
    double sk = median_of(b, nb);
    double f = 0.0;
    for (int32_t k = 0; k < S * S; k++) f += (double)st[k] - sk;
    free(b);
    p7[0] = 0.5 * (S - 1); p7[1] = 0.5 * (S - 1); p7[2] = f; p7[3] = sk;
    p7[4] = 1.6; p7[5] = 1.4; p7[6] = 0.0;
    return ORC_OK;
}

/* Cholesky solve of the 7 x 7 system A x = b in FP64; 0 if A is not
 * positive definite. */
static int chol7(const double A[49], const double b[7], double x[7]) {
    double L[49] = {0};
    for (int i = 0; i < 7; i++)
        for (int j = 0; j <= i; j++) {
            double s = A[i * 7 + j];
            for (int k = 0; k < j; k++) s -= L[i * 7 + k] * L[j * 7 + k];
            if (i == j) {
                if (!(s > 0.0)) return 0;
                L[i * 7 + i] = sqrt(s);
            } else {
                L[i * 7 + j] = s / L[j * 7 + j];
            }
        }
    double z[7];
    for (int i = 0; i < 7; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= L[i * 7 + k] * z[k];
        z[i] = s / L[i * 7 + i];
    }
    for (int i = 6; i >= 0; i--) {
        double s = z[i];
        for (int k = i + 1; k < 7; k++) s -= L[k * 7 + i] * x[k];
        x[i] = s / L[i * 7 + i];
    }
    return 1;
}

static double chi2_of(const float* d, const float* w, const double* m, int64_t n) {
    double c = 0.0;
    for (int64_t k = 0; k < n; k++) {
        double r = (double)d[k] - m[k];
        c += (w ? (double)w[k] : 1.0) * r * r;
    }
    return c;
}

/* sum of w (m - sky)^2: the weighted square of the star part of the model */
static double star_sq_of(const float* w, const double* m, double sky, int64_t n) {
    double c = 0.0;
    for (int64_t k = 0; k < n; k++) c += (w ? (double)w[k] : 1.0) * (m[k] - sky) * (m[k] - sky);
    return c;
}

/*
 * Levenberg-Marquardt (Marquardt 1963, diagonal scaling), one trial step per
 * iteration: solve (J'WJ + lambda D) delta = J'W r by Cholesky, D = diag(J'WJ)
 * with entries floored at 1e-9 of the largest; the
 * trial is accepted when chi^2 drops (lambda /= 10), otherwise rejected
 * (lambda *= 10); trials with sx or sy <= 0.05 or a non-positive-definite
 * system are rejected.  Converged, before a trial, when the Gauss-Newton
 * decrease g'(J'WJ)^-1 g (g = J'W r) is at most 1e-10 chi^2 + 1e-12 sum w
 * (m - sky)^2: the first term bounds the distance to the optimum by
 * 1.5e-4 standard errors per parameter, sqrt(1e-10 (n - 7)), the second is
 * the decrease that rounding of a single-precision model (relative error
 * ~2^-22) can fake, so that the rule can be decided in that precision too.
 * It does not depend on lambda.  Also
 * converged when lambda passes 1e10 (no step lowers chi^2; FIT_SINGULAR if
 * that came from failed factorisations); otherwise stops after max_iter
 * trials with FIT_MAXITER.  Result
 * canonicalised: sx >= sy (swap and add pi/2 to theta), theta wrapped to
 * [-pi/2, pi/2).
 */
int orc_psf_fit(const float* stamps, int64_t N, int32_t S, const float* weights,
                const float* init, int32_t model, double beta, int32_t max_iter,
                double lambda0, double* params, double* chi2, int32_t* iters,
                int32_t* flags) {
    int64_t np = (int64_t)S * S;
#pragma omp parallel
    {
    double* m = (double*)malloc(sizeof(double) * (size_t)np);
    double* J = (double*)malloc(sizeof(double) * (size_t)np * 7);
#pragma omp for schedule(dynamic, 16)
    for (int64_t s = 0; s < N; s++) {
        const float* d = stamps + s * np;
        const float* w = weights ? weights + s * np : NULL;
        double p[7], pt[7];
        if (init) for (int k = 0; k < 7; k++) p[k] = (double)init[s * 7 + k];
        else orc_psf_init(d, S, p);
        double lam = lambda0;
        orc_psf_model(p, S, model, beta, m, J);
        double c2 = chi2_of(d, w, m, np), sm2 = star_sq_of(w, m, p[3], np);
        int32_t fl = ORC_FLAG_FIT_MAXITER, it, nsing = 0;
        double Hm[49], g[7];
        int need = 1;
        for (it = 0; it < max_iter; it++) {
            if (need) {
                orc_psf_model(p, S, model, beta, m, J);
                for (int a = 0; a < 49; a++) Hm[a] = 0.0;
                for (int a = 0; a < 7; a++) g[a] = 0.0;
                for (int64_t k = 0; k < np; k++) {
                    double wk = w ? (double)w[k] : 1.0;
                    double r = (double)d[k] - m[k];
                    for (int a = 0; a < 7; a++) {
                        g[a] += wk * J[7 * k + a] * r;
                        for (int b = 0; b <= a; b++) Hm[a * 7 + b] += wk * J[7 * k + a] * J[7 * k + b];
                    }
                }
                for (int a = 0; a < 7; a++)
                    for (int b = a + 1; b < 7; b++) Hm[a * 7 + b] = Hm[b * 7 + a];
                need = 0;
            }
            double A[49], delta[7], dmax = 0.0;
            memcpy(A, Hm, sizeof(A));
            for (int a = 0; a < 7; a++) dmax = fmax(dmax, Hm[a * 7 + a]);
            /* Marquardt scaling by diag(J'WJ), each entry floored at 1e-9 of the
             * largest so that a parameter with no gradient stays damped */
            for (int a = 0; a < 7; a++) A[a * 7 + a] += lam * fmax(Hm[a * 7 + a], 1e-9 * dmax);
            if (!chol7(A, g, delta)) {
                lam *= 10.0; nsing++;
                if (lam > 1e10) { it++; break; }
                continue;
            }
            {
                /* the damped step's decrease never exceeds the Gauss-Newton one, so the
                 * undamped system is solved only when the damped one is already small */
                const double thr = 1e-10 * c2 + 1e-12 * sm2;
                double dec = 0.0;
                for (int a = 0; a < 7; a++) dec += g[a] * delta[a];
                if (dec <= thr) {
                    double A0[49], dgn[7];
                    memcpy(A0, Hm, sizeof(A0));
                    if (chol7(A0, g, dgn)) {
                        double dgnv = 0.0;
                        for (int a = 0; a < 7; a++) dgnv += g[a] * dgn[a];
                        if (dgnv <= thr) { fl = 0; break; }
                    }
                }
            }
            for (int a = 0; a < 7; a++) pt[a] = p[a] + delta[a];
            if (!(pt[4] > 0.05) || !(pt[5] > 0.05)) {
                lam *= 10.0;
                if (lam > 1e10) { fl = 0; it++; break; }
                continue;
            }
            orc_psf_model(pt, S, model, beta, m, NULL);
            double c2t = chi2_of(d, w, m, np);
            if (c2t < c2) {
                memcpy(p, pt, sizeof(p));
                c2 = c2t;
                sm2 = star_sq_of(w, m, p[3], np);
                lam /= 10.0;
                need = 1;
            } else {
                lam *= 10.0;
                if (lam > 1e10) { fl = 0; it++; break; }   /* no step lowers chi^2: at the minimum */
            }
        }
        if (nsing > 0 && fl) fl |= ORC_FLAG_FIT_SINGULAR;
        if (!(p[4] > 0.05) || !(p[5] > 0.05)) fl |= ORC_FLAG_FIT_BAD_SIGMA;
        if (p[4] < p[5]) { double t = p[4]; p[4] = p[5]; p[5] = t; p[6] += 0.5 * M_PI; }
        p[6] = p[6] - M_PI * floor((p[6] + 0.5 * M_PI) / M_PI);
        for (int k = 0; k < 7; k++) params[s * 7 + k] = p[k];
        chi2[s] = c2; iters[s] = it; flags[s] = fl;
    }
    free(m); free(J);
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Image alignment (Sec. 2.2.3): pixel -> sky -> pixel coordinate mapping
 * (Eqs. 5-7 and their inverses), the partial affine (similarity) estimate, and
 * bilinear reprojection.  Readings:
 *   pixel (column j, row i), 0-based, is FITS pixel (j + 1, i + 1);
 *   Eq. 5 is the SIP distortion applied to the offsets from the reference pixel,
 *     u = x - CRPIX1, v = y - CRPIX2:  xi = u + sum A_pq u^p v^q,
 *     eta = v + sum B_pq u^p v^q  (p + q <= order, every given term);
 *   Eq. 6 maps (xi, eta) through CD (degrees per pixel) to the standard
 *     coordinates (in radians below);
 *   Eq. 7 is the gnomonic (TAN) deprojection about (CRVAL1, CRVAL2);
 *   the inverse chain inverts Eq. 7 (the gnomonic projection about the target's
 *   CRVAL; points at or beyond 90 degrees from it have no image: NaN), Eq. 6
 *   (CD^-1) and Eq. 5 (Newton's method from (xi, eta), at most 50 steps, until
 *   the step is below 1e-12 px; not converged: NaN).
 * ------------------------------------------------------------------------- */
static const double ORC_D2R = M_PI / 180.0;

static void sip_eval(const double* c, int order, double u, double v, double* val, double* du, double* dv) {
    /* sum c[p*6+q] u^p v^q over p + q <= order, and its partial derivatives */
    double s = 0.0, su = 0.0, sv = 0.0;
    for (int p = 0; p <= order; p++) {
        for (int q = 0; q <= order - p; q++) {
            const double k = c[p * 6 + q];
            if (k == 0.0) continue;
            s += k * pow(u, p) * pow(v, q);
            if (p > 0) su += k * p * pow(u, p - 1) * pow(v, q);
            if (q > 0) sv += k * q * pow(u, p) * pow(v, q - 1);
        }
    }
    *val = s;
    if (du) *du = su;
    if (dv) *dv = sv;
}

int orc_wcs_pix2world(const orc_wcs* w, const double* x, const double* y, int64_t n, double* ra, double* dec) {
    const double a0 = w->crval[0] * ORC_D2R, d0 = w->crval[1] * ORC_D2R;
    for (int64_t k = 0; k < n; k++) {
        const double u = x[k] + 1.0 - w->crpix[0], v = y[k] + 1.0 - w->crpix[1];
        double f, g;
        sip_eval(w->a, w->a_order, u, v, &f, NULL, NULL);
        sip_eval(w->b, w->b_order, u, v, &g, NULL, NULL);
        const double xi = u + f, eta = v + g;                                   /* Eq. 5 */
        const double p = (w->cd[0] * xi + w->cd[1] * eta) * ORC_D2R;           /* Eq. 6 */
        const double q = (w->cd[2] * xi + w->cd[3] * eta) * ORC_D2R;
        const double den = cos(d0) - q * sin(d0);                               /* Eq. 7 */
        double al = a0 + atan2(p, den);
        al = fmod(al, 2.0 * M_PI);
        if (al < 0.0) al += 2.0 * M_PI;
        ra[k] = al / ORC_D2R;
        dec[k] = atan2(q * cos(d0) + sin(d0), sqrt(p * p + den * den)) / ORC_D2R;
    }
    return ORC_OK;
}

int orc_wcs_world2pix(const orc_wcs* w, const double* ra, const double* dec, int64_t n, double* x, double* y) {
    const double a0 = w->crval[0] * ORC_D2R, d0 = w->crval[1] * ORC_D2R;
    const double det = w->cd[0] * w->cd[3] - w->cd[1] * w->cd[2];
    if (det == 0.0) return ORC_INVALID_ARG;
    for (int64_t k = 0; k < n; k++) {
        const double al = ra[k] * ORC_D2R, de = dec[k] * ORC_D2R;
        /* inverse of Eq. 7: gnomonic projection about (a0, d0) */
        const double cc = sin(d0) * sin(de) + cos(d0) * cos(de) * cos(al - a0);
        if (!(cc > 0.0)) { x[k] = NAN; y[k] = NAN; continue; }
        const double p = cos(de) * sin(al - a0) / cc / ORC_D2R;
        const double q = (cos(d0) * sin(de) - sin(d0) * cos(de) * cos(al - a0)) / cc / ORC_D2R;
        /* inverse of Eq. 6 */
        const double xi = (w->cd[3] * p - w->cd[1] * q) / det;
        const double eta = (-w->cd[2] * p + w->cd[0] * q) / det;
        /* inverse of Eq. 5: Newton on (u + f(u, v) - xi, v + g(u, v) - eta) */
        double u = xi, v = eta;
        int ok = 0;
        for (int it = 0; it < 50; it++) {
            double f, fu, fv, g, gu, gv;
            sip_eval(w->a, w->a_order, u, v, &f, &fu, &fv);
            sip_eval(w->b, w->b_order, u, v, &g, &gu, &gv);
            const double r1 = u + f - xi, r2 = v + g - eta;
            const double j11 = 1.0 + fu, j12 = fv, j21 = gu, j22 = 1.0 + gv;
            const double dj = j11 * j22 - j12 * j21;
            if (dj == 0.0) break;
            const double su = (j22 * r1 - j12 * r2) / dj, sv = (-j21 * r1 + j11 * r2) / dj;
            u -= su;
            v -= sv;
            if (fabs(su) < 1e-12 && fabs(sv) < 1e-12) { ok = 1; break; }
        }
        if (!ok) { x[k] = NAN; y[k] = NAN; continue; }
        x[k] = u + w->crpix[0] - 1.0;
        y[k] = v + w->crpix[1] - 1.0;
    }
    return ORC_OK;
}

/* Source pixel -> target pixel on the node grid (j step, i step), j step <= W - 1,
 * i step <= H - 1 (the paper maps every pixel: step 1).  Row-major nodes. */
int orc_wcs_map(const orc_wcs* src, const orc_wcs* tgt, int64_t W, int64_t H, int32_t step, double* xo,
                double* yo) {
    if (step < 1 || W < 1 || H < 1) return ORC_INVALID_ARG;
    const int64_t nx = (W - 1) / step + 1, ny = (H - 1) / step + 1;
    for (int64_t i = 0; i < ny; i++) {
        for (int64_t j = 0; j < nx; j++) {
            const double x = (double)(j * step), y = (double)(i * step);
            double ra, de;
            orc_wcs_pix2world(src, &x, &y, 1, &ra, &de);
            int e = orc_wcs_world2pix(tgt, &ra, &de, 1, &xo[i * nx + j], &yo[i * nx + j]);
            if (e) return e;
        }
    }
    return ORC_OK;
}

/* Partial affine (similarity: rotation, one scale, translation) least-squares
 * estimate from point pairs (x, y) -> (xt, yt), the model of the OpenCV routine
 * the paper names (read without its outlier rejection: correspondences from a
 * WCS mapping have no outliers).  Closed form about the centroids:
 *   a = s cos t = sum(dx dxt + dy dyt) / sum(dx^2 + dy^2),
 *   b = s sin t = sum(dx dyt - dy dxt) / sum(dx^2 + dy^2),
 *   M = [a -b tx; b a ty], (tx, ty) = centroid_t - [a -b; b a] centroid.
 * Pairs with a non-finite member are skipped.  Minv is the inverse map.
 * Returns INVALID_ARG with fewer than two distinct points. */
int orc_affine_fit(const double* x, const double* y, const double* xt, const double* yt, int64_t n, double* M,
                   double* Minv) {
    double sx = 0, sy = 0, stx = 0, sty = 0;
    int64_t m = 0;
    for (int64_t k = 0; k < n; k++) {
        if (!isfinite(x[k]) || !isfinite(y[k]) || !isfinite(xt[k]) || !isfinite(yt[k])) continue;
        sx += x[k]; sy += y[k]; stx += xt[k]; sty += yt[k];
        m++;
    }
    if (m < 2) return ORC_INVALID_ARG;
    const double cx = sx / m, cy = sy / m, ctx = stx / m, cty = sty / m;
    double saa = 0, sa = 0, sb = 0;
    for (int64_t k = 0; k < n; k++) {
        if (!isfinite(x[k]) || !isfinite(y[k]) || !isfinite(xt[k]) || !isfinite(yt[k])) continue;
        const double dx = x[k] - cx, dy = y[k] - cy, ex = xt[k] - ctx, ey = yt[k] - cty;
        saa += dx * dx + dy * dy;
        sa += dx * ex + dy * ey;
        sb += dx * ey - dy * ex;
    }
    if (!(saa > 0.0)) return ORC_INVALID_ARG;
    const double a = sa / saa, b = sb / saa;
    M[0] = a; M[1] = -b; M[2] = ctx - (a * cx - b * cy);
    M[3] = b; M[4] = a;  M[5] = cty - (b * cx + a * cy);
    const double s2 = a * a + b * b;
    if (!(s2 > 0.0)) return ORC_INVALID_ARG;
    /* inverse of [a -b; b a] is [a b; -b a] / s2 */
    Minv[0] = a / s2;  Minv[1] = b / s2;  Minv[2] = -(Minv[0] * M[2] + Minv[1] * M[5]);
    Minv[3] = -b / s2; Minv[4] = a / s2;  Minv[5] = -(Minv[3] * M[2] + Minv[4] * M[5]);
    return ORC_OK;
}

/* Reprojection (Sec. 2.2.3): output pixel (j, i) of a Wo x Ho frame takes the
 * source value at (x, y) = Minv (j, i, 1), by bilinear interpolation between the
 * four surrounding pixel centres.  Defined on 0 <= x <= W - 1, 0 <= y <= H - 1
 * (at x = W - 1 the right-hand pair has weight 0 and is not read); elsewhere, or
 * when a weighted neighbour is not finite, the output is `fill`. */
int orc_reproject_affine(const float* src, int64_t W, int64_t H, const double* Minv, int64_t Wo, int64_t Ho,
                         double fill, double* out) {
    for (int64_t i = 0; i < Ho; i++) {
        for (int64_t j = 0; j < Wo; j++) {
            const double x = Minv[0] * j + Minv[1] * i + Minv[2];
            const double y = Minv[3] * j + Minv[4] * i + Minv[5];
            double r = fill;
            if (x >= 0.0 && x <= (double)(W - 1) && y >= 0.0 && y <= (double)(H - 1)) {
                int64_t x0 = (int64_t)floor(x), y0 = (int64_t)floor(y);
                if (x0 > W - 2) x0 = W - 2 < 0 ? 0 : W - 2;
                if (y0 > H - 2) y0 = H - 2 < 0 ? 0 : H - 2;
                const double t = x - x0, s = y - y0;
                double acc = 0.0;
                int bad = 0;
                for (int dy = 0; dy <= 1; dy++) {
                    for (int dx = 0; dx <= 1; dx++) {
                        const double wgt = (dx ? t : 1.0 - t) * (dy ? s : 1.0 - s);
                        if (wgt == 0.0) continue;
                        const int64_t xx = x0 + dx, yy = y0 + dy;
                        if (xx >= W || yy >= H) { bad = 1; continue; }
                        const double v = (double)src[yy * W + xx];
                        if (!isfinite(v)) bad = 1;
                        acc += wgt * v;
                    }
                }
                r = bad ? fill : acc;
            }
            out[i * Wo + j] = r;
        }
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * ZScale display limits (Sec. 2.2.6 names SAOimage's zscale; reading after the
 * published IRAF algorithm):
 *   samples: up to n_samples pixels at flat (row-major) indices k * stride,
 *     stride = max(1, W H / n_samples), non-finite ones dropped; sorted;
 *   npix samples s_0 <= ... ; zmin = s_0, zmax = s_{npix-1}; c = (npix - 1) / 2
 *     (integer); median = s_c (npix odd) or (s_c + s_{c+1}) / 2;
 *   minpix = max(5, (int)(0.5 npix)); rejections grow by h = max(1, (int)(0.01
 *     npix)) / 2 samples on each side;
 *   iteration (at most max_iter): stop when ngood >= the previous ngood or
 *     ngood < minpix; least-squares line of s_k against x_k = k - c over the
 *     good samples; flat_k = s_k - (slope x_k + intercept) for every sample;
 *     sigma = population standard deviation of flat over the good samples;
 *     a sample is rejected when |flat| > krej sigma; a sample is good when no
 *     rejected sample lies within h of it; ngood = the number of good samples;
 *   limits: with ngood >= minpix, z1 = max(zmin, median - (c - 1) slope /
 *     contrast), z2 = min(zmax, median + (npix - c) slope / contrast); otherwise
 *     (zmin, zmax).  No finite sample: INVALID_ARG.
 * ------------------------------------------------------------------------- */
static int cmp_f(const void* a, const void* b) {
    const float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

int orc_zscale(const float* img, int64_t W, int64_t H, int32_t n_samples, double contrast, double krej,
               int32_t max_iter, double* z, int32_t* counts) {
    if (W < 1 || H < 1 || n_samples < 1 || !(contrast > 0.0) || !(krej > 0.0) || max_iter < 0) return ORC_INVALID_ARG;
    const int64_t N = W * H;
    int64_t stride = N / n_samples;
    if (stride < 1) stride = 1;
    float* s = (float*)malloc(sizeof(float) * (size_t)n_samples);
    int64_t npix = 0;
    for (int64_t k = 0; k < n_samples && k * stride < N; k++) {
        const float v = img[k * stride];
        if (isfinite(v)) s[npix++] = v;
    }
    if (npix == 0) { free(s); return ORC_INVALID_ARG; }
    qsort(s, (size_t)npix, sizeof(float), cmp_f);
    const double zmin = s[0], zmax = s[npix - 1];
    const int64_t c = (npix - 1) / 2;
    const double median = (npix & 1) ? (double)s[c] : 0.5 * ((double)s[c] + (double)s[c + 1]);
    int64_t minpix = (int64_t)(0.5 * (double)npix);
    if (minpix < 5) minpix = 5;
    int64_t ngrow = (int64_t)(0.01 * (double)npix);
    if (ngrow < 1) ngrow = 1;
    const int64_t h = ngrow / 2;
    unsigned char* good = (unsigned char*)malloc((size_t)npix);
    unsigned char* bad = (unsigned char*)malloc((size_t)npix);
    double* flat = (double*)malloc(sizeof(double) * (size_t)npix);
    for (int64_t k = 0; k < npix; k++) good[k] = 1;
    int64_t ngood = npix, last = npix + 1;
    double slope = 0.0;
    for (int it = 0; it < max_iter; it++) {
        if (ngood >= last || ngood < minpix) break;
        /* least-squares line over the good samples */
        double n = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
        for (int64_t k = 0; k < npix; k++) {
            if (!good[k]) continue;
            const double x = (double)(k - c), y = s[k];
            n += 1.0; sx += x; sy += y; sxx += x * x; sxy += x * y;
        }
        const double den = n * sxx - sx * sx;
        slope = den != 0.0 ? (n * sxy - sx * sy) / den : 0.0;
        const double icpt = (sy - slope * sx) / n;
        for (int64_t k = 0; k < npix; k++) flat[k] = (double)s[k] - (slope * (double)(k - c) + icpt);
        double m = 0.0;
        for (int64_t k = 0; k < npix; k++) if (good[k]) m += flat[k];
        m /= n;
        double v = 0.0;
        for (int64_t k = 0; k < npix; k++) if (good[k]) v += (flat[k] - m) * (flat[k] - m);
        const double thr = krej * sqrt(v / n);
        for (int64_t k = 0; k < npix; k++) bad[k] = (flat[k] < -thr) || (flat[k] > thr);
        last = ngood;
        ngood = 0;
        for (int64_t k = 0; k < npix; k++) {
            int ok = 1;
            for (int64_t j = k - h; j <= k + h; j++)
                if (j >= 0 && j < npix && bad[j]) { ok = 0; break; }
            good[k] = (unsigned char)ok;
            ngood += ok;
        }
    }
    if (ngood >= minpix) {
        const double sl = slope / contrast;
        const double a = median - (double)(c - 1) * sl, b = median + (double)(npix - c) * sl;
        z[0] = a > zmin ? a : zmin;
        z[1] = b < zmax ? b : zmax;
    } else {
        z[0] = zmin;
        z[1] = zmax;
    }
    if (counts) { counts[0] = (int32_t)npix; counts[1] = (int32_t)ngood; }
    free(s); free(good); free(bad); free(flat);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Image subtraction (Sec. 2.2.4, HOTPANTS-style: Eqs. 8-10).  Readings:
 *   basis (Eq. 9): for each Gaussian k (width sig_k, degree deg_k) and every
 *     i + j <= deg_k (i outer, j inner), K_n(u, v) = exp(-(u^2 + v^2) /
 *     (2 sig_k^2)) u^i v^j on -hw <= u, v <= hw, stored row-major by v then u;
 *   convolution: (R (x) K)(x, y) = sum_{u,v} K(u, v) R(x - u, y - v);
 *   spatial terms: xs = 2x / (W - 1) - 1, ys = 2y / (H - 1) - 1 (0 for a single
 *     column or row); terms xs^p ys^q, p outer, q inner, p + q <= order;
 *   Eq. 8: a_n(x, y) = sum_s c_{n,s} P_s(x, y); Eq. 10 read as the model
 *     I + B = R (x) K with B(x, y) = sum_b d_b P_b(x, y) (background order);
 *   stamps: the frame is cut into nsx x nsy regions; in each, the brightest
 *     template pixel whose fit footprint (2 fh + 1)^2 and convolution support
 *     (2 (fh + hw) + 1)^2 lie inside the frame and are finite in R and I is a
 *     candidate when it exceeds the region's median by nsig robust sigmas
 *     (1.4826 MAD over the region's finite pixels);
 *   fit: unweighted least squares over every footprint pixel of every
 *     candidate, the kernel's spatial terms taken at the candidate's centre
 *     (constant over a footprint) and the background's at each pixel; normal
 *     equations in FP64, Cholesky;
 *   apply: the kernel is evaluated at the centre of each tile x tile block of
 *     the output (the paper's stamp-per-block convolution) and convolved with R
 *     for the block's pixels; D = I + B - R (x) K where the whole kernel support
 *     lies inside the frame, NaN elsewhere.
 * ------------------------------------------------------------------------- */
static int sub_nbasis(const int32_t* deg, int32_t nk) {
    int nb = 0;
    for (int k = 0; k < nk; k++) nb += (deg[k] + 1) * (deg[k] + 2) / 2;
    return nb;
}

int orc_sub_basis(int32_t hw, const double* sig, const int32_t* deg, int32_t nk, double* out) {
    if (hw < 0 || nk < 1) return -1;
    const int S = 2 * hw + 1;
    int n = 0;
    for (int k = 0; k < nk; k++) {
        if (!(sig[k] > 0.0) || deg[k] < 0) return -1;
        for (int i = 0; i <= deg[k]; i++) {
            for (int j = 0; j <= deg[k] - i; j++) {
                for (int v = -hw; v <= hw; v++) {
                    for (int u = -hw; u <= hw; u++) {
                        const double g = exp(-(double)(u * u + v * v) / (2.0 * sig[k] * sig[k]));
                        out[(int64_t)n * S * S + (v + hw) * S + (u + hw)] = g * pow((double)u, i) * pow((double)v, j);
                    }
                }
                n++;
            }
        }
    }
    return n;
}

static int sub_nterms(int order) { return (order + 1) * (order + 2) / 2; }

static void sub_terms(double x, double y, int64_t W, int64_t H, int order, double* t) {
    const double xs = W > 1 ? 2.0 * x / (double)(W - 1) - 1.0 : 0.0;
    const double ys = H > 1 ? 2.0 * y / (double)(H - 1) - 1.0 : 0.0;
    int n = 0;
    for (int p = 0; p <= order; p++)
        for (int q = 0; q <= order - p; q++) t[n++] = pow(xs, p) * pow(ys, q);
}

static int cmp_d(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double median_d(double* v, int64_t n) {
    qsort(v, (size_t)n, sizeof(double), cmp_d);
    return (n & 1) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

int orc_sub_stamps(const float* I, const float* R, int64_t W, int64_t H, int32_t nsx, int32_t nsy, int32_t hw,
                   int32_t fh, double nsig, int32_t* cx, int32_t* cy) {
    if (nsx < 1 || nsy < 1 || hw < 0 || fh < 0) return -1;
    const int64_t m = (int64_t)fh + hw;
    int nc = 0;
    double* buf = (double*)malloc(sizeof(double) * (size_t)(W * H / ((int64_t)nsx * nsy) + W + H + 16));
    for (int sy = 0; sy < nsy; sy++) {
        for (int sx = 0; sx < nsx; sx++) {
            const int64_t x0 = sx * W / nsx, x1 = (sx + 1) * W / nsx, y0 = sy * H / nsy, y1 = (sy + 1) * H / nsy;
            int64_t n = 0;
            for (int64_t y = y0; y < y1; y++)
                for (int64_t x = x0; x < x1; x++)
                    if (isfinite(R[y * W + x])) buf[n++] = R[y * W + x];
            if (n == 0) continue;
            const double med = median_d(buf, n);
            for (int64_t k = 0; k < n; k++) buf[k] = fabs(buf[k] - med);
            const double sgm = 1.4826 * median_d(buf, n);
            /* brightest eligible pixel, first in row-major order among equals */
            double best = -INFINITY;
            int64_t bx = -1, by = -1;
            for (int64_t y = y0; y < y1; y++) {
                for (int64_t x = x0; x < x1; x++) {
                    if (x < m || y < m || x > W - 1 - m || y > H - 1 - m) continue;
                    const double v = R[y * W + x];
                    if (!(v > best)) continue;
                    int ok = 1;
                    for (int64_t yy = y - m; yy <= y + m && ok; yy++)
                        for (int64_t xx = x - m; xx <= x + m; xx++)
                            if (!isfinite(R[yy * W + xx])) { ok = 0; break; }
                    for (int64_t yy = y - fh; yy <= y + fh && ok; yy++)
                        for (int64_t xx = x - fh; xx <= x + fh; xx++)
                            if (!isfinite(I[yy * W + xx])) { ok = 0; break; }
                    if (!ok) continue;
                    best = v; bx = x; by = y;
                }
            }
            if (bx >= 0 && best > med + nsig * sgm) {
                cx[nc] = (int32_t)bx;
                cy[nc] = (int32_t)by;
                nc++;
            }
        }
    }
    free(buf);
    return nc;
}

/* Cholesky solve of the SPD system A x = b (n x n, row-major, overwritten) */
static int chol_solve(double* A, double* b, int n) {
    for (int j = 0; j < n; j++) {
        double d = A[j * n + j];
        for (int k = 0; k < j; k++) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[j * n + j] = d;
        for (int i = j + 1; i < n; i++) {
            double s = A[i * n + j];
            for (int k = 0; k < j; k++) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / d;
        }
    }
    for (int i = 0; i < n; i++) {            /* L y = b */
        double s = b[i];
        for (int k = 0; k < i; k++) s -= A[i * n + k] * b[k];
        b[i] = s / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; i--) {       /* L' x = y */
        double s = b[i];
        for (int k = i + 1; k < n; k++) s -= A[k * n + i] * b[k];
        b[i] = s / A[i * n + i];
    }
    return 0;
}

/* The Cholesky solve above as an entry point (A and b overwritten: L and x);
 * ORC_INVALID_ARG when a pivot is not positive. */
int orc_chol_solve(double* A, double* b, int32_t n) {
    if (n < 1) return ORC_INVALID_ARG;
    return chol_solve(A, b, n) ? ORC_INVALID_ARG : ORC_OK;
}

/* Normal equations of the fit: AtA (np x np, full, row-major) and Atb (np), the
 * unknowns ordered as the coefficients below; the design row of footprint pixel
 * p of candidate c is [C_n(p) P_s(c) for n, s] then [-P_b(p) for b], its target
 * I(p), C_n = R (x) K_n. */
int orc_sub_normal(const float* I, const float* R, int64_t W, int64_t H, const int32_t* cx, const int32_t* cy,
                   int32_t nc, int32_t hw, int32_t fh, const double* sig, const int32_t* deg, int32_t nk,
                   int32_t sord, int32_t bord, double* AtA, double* Atb) {
    if (nc < 1 || sord < 0 || bord < -1) return ORC_INVALID_ARG;
    const int S = 2 * hw + 1, nb = sub_nbasis(deg, nk), ns = sub_nterms(sord), ng = bord >= 0 ? sub_nterms(bord) : 0;
    const int np = nb * ns + ng;
    double* K = (double*)malloc(sizeof(double) * (size_t)nb * S * S);
    if (orc_sub_basis(hw, sig, deg, nk, K) != nb) { free(K); return ORC_INVALID_ARG; }
    for (int64_t k = 0; k < (int64_t)np * np; k++) AtA[k] = 0.0;
    for (int k = 0; k < np; k++) Atb[k] = 0.0;
    double* row = (double*)malloc(sizeof(double) * (size_t)np);
    double* C = (double*)malloc(sizeof(double) * (size_t)nb);
    double Ps[64], Pb[64];
    for (int c = 0; c < nc; c++) {
        sub_terms((double)cx[c], (double)cy[c], W, H, sord, Ps);
        for (int dv = -fh; dv <= fh; dv++) {
            for (int du = -fh; du <= fh; du++) {
                const int64_t x = cx[c] + du, y = cy[c] + dv;
                for (int n = 0; n < nb; n++) {            /* (R (x) K_n)(x, y) */
                    double s = 0.0;
                    for (int v = -hw; v <= hw; v++)
                        for (int u = -hw; u <= hw; u++)
                            s += K[(int64_t)n * S * S + (v + hw) * S + (u + hw)] * (double)R[(y - v) * W + (x - u)];
                    C[n] = s;
                }
                for (int n = 0; n < nb; n++)
                    for (int t = 0; t < ns; t++) row[n * ns + t] = C[n] * Ps[t];
                if (ng) {
                    sub_terms((double)x, (double)y, W, H, bord, Pb);
                    for (int t = 0; t < ng; t++) row[nb * ns + t] = -Pb[t];
                }
                const double target = I[y * W + x];
                for (int a = 0; a < np; a++) {
                    Atb[a] += row[a] * target;
                    for (int b = 0; b <= a; b++) AtA[(int64_t)a * np + b] += row[a] * row[b];
                }
            }
        }
    }
    for (int a = 0; a < np; a++)
        for (int b = a + 1; b < np; b++) AtA[(int64_t)a * np + b] = AtA[(int64_t)b * np + a];
    free(K); free(row); free(C);
    return ORC_OK;
}

/* coef: [nb * ns] kernel coefficients c_{n,s} (n outer), then [nbg] background d_b:
 * the solution of the normal equations above by Cholesky */
int orc_sub_fit(const float* I, const float* R, int64_t W, int64_t H, const int32_t* cx, const int32_t* cy,
                int32_t nc, int32_t hw, int32_t fh, const double* sig, const int32_t* deg, int32_t nk, int32_t sord,
                int32_t bord, double* coef) {
    if (nc < 1 || sord < 0 || bord < -1) return ORC_INVALID_ARG;
    const int nb = sub_nbasis(deg, nk), ns = sub_nterms(sord), ng = bord >= 0 ? sub_nterms(bord) : 0;
    const int np = nb * ns + ng;
    double* AtA = (double*)malloc(sizeof(double) * (size_t)np * np);
    double* Atb = (double*)malloc(sizeof(double) * (size_t)np);
    int e = orc_sub_normal(I, R, W, H, cx, cy, nc, hw, fh, sig, deg, nk, sord, bord, AtA, Atb);
    if (!e) e = chol_solve(AtA, Atb, np) ? ORC_INVALID_ARG : ORC_OK;
    if (!e) memcpy(coef, Atb, sizeof(double) * (size_t)np);
    free(AtA); free(Atb);
    return e;
}

int orc_sub_apply(const float* I, const float* R, int64_t W, int64_t H, int32_t hw, const double* sig,
                  const int32_t* deg, int32_t nk, int32_t sord, int32_t bord, const double* coef, int32_t tile,
                  double* D) {
    if (tile < 1) return ORC_INVALID_ARG;
    const int S = 2 * hw + 1, nb = sub_nbasis(deg, nk), ns = sub_nterms(sord), ng = bord >= 0 ? sub_nterms(bord) : 0;
    double* K = (double*)malloc(sizeof(double) * (size_t)nb * S * S);
    if (orc_sub_basis(hw, sig, deg, nk, K) != nb) { free(K); return ORC_INVALID_ARG; }
    double* Kt = (double*)malloc(sizeof(double) * (size_t)S * S);
    double Ps[64], Pb[64];
    const int64_t ntx = (W + tile - 1) / tile, nty = (H + tile - 1) / tile;
    for (int64_t ty = 0; ty < nty; ty++) {
        for (int64_t tx = 0; tx < ntx; tx++) {
            /* Eq. 8 at the tile centre */
            sub_terms((double)(tx * tile) + 0.5 * (tile - 1), (double)(ty * tile) + 0.5 * (tile - 1), W, H, sord, Ps);
            for (int k = 0; k < S * S; k++) Kt[k] = 0.0;
            for (int n = 0; n < nb; n++) {
                double a = 0.0;
                for (int t = 0; t < ns; t++) a += coef[n * ns + t] * Ps[t];
                for (int k = 0; k < S * S; k++) Kt[k] += a * K[(int64_t)n * S * S + k];
            }
            for (int64_t y = ty * tile; y < (ty + 1) * tile && y < H; y++) {
                for (int64_t x = tx * tile; x < (tx + 1) * tile && x < W; x++) {
                    if (x < hw || y < hw || x > W - 1 - hw || y > H - 1 - hw) { D[y * W + x] = NAN; continue; }
                    double s = 0.0;
                    for (int v = -hw; v <= hw; v++)
                        for (int u = -hw; u <= hw; u++)
                            s += Kt[(v + hw) * S + (u + hw)] * (double)R[(y - v) * W + (x - u)];
                    double b = 0.0;
                    if (ng) {
                        sub_terms((double)x, (double)y, W, H, bord, Pb);
                        for (int t = 0; t < ng; t++) b += coef[nb * ns + t] * Pb[t];
                    }
                    D[y * W + x] = (double)I[y * W + x] + b - s;
                }
            }
        }
    }
    free(K); free(Kt);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Natural-spline background map (Sec. 2.2.2 scales the filtered mesh back to
 * full resolution by spline interpolation; the Keys cubic above is the default
 * reading, this is the natural cubic spline variant).  Tensor product of 1-D
 * natural cubic splines through the mesh nodes (node (p, q) at pixel
 * ((q + 1/2) mesh_w - 1/2, (p + 1/2) mesh_h - 1/2), unit spacing in node
 * coordinates): second derivatives zero at the end nodes, interior ones from
 * M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}) (Thomas algorithm);
 * beyond the end nodes the spline continues as the line with the end slope (the
 * natural spline's C2 extension).  First along x through each node row, then
 * along y through those values for each pixel column.
 * ------------------------------------------------------------------------- */
static void nspline_m(const double* y, int64_t n, double* M, double* c) {
    /* M[0] = M[n-1] = 0; c: scratch of n doubles */
    for (int64_t k = 0; k < n; k++) M[k] = 0.0;
    if (n < 3) return;
    /* forward sweep on rows k = 1 .. n-2: M_{k-1} + 4 M_k + M_{k+1} = r_k */
    double prev_c = 0.0, prev_d = 0.0;
    for (int64_t k = 1; k <= n - 2; k++) {
        const double r = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]);
        const double den = 4.0 - (k > 1 ? prev_c : 0.0);
        const double ck = 1.0 / den;
        const double dk = (r - (k > 1 ? prev_d : 0.0)) / den;
        c[k] = ck;
        M[k] = dk;
        prev_c = ck;
        prev_d = dk;
    }
    for (int64_t k = n - 3; k >= 1; k--) M[k] -= c[k] * M[k + 1];
}

static double nspline_eval(const double* y, const double* M, int64_t n, double u) {
    if (n == 1) return y[0];
    if (u < 0.0) {
        const double d0 = (y[1] - y[0]) - (2.0 * M[0] + M[1]) / 6.0;
        return y[0] + u * d0;
    }
    if (u > (double)(n - 1)) {
        const double d1 = (y[n - 1] - y[n - 2]) + (M[n - 2] + 2.0 * M[n - 1]) / 6.0;
        return y[n - 1] + (u - (double)(n - 1)) * d1;
    }
    int64_t k = (int64_t)floor(u);
    if (k > n - 2) k = n - 2;
    const double b = u - (double)k, a = 1.0 - b;
    return a * y[k] + b * y[k + 1] + ((a * a * a - a) * M[k] + (b * b * b - b) * M[k + 1]) / 6.0;
}

int orc_spline_map(const float* mesh, int64_t nx, int64_t ny, int32_t mesh_w, int32_t mesh_h, int64_t W, int64_t H,
                   double* out) {
    if (!mesh || !out || nx < 1 || ny < 1 || mesh_w < 1 || mesh_h < 1) return ORC_INVALID_ARG;
    double* rows = (double*)malloc(sizeof(double) * (size_t)(ny * W));   /* row p at each pixel column */
    const int64_t nm = nx > ny ? nx : ny;
    double* y = (double*)malloc(sizeof(double) * (size_t)nm);
    double* M = (double*)malloc(sizeof(double) * (size_t)nm);
    double* c = (double*)malloc(sizeof(double) * (size_t)nm);
    for (int64_t p = 0; p < ny; p++) {
        for (int64_t q = 0; q < nx; q++) y[q] = mesh[p * nx + q];
        nspline_m(y, nx, M, c);
        for (int64_t j = 0; j < W; j++) rows[p * W + j] = nspline_eval(y, M, nx, ((double)j + 0.5) / mesh_w - 0.5);
    }
    for (int64_t j = 0; j < W; j++) {
        for (int64_t p = 0; p < ny; p++) y[p] = rows[p * W + j];
        nspline_m(y, ny, M, c);
        for (int64_t i = 0; i < H; i++) out[i * W + j] = nspline_eval(y, M, ny, ((double)i + 0.5) / mesh_h - 0.5);
    }
    free(rows); free(y); free(M); free(c);
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Cleaning of the deblended objects (Sec. 2.2.5: each object is tested
 * against its neighbours and merged when it does not stand out from them).
 * Reading after SExtractor's cleaning:
 *   per object, from its pixels (sub values f): the peak (largest f, first in
 *     raster order), the barycentre and second moments weighted by max(f, 0)
 *     (1/12 added to x2 and y2 when x2 y2 - xy^2 < 1/144; a footprint with no
 *     positive pixel takes its unweighted centre, x2 = y2 = 1/12, xy = 0);
 *   model of object j: an elliptical Moffat profile peak_j (1 + r^2 / a^2)^-beta,
 *     r^2 = (y2 dx^2 - 2 xy dx dy + x2 dy^2) / (x2 y2 - xy^2) about its
 *     barycentre, a = sqrt(2 ln 2) / sqrt(2^(1/beta) - 1) so that its FWHM is the
 *     FWHM of the Gaussian with the object's moments;
 *   object i is spurious when its peak value minus the models of every brighter
 *     object (larger peak; equal peaks: smaller label) at i's peak pixel is
 *     below the detection threshold there; it is merged into the brighter
 *     object whose model is largest there (ties: smaller label), following
 *     merges to an object that is kept;
 *   kept objects are renumbered 1.. in the order of their labels (a label with
 *     no pixel is no object and takes no number).
 * ------------------------------------------------------------------------- */
/* Per-object statistics of the cleaning test (arrays of nobj + 1, index = label):
 * peak value and its raster index (-1 for an empty label), barycentre and second
 * moments as stated above. */
int orc_clean_stats(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t nobj, double* pk,
                    int64_t* pidx, double* cx, double* cy, double* x2, double* y2, double* xy) {
    if (nobj < 0) return ORC_INVALID_ARG;
    const int64_t n = nobj;
    double *sw = calloc(n + 1, sizeof(double)), *sx = calloc(n + 1, sizeof(double)), *sy = calloc(n + 1, sizeof(double));
    double *sxx = calloc(n + 1, sizeof(double)), *syy = calloc(n + 1, sizeof(double)), *sxy = calloc(n + 1, sizeof(double));
    double *ux = calloc(n + 1, sizeof(double)), *uy = calloc(n + 1, sizeof(double)), *cnt = calloc(n + 1, sizeof(double));
    for (int64_t k = 0; k <= n; k++) { pk[k] = -INFINITY; pidx[k] = -1; }
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++) {
            const int32_t l = labels[i * W + j];
            if (l <= 0 || l > n) continue;
            const double f = sub[i * W + j];
            if (f > pk[l]) { pk[l] = f; pidx[l] = i * W + j; }
            cnt[l] += 1.0; ux[l] += j; uy[l] += i;
            if (f > 0.0) { sw[l] += f; sx[l] += f * j; sy[l] += f * i; }
        }
    }
    for (int64_t l = 0; l <= n; l++) {
        if (l > 0 && sw[l] > 0.0) { cx[l] = sx[l] / sw[l]; cy[l] = sy[l] / sw[l]; }
        else if (l > 0 && cnt[l] > 0.0) { cx[l] = ux[l] / cnt[l]; cy[l] = uy[l] / cnt[l]; }
        else { cx[l] = cy[l] = 0.0; }
    }
    for (int64_t i = 0; i < H; i++) {
        for (int64_t j = 0; j < W; j++) {
            const int32_t l = labels[i * W + j];
            if (l <= 0 || l > n) continue;
            const double f = sub[i * W + j];
            if (!(f > 0.0)) continue;
            const double dx = j - cx[l], dy = i - cy[l];
            sxx[l] += f * dx * dx; syy[l] += f * dy * dy; sxy[l] += f * dx * dy;
        }
    }
    for (int64_t l = 0; l <= n; l++) {
        if (l > 0 && sw[l] > 0.0) {
            x2[l] = sxx[l] / sw[l]; y2[l] = syy[l] / sw[l]; xy[l] = sxy[l] / sw[l];
            if (x2[l] * y2[l] - xy[l] * xy[l] < 1.0 / 144.0) { x2[l] += 1.0 / 12.0; y2[l] += 1.0 / 12.0; }
        } else {
            x2[l] = y2[l] = 1.0 / 12.0; xy[l] = 0.0;
        }
    }
    free(sw); free(sx); free(sy); free(sxx); free(syy); free(sxy); free(ux); free(uy); free(cnt);
    return ORC_OK;
}

int64_t orc_clean(const float* sub, const int32_t* labels, int64_t W, int64_t H, int64_t nobj, const float* thr,
                  double beta, int32_t* out) {
    if (!(beta > 0.0) || nobj < 0) return -1;
    const int64_t n = nobj;
    double* pk = malloc(sizeof(double) * (n + 1));
    int64_t* pidx = malloc(sizeof(int64_t) * (n + 1));
    double *cx = malloc(sizeof(double) * (n + 1)), *cy = malloc(sizeof(double) * (n + 1));
    double *x2 = malloc(sizeof(double) * (n + 1)), *y2 = malloc(sizeof(double) * (n + 1)), *xy = malloc(sizeof(double) * (n + 1));
    orc_clean_stats(sub, labels, W, H, n, pk, pidx, cx, cy, x2, y2, xy);
    const double a2 = 2.0 * log(2.0) / (pow(2.0, 1.0 / beta) - 1.0);
    int64_t* into = malloc(sizeof(int64_t) * (n + 1));
    for (int64_t i = 1; i <= n; i++) {
        into[i] = i;
        if (pidx[i] < 0) continue;
        const double px = (double)(pidx[i] % W), py = (double)(pidx[i] / W);
        double sum = 0.0, best = -1.0;
        int64_t bj = -1;
        for (int64_t j = 1; j <= n; j++) {
            if (j == i || pidx[j] < 0) continue;
            if (!(pk[j] > pk[i] || (pk[j] == pk[i] && j < i))) continue;
            const double dx = px - cx[j], dy = py - cy[j];
            const double det = x2[j] * y2[j] - xy[j] * xy[j];
            const double r2 = (y2[j] * dx * dx - 2.0 * xy[j] * dx * dy + x2[j] * dy * dy) / det;
            const double m = pk[j] * pow(1.0 + r2 / a2, -beta);
            sum += m;
            if (m > best) { best = m; bj = j; }
        }
        if (bj > 0 && pk[i] - sum < (double)thr[pidx[i]]) into[i] = bj;
    }
    /* follow merges to a kept object (targets are strictly brighter: no cycle) */
    int64_t* root = malloc(sizeof(int64_t) * (n + 1));
    for (int64_t i = 1; i <= n; i++) { int64_t r = i; while (into[r] != r) r = into[r]; root[i] = r; }
    int64_t* num = calloc(n + 1, sizeof(int64_t));
    int64_t k = 0;
    for (int64_t i = 1; i <= n; i++) if (root[i] == i && pidx[i] >= 0) num[i] = ++k;  /* an empty label is no object */
    for (int64_t p = 0; p < W * H; p++) {
        const int32_t l = labels[p];
        out[p] = (l <= 0 || l > n) ? 0 : (int32_t)num[root[l]];
    }
    free(pk); free(pidx); free(cx); free(cy); free(x2); free(y2); free(xy); free(into); free(root); free(num);
    return k;
}

/* Node quantities of the same tensor-product spline: second derivatives along x
 * of each node row (Mx), along y of each node column (My), and along y of the Mx
 * columns (Mxy), each [ny][nx].  With the node values they fix the spline
 * between any 2 x 2 nodes. */
int orc_spline_nodes(const float* mesh, int64_t nx, int64_t ny, double* Mx, double* My, double* Mxy) {
    if (!mesh || nx < 1 || ny < 1) return ORC_INVALID_ARG;
    const int64_t nm = nx > ny ? nx : ny;
    double* y = (double*)malloc(sizeof(double) * (size_t)nm);
    double* M = (double*)malloc(sizeof(double) * (size_t)nm);
    double* c = (double*)malloc(sizeof(double) * (size_t)nm);
    for (int64_t p = 0; p < ny; p++) {
        for (int64_t q = 0; q < nx; q++) y[q] = mesh[p * nx + q];
        nspline_m(y, nx, M, c);
        for (int64_t q = 0; q < nx; q++) Mx[p * nx + q] = M[q];
    }
    for (int64_t q = 0; q < nx; q++) {
        for (int64_t p = 0; p < ny; p++) y[p] = mesh[p * nx + q];
        nspline_m(y, ny, M, c);
        for (int64_t p = 0; p < ny; p++) My[p * nx + q] = M[p];
        for (int64_t p = 0; p < ny; p++) y[p] = Mx[p * nx + q];
        nspline_m(y, ny, M, c);
        for (int64_t p = 0; p < ny; p++) Mxy[p * nx + q] = M[p];
    }
    free(y); free(M); free(c);
    return ORC_OK;
}
