// align.cu -- image alignment of Sec. 2.2.3: coordinate mapping of a source
// frame into a target frame through both frames' WCS (Eqs. 5-7 and the inverse
// chain), the partial affine (similarity) estimate, and bilinear reprojection.
//
// Mapping, per node in FP64: SIP offsets (Eq. 5), CD (Eq. 6), then the gnomonic
// deprojection about the source tangent point followed by the projection about
// the target's.  The two are composed as one rotation: the point (p, q) of the
// source tangent plane is the direction p e + q n + c of the source's east,
// north and centre unit vectors, and its target standard coordinates are
// (R0 . w, R1 . w) / (R2 . w) with R the target basis expressed in the source
// basis -- the same mathematics as Eq. 7 and its inverse without a
// trigonometric call per node.  Then CD^-1 and Newton's method on the target's
// SIP polynomial (at most 50 steps, stop below 1e-12 px; otherwise NaN).
//
// Reprojection: output pixel (j, i) samples the source at Minv (j, i, 1).  Each
// warp takes 128 consecutive output pixels of a row: the segment's first source
// position is formed in double-float arithmetic (FP32 pairs; the FP64 pipe of
// this GPU is too narrow even for one FP64 evaluation per segment) and split
// into an integer part and a fraction, and the lanes offset it in FP32
// (|offset| <= 128 px, so the position error stays near 1e-5 px).
#include <math.h>

#include <algorithm>

#include "jobs.cuh"

namespace ipp {

constexpr int AL_T = 256;
constexpr double AL_D2R = 3.14159265358979323846 / 180.0;

struct WcsDev {
    double crpix[2], crval[2], cd[4];
    int a_order, b_order;
    double a[36], b[36];
};

__device__ __forceinline__ void sip_val_grad(const double* c, int order, double u, double v, double& f, double& fu,
                                             double& fv) {
    double up[6], vp[6];
    up[0] = vp[0] = 1.0;
#pragma unroll
    for (int k = 1; k < 6; k++) {
        up[k] = up[k - 1] * u;
        vp[k] = vp[k - 1] * v;
    }
    f = fu = fv = 0.0;
    // fully unrolled: constant coefficient indices, terms above `order` skipped
#pragma unroll
    for (int p = 0; p < 6; p++) {
#pragma unroll
        for (int q = 0; q < 6 - p; q++) {
            if (p + q > order) continue;
            const double k = c[p * 6 + q];
            f += k * up[p] * vp[q];
            if (p > 0) fu += k * p * up[p - 1] * vp[q];
            if (q > 0) fv += k * q * up[p] * vp[q - 1];
        }
    }
}

__device__ __forceinline__ double sip_val(const double* c, int order, double u, double v) {
    double f, fu, fv;
    sip_val_grad(c, order, u, v, f, fu, fv);
    return f;
}

// target basis (east, north, centre) in the source basis: R[r][c] = t_r . s_c
__device__ void wcs_rotation(const WcsDev& s, const WcsDev& t, double R[9]) {
    double sa, ca, sd, cd, ta, tca, td, tcd;
    sincos(s.crval[0] * AL_D2R, &sa, &ca);
    sincos(s.crval[1] * AL_D2R, &sd, &cd);
    sincos(t.crval[0] * AL_D2R, &ta, &tca);
    sincos(t.crval[1] * AL_D2R, &td, &tcd);
    const double S[3][3] = {{-sa, ca, 0.0}, {-sd * ca, -sd * sa, cd}, {cd * ca, cd * sa, sd}};      // e, n, c
    const double T[3][3] = {{-ta, tca, 0.0}, {-td * tca, -td * ta, tcd}, {tcd * tca, tcd * ta, td}};
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) R[r * 3 + c] = T[r][0] * S[c][0] + T[r][1] * S[c][1] + T[r][2] * S[c][2];
}

__global__ void __launch_bounds__(AL_T) k_wcs_map(WcsDev src, WcsDev tgt, int64_t nx, int64_t ny, int step,
                                                  double* __restrict__ xo, double* __restrict__ yo) {
    __shared__ double R[9];
    if (threadIdx.x < 32) {
        double r[9];
        wcs_rotation(src, tgt, r);
        if (threadIdx.x < 9) R[threadIdx.x] = r[threadIdx.x];
    }
    __syncthreads();
    const double det = tgt.cd[0] * tgt.cd[3] - tgt.cd[1] * tgt.cd[2];
    const int64_t n = nx * ny;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / nx, j = k - i * nx;
        // Eq. 5 on the source (FITS pixel = 0-based + 1)
        const double u = (double)(j * step) + 1.0 - src.crpix[0], v = (double)(i * step) + 1.0 - src.crpix[1];
        const double xi = u + sip_val(src.a, src.a_order, u, v);
        const double eta = v + sip_val(src.b, src.b_order, u, v);
        // Eq. 6, radians
        const double p = (src.cd[0] * xi + src.cd[1] * eta) * AL_D2R;
        const double q = (src.cd[2] * xi + src.cd[3] * eta) * AL_D2R;
        // Eq. 7 and the target's gnomonic projection, composed
        const double X = R[0] * p + R[1] * q + R[2];
        const double Y = R[3] * p + R[4] * q + R[5];
        const double Z = R[6] * p + R[7] * q + R[8];
        double ox = NAN, oy = NAN;
        if (Z > 0.0) {
            const double pt = X / Z / AL_D2R, qt = Y / Z / AL_D2R;
            const double xt = (tgt.cd[3] * pt - tgt.cd[1] * qt) / det;
            const double et = (-tgt.cd[2] * pt + tgt.cd[0] * qt) / det;
            double uu = xt, vv = et;
            bool ok = false;
            for (int it = 0; it < 50; it++) {
                double f, fu, fv, g, gu, gv;
                sip_val_grad(tgt.a, tgt.a_order, uu, vv, f, fu, fv);
                sip_val_grad(tgt.b, tgt.b_order, uu, vv, g, gu, gv);
                const double r1 = uu + f - xt, r2 = vv + g - et;
                const double j11 = 1.0 + fu, j12 = fv, j21 = gu, j22 = 1.0 + gv;
                const double dj = j11 * j22 - j12 * j21;
                if (dj == 0.0) break;
                const double su = (j22 * r1 - j12 * r2) / dj, sv = (-j21 * r1 + j11 * r2) / dj;
                uu -= su;
                vv -= sv;
                if (fabs(su) < 1e-12 && fabs(sv) < 1e-12) {
                    ok = true;
                    break;
                }
            }
            if (ok) {
                ox = uu + tgt.crpix[0] - 1.0;
                oy = vv + tgt.crpix[1] - 1.0;
            }
        }
        xo[k] = ox;
        yo[k] = oy;
    }
}

// ---- partial affine estimate -----------------------------------------------------
constexpr int AF_BLOCKS = 152;

struct AffPts {
    const double *x, *y, *xt, *yt;
    int64_t n, grid_nx;
    int step;
    __device__ __forceinline__ bool get(int64_t k, double& a, double& b, double& c, double& d) const {
        if (x) {
            a = x[k];
            b = y[k];
        } else {
            const int64_t i = k / grid_nx;
            a = (double)((k - i * grid_nx) * step);
            b = (double)(i * step);
        }
        c = xt[k];
        d = yt[k];
        return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
    }
};

// block sum of NV doubles in a fixed order (warp butterfly, then warps in order)
template <int NV>
__device__ void block_sum(double v[NV], double (*red)[AL_T / 32]) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NV; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
        if (lane == 0) red[c][wi] = v[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NV; c++) {
        double s = 0.0;
        for (int k = 0; k < AL_T / 32; k++) s += red[c][k];
        v[c] = s;
    }
    __syncthreads();
}

// pass 1: per-block count and coordinate sums
__global__ void __launch_bounds__(AL_T) k_aff_sum1(AffPts P, double* __restrict__ part) {
    __shared__ double red[5][AL_T / 32];
    double v[5] = {0, 0, 0, 0, 0};
    for (int64_t k = (int64_t)blockIdx.x * AL_T + threadIdx.x; k < P.n; k += (int64_t)gridDim.x * AL_T) {
        double a, b, c, d;
        if (!P.get(k, a, b, c, d)) continue;
        v[0] += 1.0;
        v[1] += a;
        v[2] += b;
        v[3] += c;
        v[4] += d;
    }
    block_sum<5>(v, red);
    if (threadIdx.x < 5) part[blockIdx.x * 8 + threadIdx.x] = v[threadIdx.x];
}

// sum of column q of the per-block partials, in the same order wherever it is
// formed (lane l adds blocks l, l + 32, ...; then a butterfly): called by a full warp
__device__ __forceinline__ double aff_col(const double* part, int nb, int q) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += part[b * 8 + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// pass 2: per-block centred moments
__global__ void __launch_bounds__(AL_T) k_aff_sum2(AffPts P, const double* __restrict__ part1,
                                                   double* __restrict__ part2) {
    __shared__ double red[3][AL_T / 32];
    __shared__ double cs[5];
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < 5; q++) {
            const double v = aff_col(part1, gridDim.x, q);
            if (threadIdx.x == 0) cs[q] = v;
        }
    }
    __syncthreads();
    const double s[5] = {cs[0], cs[1], cs[2], cs[3], cs[4]};
    const double m = s[0] > 0.0 ? s[0] : 1.0;
    const double cx = s[1] / m, cy = s[2] / m, ctx = s[3] / m, cty = s[4] / m;
    double v[3] = {0, 0, 0};
    for (int64_t k = (int64_t)blockIdx.x * AL_T + threadIdx.x; k < P.n; k += (int64_t)gridDim.x * AL_T) {
        double a, b, c, d;
        if (!P.get(k, a, b, c, d)) continue;
        const double dx = a - cx, dy = b - cy, ex = c - ctx, ey = d - cty;
        v[0] += dx * dx + dy * dy;
        v[1] += dx * ex + dy * ey;
        v[2] += dx * ey - dy * ex;
    }
    block_sum<3>(v, red);
    if (threadIdx.x < 3) part2[blockIdx.x * 8 + threadIdx.x] = v[threadIdx.x];
}

__global__ void k_aff_solve(const double* __restrict__ part1, const double* __restrict__ part2, int nb,
                            double* __restrict__ M, int32_t* __restrict__ status) {
    double s[5];
#pragma unroll
    for (int q = 0; q < 5; q++) s[q] = aff_col(part1, nb, q);
    const double saa = aff_col(part2, nb, 0), sa = aff_col(part2, nb, 1), sb = aff_col(part2, nb, 2);
    if (threadIdx.x != 0) return;
    const double m = s[0];
    if (!(m >= 2.0) || !(saa > 0.0)) {
        for (int k = 0; k < 12; k++) M[k] = NAN;
        if (status) *status = IPP_ERR_DEGENERATE;
        return;
    }
    const double cx = s[1] / m, cy = s[2] / m, ctx = s[3] / m, cty = s[4] / m;
    const double a = sa / saa, b = sb / saa, s2 = a * a + b * b;
    M[0] = a;
    M[1] = -b;
    M[2] = ctx - (a * cx - b * cy);
    M[3] = b;
    M[4] = a;
    M[5] = cty - (b * cx + a * cy);
    M[6] = a / s2;
    M[7] = b / s2;
    M[8] = -(M[6] * M[2] + M[7] * M[5]);
    M[9] = -b / s2;
    M[10] = a / s2;
    M[11] = -(M[9] * M[2] + M[10] * M[5]);
    if (status) *status = (s2 > 0.0) ? IPP_OK : IPP_ERR_DEGENERATE;
}

// ---- bilinear reprojection ---------------------------------------------------------
constexpr int RP_SEG = 128;   // output pixels per warp task (4 per lane)

// df x exact float (|n| < 2^24): the product to ~2^-46 relative
__device__ __forceinline__ df df_mul_exact(df m, float n) {
    const float p = __fmul_rn(m.hi, n);
    const float e = __fmaf_rn(m.hi, n, -p);
    return two_sum(p, __fmaf_rn(m.lo, n, e));
}

// integer part and fraction in [0, 1) of a double-float (|value| < 2^30)
__device__ __forceinline__ void df_floor(df a, int& ip, float& frac) {
    float fh = floorf(a.hi);
    df r = two_sum(__fsub_rn(a.hi, fh), a.lo);   // a.hi - fh is exact
    float f = r.hi;
    if (f < 0.f) {
        fh -= 1.f;
        f += 1.f;
        if (f >= 1.f) {   // a fraction just below 0 that rounds to 1 is the next integer
            fh += 1.f;
            f = 0.f;
        }
    } else if (f >= 1.f) {
        fh += 1.f;
        f -= 1.f;
    }
    ip = (int)fh;
    frac = f;
}

// one output pixel at source position (ix + tx, iy + ty): 0 <= x <= W - 1 and
// 0 <= y <= H - 1, the pair beyond the last column / row not read, `fill` when
// outside or when a neighbour of non-zero weight is not finite
__device__ __forceinline__ float rp_careful(const float* __restrict__ src, int64_t pitch, int Wi, int Hi, int ix,
                                           int iy, float tx, float ty, float fill) {
    const bool in = ix >= 0 && iy >= 0 && (ix < Wi - 1 || (ix == Wi - 1 && tx == 0.f)) &&
                    (iy < Hi - 1 || (iy == Hi - 1 && ty == 0.f));
    if (!in) return fill;
    // the left / top pair of the last column / row is the one below the edge
    const int x0 = min(ix, max(Wi - 2, 0)), y0 = min(iy, max(Hi - 2, 0));
    const float t = tx + (float)(ix - x0), s = ty + (float)(iy - y0);
    const float w00 = (1.f - t) * (1.f - s), w10 = t * (1.f - s), w01 = (1.f - t) * s, w11 = t * s;
    const float* row = src + (int64_t)y0 * pitch + x0;
    float acc = 0.f;
    bool bad = false;
    if (w00 != 0.f) { const float q = __ldg(row); bad |= !isfinite(q); acc = fmaf(w00, q, acc); }
    if (w10 != 0.f) { const float q = __ldg(row + 1); bad |= !isfinite(q); acc = fmaf(w10, q, acc); }
    if (w01 != 0.f) { const float q = __ldg(row + pitch); bad |= !isfinite(q); acc = fmaf(w01, q, acc); }
    if (w11 != 0.f) { const float q = __ldg(row + pitch + 1); bad |= !isfinite(q); acc = fmaf(w11, q, acc); }
    return bad ? fill : acc;
}

__global__ void __launch_bounds__(AL_T) k_reproject(const float* __restrict__ src, int64_t W, int64_t H,
                                                    int64_t pitch, const double* __restrict__ Minv, int64_t Wo,
                                                    int64_t Ho, float fill, float* __restrict__ out,
                                                    int64_t opitch, bool vout) {
    // the transform as double-floats, converted once per block: FP64 work on
    // this GPU's narrow FP64 pipe stays off the per-pixel and per-segment path
    __shared__ float mh[6], ml[6];
    __shared__ int msane;
    if (threadIdx.x < 6) {
        const double m = Minv[threadIdx.x];
        const float h = (float)m;
        mh[threadIdx.x] = h;
        ml[threadIdx.x] = (float)(m - (double)h);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        for (int q = 0; q < 6; q++) ok = ok && isfinite(mh[q]) && fabsf(mh[q]) < 1073741824.f;
        // steps above 2^20 px per pixel map every pixel but one outside the frame
        msane = ok && fabsf(mh[0]) < 1048576.f && fabsf(mh[3]) < 1048576.f;
    }
    __syncthreads();
    const df m0{mh[0], ml[0]}, m1{mh[1], ml[1]}, m2{mh[2], ml[2]};
    const df m3{mh[3], ml[3]}, m4{mh[4], ml[4]}, m5{mh[5], ml[5]};
    const float f0 = mh[0], f3 = mh[3];
    const bool sane = msane != 0;
    const int lane = threadIdx.x & 31;
    const int64_t segs = (Wo + RP_SEG - 1) / RP_SEG, tasks = segs * Ho;
    const int64_t warps = (int64_t)gridDim.x * (AL_T / 32);
    const float lim = 1073741824.f;   // 2^30: positions beyond are outside any frame
    const int Wi = (int)W, Hi = (int)H;
    for (int64_t t = (int64_t)blockIdx.x * (AL_T / 32) + (threadIdx.x >> 5); t < tasks; t += warps) {
        const int64_t i = t / segs, j0 = (t - i * segs) * RP_SEG;
        // first source position of the segment, Minv (j0, i, 1), in double-float
        const float fj = (float)(int)j0, fi = (float)(int)i;   // exact: Wo, Ho < 2^24
        const df X0 = df_add(df_add(df_mul_exact(m0, fj), df_mul_exact(m1, fi)), m2);
        const df Y0 = df_add(df_add(df_mul_exact(m3, fj), df_mul_exact(m4, fi)), m5);
        const bool base_ok = sane && fabsf(X0.hi) < lim && fabsf(Y0.hi) < lim;
        int ibx = 0, iby = 0;
        float fbx = 0.f, fby = 0.f;
        if (base_ok) {
            df_floor(X0, ibx, fbx);
            df_floor(Y0, iby, fby);
        }
        // the positions are monotone along the segment: when both ends have all four
        // neighbours inside the frame, so has every pixel between (no per-pixel
        // bounds tests, four unconditional loads)
        const int kmax = (int)min((int64_t)RP_SEG, Wo - j0) - 1;
        bool interior = false;
        if (base_ok) {
            const float xb = fmaf(f0, (float)kmax, fbx), yb = fmaf(f3, (float)kmax, fby);
            const int ixa = ibx + (int)floorf(fbx), ixb = ibx + (int)floorf(xb);
            const int iya = iby + (int)floorf(fby), iyb = iby + (int)floorf(yb);
            interior = min(ixa, ixb) >= 0 && max(ixa, ixb) <= Wi - 2 && min(iya, iyb) >= 0 && max(iya, iyb) <= Hi - 2;
        }
        float v[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int k = lane * 4 + c;
            float r = fill;
            if (base_ok && k <= kmax) {
                const float fx = fmaf(f0, (float)k, fbx), fy = fmaf(f3, (float)k, fby);
                const float flx = floorf(fx), fly = floorf(fy);
                const int ix = ibx + (int)flx, iy = iby + (int)fly;
                const float tx = fx - flx, ty = fy - fly;
                if (interior) {
                    const float* row = src + (int64_t)iy * pitch + ix;
                    const float q00 = __ldg(row), q10 = __ldg(row + 1);
                    const float q01 = __ldg(row + pitch), q11 = __ldg(row + pitch + 1);
                    const float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty), w01 = (1.f - tx) * ty,
                                w11 = tx * ty;
                    // the same sum, in the same order, as the careful form: a term of
                    // zero weight adds 0 exactly when its value is finite
                    const float acc = fmaf(w11, q11, fmaf(w01, q01, fmaf(w10, q10, w00 * q00)));
                    r = isfinite(acc) ? acc : rp_careful(src, pitch, Wi, Hi, ix, iy, tx, ty, fill);
                } else {
                    r = rp_careful(src, pitch, Wi, Hi, ix, iy, tx, ty, fill);
                }
            }
            v[c] = r;
        }
        const int64_t jj = j0 + lane * 4;
        float* orow = out + i * opitch;
        if (vout && jj + 4 <= Wo) {
            *reinterpret_cast<float4*>(orow + jj) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (jj + c < Wo) orow[jj + c] = v[c];
        }
    }
}

}  // namespace ipp

using namespace ipp;

static unsigned al_grid(int64_t units_per_block_task, int64_t tasks, int per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (tasks + units_per_block_task - 1) / units_per_block_task;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)(sms > 0 ? sms : 152) * per_sm));
}

static WcsDev to_dev(const ipp_wcs& w) {
    WcsDev d;
    for (int k = 0; k < 2; k++) {
        d.crpix[k] = w.crpix[k];
        d.crval[k] = w.crval[k];
    }
    for (int k = 0; k < 4; k++) d.cd[k] = w.cd[k];
    d.a_order = w.a_order;
    d.b_order = w.b_order;
    for (int k = 0; k < 36; k++) {
        d.a[k] = w.a[k];
        d.b[k] = w.b[k];
    }
    return d;
}

int ipp_launch_wcs_map(const ipp_wcs& src, const ipp_wcs& tgt, int64_t nx, int64_t ny, int step, double* xo,
                       double* yo, cudaStream_t s) {
    // FP64-bound: 64-thread blocks so that small node grids still reach every SM
    k_wcs_map<<<al_grid(64, nx * ny, 16), 64, 0, s>>>(to_dev(src), to_dev(tgt), nx, ny, step, xo, yo);
    return ipp_check_launch("k_wcs_map");
}

size_t ipp_affine_ws_bytes() { return (size_t)AF_BLOCKS * 8 * sizeof(double) * 2; }

int ipp_launch_affine_fit(const double* x, const double* y, const double* xt, const double* yt, int64_t n,
                          int64_t grid_nx, int step, double* M, int32_t* status, void* ws, cudaStream_t s) {
    AffPts P{x, y, xt, yt, n, grid_nx, step};
    double* p1 = (double*)ws;
    double* p2 = p1 + AF_BLOCKS * 8;
    k_aff_sum1<<<AF_BLOCKS, AL_T, 0, s>>>(P, p1);
    if (int e = ipp_check_launch("k_aff_sum1")) return e;
    k_aff_sum2<<<AF_BLOCKS, AL_T, 0, s>>>(P, p1, p2);
    if (int e = ipp_check_launch("k_aff_sum2")) return e;
    k_aff_solve<<<1, 32, 0, s>>>(p1, p2, AF_BLOCKS, M, status);
    return ipp_check_launch("k_aff_solve");
}

int ipp_launch_reproject(const float* src, int64_t W, int64_t H, int64_t pitch, const double* Minv, int64_t Wo,
                         int64_t Ho, float fill, float* out, int64_t opitch, cudaStream_t s) {
    const bool vout = (opitch % 4 == 0) && (((uintptr_t)out & 15) == 0);
    const int64_t tasks = ((Wo + RP_SEG - 1) / RP_SEG) * Ho;
    k_reproject<<<al_grid(AL_T / 32, tasks, 8), AL_T, 0, s>>>(src, W, H, pitch, Minv, Wo, Ho, fill, out, opitch,
                                                               vout);
    return ipp_check_launch("k_reproject");
}
