// psf.cu -- batched differentiable PSF model and Levenberg-Marquardt fit
// (paper-silent reading of the photometry of Sec. 2.2.5; elliptical Moffat or
// Gaussian, 7 parameters x0, y0, F, sky, sx, sy, theta, point-sampled at the
// pixel centres of an S x S stamp).
//
// The fit (k_psf_fit) runs one stamp per lane: each lane keeps its LM state,
// J'WJ (28 terms), J'W r (7) and chi^2 in registers and evaluates its stamp from
// a column of the warp's shared-memory tile.  The damped 7 x 7 normal equations
// are solved in FP64 (LDL', no square roots), one system per lane, so one FP64
// instruction of the warp serves 32 stamps.  The forward model and its adjoint
// (k_psf_fwd, k_psf_adj) evaluate the same point-sampled model.
#include <math.h>

#include <algorithm>

#include "jobs.cuh"

namespace ipp {

constexpr float F_PI = 3.14159265358979f;

struct PsfPix {  // model value and the 7 derivatives at one pixel
    float m;
    float j[7];
};

__device__ __forceinline__ void psf_eval(const float p[7], float dx, float dy, int model, float beta,
                                         float c, float s, bool want_j, PsfPix& o) {
    const float sx = p[4], sy = p[5], F = p[2];
    const float u = c * dx + s * dy, v = -s * dx + c * dy;
    const float isx2 = 1.0f / (sx * sx), isy2 = 1.0f / (sy * sy);
    const float q = u * u * isx2 + v * v * isy2;
    float P, dPdq, A1;
    if (model == IPP_PSF_GAUSS) {
        A1 = 1.0f / (2.0f * F_PI * sx * sy);
        float e = expf(-0.5f * q);
        P = F * A1 * e;
        A1 *= e;  // dP/dF
        dPdq = -0.5f * P;
    } else {
        const float base = 1.0f + q;
        const float pw = exp2f(-beta * log2f(base));
        A1 = (beta - 1.0f) / (F_PI * sx * sy) * pw;  // dP/dF
        P = F * A1;
        dPdq = -beta * P / base;
    }
    o.m = P + p[3];
    if (!want_j) return;
    const float dqdu = 2.0f * u * isx2, dqdv = 2.0f * v * isy2;
    o.j[0] = dPdq * (-dqdu * c + dqdv * s);
    o.j[1] = dPdq * (-dqdu * s - dqdv * c);
    o.j[2] = A1;
    o.j[3] = 1.0f;
    o.j[4] = -P / sx - dPdq * 2.0f * u * u * isx2 / sx;
    o.j[5] = -P / sy - dPdq * 2.0f * v * v * isy2 / sy;
    // dq/dtheta = 2uv (1/sx^2 - 1/sy^2), written without the cancellation of
    // the difference when sx ~ sy
    o.j[6] = dPdq * 2.0f * u * v * ((sy - sx) * (sy + sx)) * isx2 * isy2;
}

// The FP64 pipe of this part is narrow (1/64 of the FP32 rate), so the solve
// spends it on the arithmetic of the factorisation alone: the widening of the
// FP32 normal equations, the pivot tests and the reciprocal seeds are integer
// operations on the IEEE-754 bit patterns.

// Exact float -> double (sign, exponent rebiased by 1023 - 127, mantissa
// shifted up by 52 - 23 bits); zeros, infinities and NaNs map to their double
// counterparts, subnormals take the conversion instruction.
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu, m = u & 0x7fffffu, sg = u & 0x80000000u;
    if (e == 0u && m != 0u) return (double)f;
    const uint32_t e64 = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);
    return __hiloint2double((int)(sg | (e64 << 20) | (m >> 3)), (int)(m << 29));
}

// double -> float rounded to nearest (ties away from zero) for |v| in the
// normal single range, 0 below it and infinity above it.
__device__ __forceinline__ float narrow(double v) {
    const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    const uint32_t sg = hi & 0x80000000u;
    if (e <= 0) return __uint_as_float(sg);
    if (e >= 255) return __uint_as_float(sg | 0x7f800000u);
    // exponent and the top 23 mantissa bits, plus the first discarded bit
    // (a carry out of the mantissa moves into the exponent, as it should)
    const uint32_t body = ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float(sg | (body + ((lo >> 28) & 1u)));
}

// 1/d for a pivot d by Newton's iteration x <- x + x (1 - d x) from a
// single-precision seed; each step doubles the correct bits (about 22 -> 44 ->
// beyond double precision).  Pivots outside 2^-100 .. 2^100 divide.
__device__ __forceinline__ double recip_pivot(double d) {
    const int e = (__double2hiint(d) >> 20) & 0x7ff;
    if (e > 923 && e < 1123) {
        double x = widen(__fdividef(1.0f, narrow(d)));
        x = fma(x, fma(-d, x, 1.0), x);
        return fma(x, fma(-d, x, 1.0), x);
    }
    return 1.0 / d;
}

// d > 0, finite and normal: sign clear, exponent field in 1 .. 2046
__device__ __forceinline__ bool pivot_ok(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d);
    return hi - 0x00100000u < 0x7fe00000u;
}

__device__ __forceinline__ int tri(int i, int j) { return i * (i - 1) / 2 + j; }  // strictly lower, j < i

// Solve (H + lambda D) x = g, D = diag(H) floored at 1e-9 max(diag), in FP64 by
// an LDL' factorisation (no square roots).  H packed upper-triangular row-major
// (28 entries).  Row-oriented: row i of L is formed from the earlier rows with
// W(q) = L(i,q) D(q) held as a temporary, so each product L(i,q) D(q) L(j,q)
// costs one fused multiply-add.  Returns false if a pivot is not positive.
__device__ __forceinline__ bool solve7(const float Hf[28], const float gf[7], double lam, double x[7]) {
    double L[21], iD[7];
    float dmaxf = 0.f;
#pragma unroll
    for (int a = 0; a < 7; a++) dmaxf = fmaxf(dmaxf, Hf[a * 7 - a * (a - 1) / 2]);
    const double floor_d = 1e-9 * widen(dmaxf);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 7; i++) {
        double W[7];
#pragma unroll
        for (int j = 0; j < i; j++) {
            // H(j, i) from the upper row-major packing
            double t = widen(Hf[j * 7 - j * (j - 1) / 2 + (i - j)]);
#pragma unroll
            for (int q = 0; q < j; q++) t = fma(-W[q], L[tri(j, q)], t);
            W[j] = t;
            L[tri(i, j)] = t * iD[j];
        }
        const double h = widen(Hf[i * 7 - i * (i - 1) / 2]);
        double d = fma(lam, fmax(h, floor_d), h);
#pragma unroll
        for (int q = 0; q < i; q++) d = fma(-W[q], L[tri(i, q)], d);
        ok = ok && pivot_ok(d);
        iD[i] = recip_pivot(d);
    }
    if (!ok) return false;
    double z[7];
#pragma unroll
    for (int i = 0; i < 7; i++) {
        double t = widen(gf[i]);
#pragma unroll
        for (int q = 0; q < i; q++) t = fma(-L[tri(i, q)], z[q], t);
        z[i] = t;
    }
#pragma unroll
    for (int i = 6; i >= 0; i--) {
        double t = z[i] * iD[i];
#pragma unroll
        for (int q = i + 1; q < 7; q++) t = fma(-L[tri(q, i)], x[q], t);
        x[i] = t;
    }
    return true;
}

// ---------------------------------------------------------------------------
// LM fit, G lanes per stamp.  A warp (one block) owns a contiguous chunk of
// stamps and fits 32/G of them at a time, one per slot; the G lanes of a slot
// hold identical copies of its LM state and all slots step through the same
// round:
//   (1) idle slots take the next stamps of the chunk, in slot order; the warp
//       stages each new stamp in shared memory (pixel k of slot s at
//       k (32/G + 1) + s, so a column is written and a row read without bank
//       conflicts) and computes its default starting point together;
//   (2) slots with a fit in progress solve their damped normal equations (FP64);
//   (3) every slot with a point to try evaluates chi^2, J'WJ and J'Wr there,
//       each lane of the slot over every G-th stamp row, and the slot's lanes
//       add their sums with shuffles;
//   (4) each slot accepts, rejects or stops.
// The Jacobian is evaluated at every trial point, not only after an accepted
// step: a rejected trial wastes its normal equations, but no slot of the warp
// waits for another slot's extra evaluation.  Per-lane accumulation over the
// pixels is sequential; chi^2 is summed per stamp row first, so its rounding
// stays near that of a 2 x S-term sum.
//
// G = 1 for large batches: one FP64 instruction serves 32 solves, and G = 2
// (12 warps an SM instead of 7) measured slower on 200,000 stamps because it
// repeats every solve on both lanes of a slot, the FP64 pipe of this part
// running at 1/64 of the FP32 rate.  Batches too small to give every lane a
// stamp take G = 2 or 4 (fit_lanes_per_stamp), where the shorter rounds win.
constexpr int FL_MAX_WARPS = 8;

// chi^2, J'WJ and J'Wr of one stamp at pp.  The model of psf_eval with the
// per-trial constants (reciprocal widths, normalisation, trig) taken out of the
// pixel loop and its derivatives regrouped around T = 2 dP/dq, a = u/sx^2 and
// b = v/sy^2:
//   dm/dx0 = T (b s - a c),  dm/dy0 = -T (a s + b c),  dm/dF = P/F,  dm/dsky = 1,
//   dm/dsx = -(P + T a u)/sx,  dm/dsy = -(P + T b v)/sy,
//   dm/dtheta = T u v (sy^2 - sx^2)/(sx^2 sy^2).
// Moffat (1+q)^-beta is exp2(-beta log2(1+q)) with the fast base-2 logarithm
// (absolute error ~2^-22 on the exponent, a few ulp in P).
template <int MODEL, bool WEIGHTED, int G, int PITCH>
__device__ __forceinline__ float eval_lane(const float* __restrict__ col, const float* __restrict__ wts, int S,
                                           float beta, const float pp[7], float Ht[28], float gt[7], float* sm2) {
    const int h = (threadIdx.x & 31) % G;
#pragma unroll
    for (int a = 0; a < 28; a++) Ht[a] = 0.f;
#pragma unroll
    for (int a = 0; a < 7; a++) gt[a] = 0.f;
    float sn, cs;
    sincosf(pp[6], &sn, &cs);
    const float x0 = pp[0], F = pp[2], sky = pp[3];
    const float isx = 1.0f / pp[4], isy = 1.0f / pp[5];
    const float isx2 = isx * isx, isy2 = isy * isy;
    const float kth = (pp[5] - pp[4]) * (pp[5] + pp[4]) * isx2 * isy2;
    const float A0 = (MODEL == IPP_PSF_GAUSS ? 0.5f / F_PI : (beta - 1.0f) / F_PI) * isx * isy;
    const float tq = MODEL == IPP_PSF_GAUSS ? -1.0f : -2.0f * beta;  // T = tq P / (1+q) (Moffat), -P (Gauss)
    float chi = 0.f, star2 = 0.f;  // chi^2 and sum w P^2 (the star part of the model, squared)
    for (int i = h; i < S; i += G) {
        const float dy = (float)i - pp[1];
        const float sdy = sn * dy, cdy = cs * dy;
        const float* row = col + i * S * PITCH;
        float rowc = 0.f, rows = 0.f;
        float jf = 0.f;
#pragma unroll 5
        for (int j = 0; j < S; j++, jf += 1.0f) {
            const float dx = jf - x0;
            const float u = fmaf(cs, dx, sdy), v = fmaf(-sn, dx, cdy);
            const float a = u * isx2, b = v * isy2;
            const float q = fmaf(u, a, v * b);
            float A1, P, T;
            if (MODEL == IPP_PSF_GAUSS) {
                A1 = A0 * exp2f(-0.72134752f * q);  // exp(-q/2)
                P = F * A1;
                T = -P;
            } else {
                const float base = 1.0f + q;
                A1 = A0 * exp2f(-beta * __log2f(base));
                P = F * A1;
                T = __fdividef(tq * P, base);
            }
            const float wk = WEIGHTED ? __ldg(wts + i * S + j) : 1.0f;
            const float r = row[j * PITCH] - (P + sky);
            rowc = fmaf(wk * r, r, rowc);
            rows = fmaf(wk * P, P, rows);
            float e[7];
            e[0] = T * fmaf(b, sn, -a * cs);
            e[1] = -T * fmaf(a, sn, b * cs);
            e[2] = A1;
            e[3] = 1.0f;
            e[4] = -isx * fmaf(T * a, u, P);
            e[5] = -isy * fmaf(T * b, v, P);
            e[6] = T * u * v * kth;
            int t = 0;
#pragma unroll
            for (int c = 0; c < 7; c++) {
                const float wa = wk * e[c];
                gt[c] = fmaf(wa, r, gt[c]);
#pragma unroll
                for (int d = c; d < 7; d++) { Ht[t] = fmaf(wa, e[d], Ht[t]); t++; }
            }
        }
        chi += rowc;
        star2 += rows;
    }
    if (G > 1) {  // all lanes of the slot are here (their states are identical)
        const unsigned pm = ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
#pragma unroll
            for (int a = 0; a < 28; a++) Ht[a] += __shfl_xor_sync(pm, Ht[a], o);
#pragma unroll
            for (int a = 0; a < 7; a++) gt[a] += __shfl_xor_sync(pm, gt[a], o);
            chi += __shfl_xor_sync(pm, chi, o);
            star2 += __shfl_xor_sync(pm, star2, o);
        }
    }
    *sm2 = star2;
    return chi;
}

// Pixel index of border pixel b (0 <= b < 4S-4) of an S x S stamp: the top
// row, the bottom row, then rows 1..S-2 alternating left and right edge.
__device__ __forceinline__ int border_k(int b, int S) {
    if (b < S) return b;
    if (b < 2 * S) return (S - 1) * S + (b - S);
    const int c = b - 2 * S;
    return (1 + (c >> 1)) * S + ((c & 1) ? S - 1 : 0);
}

// Default start of stamp `sr` staged in column r: centre, border-median sky, sum
// above sky, widths 1.6 / 1.4, theta 0.  All lanes of the warp take part and all
// return the same values.  The border keys (at most 4 a lane for S <= 32) stay
// in registers during the bisection for the two middle order statistics.
template <int PITCH>
__device__ __forceinline__ void init_coop(const float* __restrict__ sm, int r, int S, float p[7]) {
    const int lane = threadIdx.x & 31;
    const int NP = S * S, nb = 4 * S - 4;
    const int k0 = (nb - 1) / 2, k1 = nb / 2;
    uint32_t key[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int b = lane + 32 * t;
        key[t] = b < nb ? fkey(sm[border_k(b, S) * PITCH + r]) : 0xffffffffu;
    }
    const int nmine = (nb - lane + 31) >> 5;  // border values this lane holds
    uint32_t lo = 0u, hi = 0xffffffffu;
    while (lo < hi) {  // smallest key with more than k0 border values at or below it
        const uint32_t mid = lo + ((hi - lo) >> 1);
        int c = 0;
#pragma unroll
        for (int t = 0; t < 4; t++) c += t < nmine && key[t] <= mid;
        c = warp_sum_i(c);
        if (c > k0) hi = mid; else lo = mid + 1;
    }
    const uint32_t ka = lo;
    int cle = 0;
    uint32_t nxt = 0xffffffffu;
#pragma unroll
    for (int t = 0; t < 4; t++) {
        if (t < nmine) {
            cle += key[t] <= ka;
            if (key[t] > ka && key[t] < nxt) nxt = key[t];
        }
    }
    cle = warp_sum_i(cle);
    nxt = __reduce_min_sync(0xffffffffu, nxt);
    const uint32_t kb = cle > k1 ? ka : nxt;
    const float sky0 = (float)(0.5 * ((double)fkey_inv(ka) + (double)fkey_inv(kb)));
    float fs = 0.f;
    for (int k = lane; k < NP; k += 32) fs += sm[k * PITCH + r] - sky0;
    fs = warp_sum(fs);
    p[0] = 0.5f * (S - 1); p[1] = 0.5f * (S - 1); p[2] = fs; p[3] = sky0;
    p[4] = 1.6f; p[5] = 1.4f; p[6] = 0.f;
}

template <int MODEL, bool WEIGHTED, int G>
__global__ void __launch_bounds__(32 * FL_MAX_WARPS) k_psf_fit(FitJob J, int64_t chunk) {
    constexpr int SLOTS = 32 / G, PITCH = SLOTS + 1;
    extern __shared__ float fl_sm_all[];  // per warp [S*S][PITCH]: pixel k of slot s's stamp in column s
    __shared__ unsigned long long blk_next;  // next stamp of the block's chunk
    const unsigned FULL = 0xffffffffu;
    const unsigned HEADS = G == 1 ? FULL : (G == 2 ? 0x55555555u : 0x11111111u);  // first lane of each slot
    const int lane = threadIdx.x & 31;
    const int slot = lane / G;
    const int S = J.S, NP = S * S;
    float* fl_sm = fl_sm_all + (threadIdx.x >> 5) * NP * PITCH;
    // stamps to fit: N, or the device count when one is given; the chunks are
    // cut from that count here, so a count known only on the device needs no sync
    int64_t nfit = J.N;
    if (J.n_dev) nfit = min(nfit, (int64_t)max(__ldg(J.n_dev), 0));
    if (chunk <= 0) chunk = (nfit + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = (int64_t)blockIdx.x * chunk;
    const int64_t c1 = c0 + chunk < nfit ? c0 + chunk : nfit;
    if (threadIdx.x == 0) blk_next = (unsigned long long)c0;
    __syncthreads();
    bool drained = false;  // the block's chunk has been handed out
    int64_t st = -1;
    float p[7], H[28], g[7], chi2 = 0.f, sm2 = 0.f;
    double lam = 0.0;
    int it = 0, nsing = 0;
    bool fresh = false;
#pragma unroll
    for (int a = 0; a < 7; a++) p[a] = 0.f;
    while (true) {
        const unsigned idle = __ballot_sync(FULL, st < 0) & HEADS;
        if (idle && !drained) {
            // the warp takes as many stamps as it has idle slots from the
            // block's chunk; the shared cursor may run past c1
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&blk_next, (unsigned long long)__popc(idle));
            const int64_t next = (int64_t)__shfl_sync(FULL, base, 0);
            drained = next + __popc(idle) >= c1;
            const int rank = __popc(idle & ((1u << (slot * G)) - 1u));
            if (st < 0 && next + rank < c1) {
                st = next + rank;
                fresh = true;
                it = 0; nsing = 0;
                lam = (double)J.lambda0;
            }
            unsigned nm = __ballot_sync(FULL, fresh) & HEADS;
            while (nm) {
                const int rl = __ffs(nm) - 1, r = rl / G;
                nm &= nm - 1u;
                const int64_t sr = __shfl_sync(FULL, st, rl);
                const float* src = J.stamps + sr * NP;
                for (int k = lane; k < NP; k += 32) fl_sm[k * PITCH + r] = __ldg(src + k);
                __syncwarp();
                if (J.init) {
                    if (slot == r) {
#pragma unroll
                        for (int a = 0; a < 7; a++) p[a] = __ldg(J.init + sr * 7 + a);
                    }
                } else {
                    float q[7];
                    init_coop<PITCH>(fl_sm, r, S, q);
                    if (slot == r) {
#pragma unroll
                        for (int a = 0; a < 7; a++) p[a] = q[a];
                    }
                }
            }
        }
        if (!__any_sync(FULL, st >= 0)) break;

        float pt[7];
        bool try_pt = false;
        int fl = -1;
        if (st >= 0) {
            if (fresh) {
#pragma unroll
                for (int a = 0; a < 7; a++) pt[a] = p[a];
                try_pt = true;
            } else {
                double delta[7];
                if (!solve7(H, g, lam, delta)) {
                    lam *= 10.0;
                    nsing++;
                    it++;
                    if (lam > 1e10) fl = IPP_FLAG_FIT_MAXITER;
                } else {
                    {
                        // converged when the Gauss-Newton decrease g'H^-1 g is below what the
                        // distance to the optimum (1e-10 chi^2) and the model's FP32 rounding
                        // (1e-12 sum w P^2) allow; the damped step's decrease never exceeds
                        // it, so the undamped system is solved only when that one is small
                        const double thr = 1e-10 * widen(chi2) + 1e-12 * widen(sm2);
                        double dec = 0.0;
#pragma unroll
                        for (int a = 0; a < 7; a++) dec = fma(widen(g[a]), delta[a], dec);
                        if (dec <= thr) {
                            double dgn[7];
                            if (solve7(H, g, 0.0, dgn)) {
                                double dg = 0.0;
#pragma unroll
                                for (int a = 0; a < 7; a++) dg = fma(widen(g[a]), dgn[a], dg);
                                if (dg <= thr) fl = 0;
                            }
                        }
                    }
#pragma unroll
                    for (int a = 0; a < 7; a++) pt[a] = narrow(widen(p[a]) + delta[a]);
                    if (fl == 0) {
                        // stopped at p
                    } else if (!(pt[4] > 0.05f) || !(pt[5] > 0.05f)) {
                        lam *= 10.0;
                        it++;
                        if (lam > 1e10) fl = 0;
                    } else {
                        try_pt = true;
                    }
                }
            }
        }
        float Ht[28], gt[7], c2t = 0.f, s2t = 0.f;
        // both lanes of a slot take the same branch: their states are identical
        if (try_pt) {
            const float* wts = WEIGHTED ? J.weights + st * NP : nullptr;
            c2t = eval_lane<MODEL, WEIGHTED, G, PITCH>(fl_sm + slot, wts, S, J.beta, pt, Ht, gt, &s2t);
        }
        if (try_pt) {
            bool take = fresh;
            if (!fresh) {
                it++;
                if (c2t < chi2) {
                    take = true;
                    lam /= 10.0;   // as the oracle: 1e-3 * 0.1 rounds above 1e-4 in FP64
                } else {
                    lam *= 10.0;
                    if (lam > 1e10) fl = 0;
                }
            }
            if (take) {
#pragma unroll
                for (int a = 0; a < 7; a++) p[a] = pt[a];
#pragma unroll
                for (int a = 0; a < 28; a++) H[a] = Ht[a];
#pragma unroll
                for (int a = 0; a < 7; a++) g[a] = gt[a];
                chi2 = c2t;
                sm2 = s2t;
            }
            fresh = false;
        }
        if (st >= 0 && fl < 0 && it >= J.max_iter) fl = IPP_FLAG_FIT_MAXITER;
        if (fl >= 0) {
            if (nsing > 0 && fl) fl |= IPP_FLAG_FIT_SINGULAR;
            if (!(p[4] > 0.05f) || !(p[5] > 0.05f)) fl |= IPP_FLAG_FIT_BAD_SIGMA;
            float q[7];
#pragma unroll
            for (int a = 0; a < 7; a++) q[a] = p[a];
            if (q[4] < q[5]) { const float t = q[4]; q[4] = q[5]; q[5] = t; q[6] += 0.5f * F_PI; }
            q[6] = q[6] - F_PI * floorf((q[6] + 0.5f * F_PI) / F_PI);
            if (lane % G == 0) {
#pragma unroll
                for (int a = 0; a < 7; a++) J.params[st * 7 + a] = q[a];
                J.chi2[st] = chi2;
                if (J.iters) J.iters[st] = it;
                if (J.flags) J.flags[st] = fl;
            }
            st = -1;
        }
        __syncwarp();
    }
}

// forward model: one thread per pixel
__global__ void k_psf_fwd(const float* params, int64_t N, int S, int model, float beta, float* out) {
    const int64_t NP = (int64_t)S * S;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * NP;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t n = t / NP;
        int k = (int)(t - n * NP), i = k / S, j = k - i * S;
        float p[7];
#pragma unroll
        for (int a = 0; a < 7; a++) p[a] = __ldg(params + n * 7 + a);
        PsfPix e;
        psf_eval(p, (float)j - p[0], (float)i - p[1], model, beta, cosf(p[6]), sinf(p[6]), false, e);
        out[t] = e.m;
    }
}

// adjoint: grad_params[n] = J(n)' grad_model[n], one warp per stamp
__global__ void k_psf_adj(const float* params, int64_t N, int S, int model, float beta, const float* grad,
                          float* gout) {
    const int lane = threadIdx.x & 31;
    const int64_t NP = (int64_t)S * S;
    for (int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; n < N;
         n += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float p[7];
#pragma unroll
        for (int a = 0; a < 7; a++) p[a] = __ldg(params + n * 7 + a);
        const float c = cosf(p[6]), s = sinf(p[6]);
        float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = lane; k < NP; k += 32) {
            int i = k / S, j = k - i * S;
            PsfPix e;
            psf_eval(p, (float)j - p[0], (float)i - p[1], model, beta, c, s, true, e);
            float gm = __ldg(grad + n * NP + k);
#pragma unroll
            for (int a = 0; a < 7; a++) acc[a] = fmaf(gm, e.j[a], acc[a]);
        }
#pragma unroll
        for (int a = 0; a < 7; a++) acc[a] = warp_sum(acc[a]);
        if (lane < 7) {
            float v = acc[0];
#pragma unroll
            for (int a = 1; a < 7; a++) v = (lane == a) ? acc[a] : v;
            gout[n * 7 + lane] = v;
        }
    }
}

}  // namespace ipp

using namespace ipp;

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 132;
}

static size_t fit_warp_bytes(int S, int G) { return (size_t)S * S * (32 / G + 1) * sizeof(float); }
static int fit_max_warps(int S, int G) {
    return (int)std::min<size_t>(FL_MAX_WARPS, (size_t)(227 * 1024) / fit_warp_bytes(S, G));
}

template <int MODEL, bool WEIGHTED, int G>
static int launch_fit(const FitJob& J, cudaStream_t s) {
    auto k = k_psf_fit<MODEL, WEIGHTED, G>;
    const size_t per_warp = fit_warp_bytes(J.S, G);
    // warps of one block share a chunk of stamps: the block's chunk drains with
    // every slot busy until its last few stamps, so the larger the block, the
    // smaller the idle tail.  One block per SM, as many warps as its shared
    // memory holds.
    const int wmax = fit_max_warps(J.S, G);
    const int64_t warps = std::min<int64_t>((int64_t)sm_count() * wmax, (J.N + 32 / G - 1) / (32 / G));
    const int64_t blocks = std::min<int64_t>(sm_count(), warps);
    const int wpb = (int)((warps + blocks - 1) / blocks);
    const size_t smem = per_warp * wpb;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    const int64_t chunk = J.n_dev ? 0 : (J.N + blocks - 1) / blocks;   // 0: from the device count
    k<<<(unsigned)blocks, 32 * wpb, smem, s>>>(J, chunk);
    return ipp_check_launch("k_psf_fit");
}

// Lanes per stamp: 1 when the stamps fill every lane the GPU can hold (one FP64
// instruction then serves 32 solves); for smaller batches 2 or 4 lanes share a
// stamp, so that the batch still spreads over the lanes and each round is
// shorter.  G is taken while N G stays within 1.25 x the lanes resident at G
// (measured on 152 SMs, 15 x 15 stamps: G = 4 up to ~12,000 stamps, G = 2 up
// to ~24,000, G = 1 beyond).
static int fit_lanes_per_stamp(const FitJob& J) {
    const int64_t sms = sm_count();
    for (int G = 4; G > 1; G >>= 1)
        if (J.N * G * 4 <= sms * fit_max_warps(J.S, G) * 32 * 5) return G;
    return 1;
}

template <int MODEL, bool WEIGHTED>
static int launch_fit_g(const FitJob& J, cudaStream_t s) {
    switch (fit_lanes_per_stamp(J)) {
        case 4: return launch_fit<MODEL, WEIGHTED, 4>(J, s);
        case 2: return launch_fit<MODEL, WEIGHTED, 2>(J, s);
        default: return launch_fit<MODEL, WEIGHTED, 1>(J, s);
    }
}

int ipp_launch_psf_fit(const FitJob& J, cudaStream_t s) {
    if (fit_warp_bytes(J.S, 1) > 227 * 1024)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "stamp size %d above 32", J.S);
    if (J.model == IPP_PSF_GAUSS)
        return J.weights ? launch_fit_g<IPP_PSF_GAUSS, true>(J, s) : launch_fit_g<IPP_PSF_GAUSS, false>(J, s);
    return J.weights ? launch_fit_g<IPP_PSF_MOFFAT, true>(J, s) : launch_fit_g<IPP_PSF_MOFFAT, false>(J, s);
}

int ipp_launch_psf_fwd(const float* params, int64_t N, int S, int model, float beta, float* out, cudaStream_t s) {
    int64_t tot = N * S * S;
    int blocks = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)sm_count() * 32);
    k_psf_fwd<<<std::max(blocks, 1), 256, 0, s>>>(params, N, S, model, beta, out);
    return ipp_check_launch("k_psf_fwd");
}

int ipp_launch_psf_adj(const float* params, int64_t N, int S, int model, float beta, const float* grad,
                       float* gout, cudaStream_t s) {
    int blocks = (int)std::min<int64_t>((N * 32 + 255) / 256, (int64_t)sm_count() * 32);
    k_psf_adj<<<std::max(blocks, 1), 256, 0, s>>>(params, N, S, model, beta, grad, gout);
    return ipp_check_launch("k_psf_adj");
}
