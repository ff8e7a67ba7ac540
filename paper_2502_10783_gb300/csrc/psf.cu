// psf.cu -- batched differentiable PSF model and Levenberg-Marquardt fit
// (paper-silent reading of the photometry of Sec. 2.2.5; elliptical Moffat or
// Gaussian, 7 parameters x0, y0, F, sky, sx, sy, theta, point-sampled at the
// pixel centres of an S x S stamp).
//
// A group of G lanes owns one stamp: the stamp stays in registers for the whole
// fit, each lane accumulates J'WJ (28 terms), J'W r (7) and chi^2 over its
// pixels in FP32, and the group reduces them with shuffles.  The damped 7 x 7
// normal equations are solved in FP64 (LDL', no square roots) by every lane of
// the group on identical data.  Shuffles name only the group's lanes, so the
// groups of a warp run their fits independently.
#include <math.h>

#include <algorithm>

#include "jobs.cuh"

namespace ipp {

constexpr int F_THREADS = 128;
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

// Reductions inside a group of G lanes; the mask names only the group, so
// groups of one warp may diverge (each runs its own fit).
template <int G>
__device__ __forceinline__ unsigned gmask() {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
    }
}
template <int G>
__device__ __forceinline__ float gsum(float v) {
    const unsigned m = gmask<G>();
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ int gsum_i(int v) {
    const unsigned m = gmask<G>();
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
}

// Solve (H + lambda D) x = g, D = diag(H) floored at 1e-9 max(diag), by LDL' in
// FP64, in place on the packed lower triangle.  H packed upper-triangular
// row-major (28 entries, the same numbers as the lower triangle).  Returns false
// if a pivot is not positive (matrix not positive definite).
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

__device__ bool solve7(const float Hf[28], const float gf[7], double lam, double x[7]) {
    double A[28];
    double dmax = 0.0;
#pragma unroll
    for (int a = 0; a < 7; a++) {
        // upper-row-major index of (a, b), b >= a:  a*7 - a*(a-1)/2 + (b - a)
#pragma unroll
        for (int b = a; b < 7; b++) A[tri(b, a)] = (double)Hf[a * 7 - a * (a - 1) / 2 + (b - a)];
    }
#pragma unroll
    for (int a = 0; a < 7; a++) dmax = fmax(dmax, A[tri(a, a)]);
#pragma unroll
    for (int a = 0; a < 7; a++) A[tri(a, a)] += lam * fmax(A[tri(a, a)], 1e-9 * dmax);
    // A[tri(i,j)] becomes L(i,j) * D(j) for j < i and D(i) on the diagonal
    double iD[7];
#pragma unroll
    for (int j = 0; j < 7; j++) {
#pragma unroll
        for (int i = j; i < 7; i++) {
            double t = A[tri(i, j)];
#pragma unroll
            for (int q = 0; q < j; q++) t -= A[tri(i, q)] * A[tri(j, q)] * iD[q];
            A[tri(i, j)] = t;
        }
        if (!(A[tri(j, j)] > 0.0)) return false;
        iD[j] = 1.0 / A[tri(j, j)];
    }
    double z[7];
#pragma unroll
    for (int i = 0; i < 7; i++) {
        double t = (double)gf[i];
#pragma unroll
        for (int q = 0; q < i; q++) t -= A[tri(i, q)] * iD[q] * z[q];
        z[i] = t;
    }
#pragma unroll
    for (int i = 6; i >= 0; i--) {
        double t = z[i] * iD[i];
#pragma unroll
        for (int q = i + 1; q < 7; q++) t -= A[tri(q, i)] * iD[i] * x[q];
        x[i] = t;
    }
    return true;
}

template <int G, int NPL>
__global__ void __launch_bounds__(F_THREADS) k_psf_fit(FitJob J) {
    const int lg = threadIdx.x % G;
    const int64_t group = ((int64_t)blockIdx.x * F_THREADS + threadIdx.x) / G;
    const int64_t ngroups = ((int64_t)gridDim.x * F_THREADS) / G;
    const int S = J.S, NP = S * S;
    const unsigned gm = gmask<G>();
    for (int64_t st = group; st < J.N; st += ngroups) {
        const float* stamp = J.stamps + st * NP;
        const float* wts = J.weights ? J.weights + st * NP : nullptr;
        float d[NPL];
#pragma unroll
        for (int m = 0; m < NPL; m++) {
            int k = lg + G * m;
            d[m] = k < NP ? __ldg(stamp + k) : 0.f;
        }
        float p[7];
        if (J.init) {
#pragma unroll
            for (int a = 0; a < 7; a++) p[a] = __ldg(J.init + st * 7 + a);
        } else {
            // start: centre, border median sky, sum above sky, widths 1.6 / 1.4
            const int nb = 4 * S - 4;
            uint32_t lo = 0u, hi = 0xffffffffu;
            const int k0 = (nb - 1) / 2, k1 = nb / 2;
            while (lo < hi) {
                uint32_t mid = lo + ((hi - lo) >> 1);
                int c = 0;
#pragma unroll
                for (int m = 0; m < NPL; m++) {
                    int k = lg + G * m, i = k / S, j = k - i * S;
                    bool border = k < NP && (i == 0 || j == 0 || i == S - 1 || j == S - 1);
                    c += border && fkey(d[m]) <= mid;
                }
                c = gsum_i<G>(c);
                if (c > k0) hi = mid; else lo = mid + 1;
            }
            const uint32_t ka = lo;
            int cle = 0;
            uint32_t nxt = 0xffffffffu;
#pragma unroll
            for (int m = 0; m < NPL; m++) {
                int k = lg + G * m, i = k / S, j = k - i * S;
                bool border = k < NP && (i == 0 || j == 0 || i == S - 1 || j == S - 1);
                if (border) {
                    uint32_t kk = fkey(d[m]);
                    cle += kk <= ka;
                    if (kk > ka && kk < nxt) nxt = kk;
                }
            }
            cle = gsum_i<G>(cle);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) nxt = min(nxt, __shfl_xor_sync(gm, nxt, o));
            const uint32_t kb = cle > k1 ? ka : nxt;
            const float sky0 = (float)(0.5 * ((double)fkey_inv(ka) + (double)fkey_inv(kb)));
            float fs = 0.f;
#pragma unroll
            for (int m = 0; m < NPL; m++)
                if (lg + G * m < NP) fs += d[m] - sky0;
            fs = gsum<G>(fs);
            p[0] = 0.5f * (S - 1); p[1] = 0.5f * (S - 1); p[2] = fs; p[3] = sky0;
            p[4] = 1.6f; p[5] = 1.4f; p[6] = 0.f;
        }
        // chi^2 and, when `full`, J'WJ (packed upper triangle) and J'W r at pp
        float H[28], g[7];
        auto evaluate = [&](const float pp[7], bool full) -> float {
            const float c = cosf(pp[6]), s = sinf(pp[6]);
            float chi = 0.f;
            if (full) {
#pragma unroll
                for (int a = 0; a < 28; a++) H[a] = 0.f;
#pragma unroll
                for (int a = 0; a < 7; a++) g[a] = 0.f;
            }
#pragma unroll
            for (int m = 0; m < NPL; m++) {
                int k = lg + G * m;
                if (k < NP) {
                    int i = k / S, j = k - i * S;
                    PsfPix e;
                    psf_eval(pp, (float)j - pp[0], (float)i - pp[1], J.model, J.beta, c, s, full, e);
                    float wk = wts ? __ldg(wts + k) : 1.0f;
                    float r = d[m] - e.m;
                    chi = fmaf(wk * r, r, chi);
                    if (full) {
                        int t = 0;
#pragma unroll
                        for (int a = 0; a < 7; a++) {
                            float wa = wk * e.j[a];
                            g[a] = fmaf(wa, r, g[a]);
#pragma unroll
                            for (int b = a; b < 7; b++) { H[t] = fmaf(wa, e.j[b], H[t]); t++; }
                        }
                    }
                }
            }
            chi = gsum<G>(chi);
            if (full) {
#pragma unroll
                for (int a = 0; a < 28; a++) H[a] = gsum<G>(H[a]);
#pragma unroll
                for (int a = 0; a < 7; a++) g[a] = gsum<G>(g[a]);
            }
            return chi;
        };
        float chi2 = evaluate(p, true);
        double lam = (double)J.lambda0;
        int fl = IPP_FLAG_FIT_MAXITER, it, nsing = 0;
        for (it = 0; it < J.max_iter; it++) {
            double delta[7];
            if (!solve7(H, g, lam, delta)) {
                lam *= 10.0;
                nsing++;
                if (lam > 1e10) { it++; break; }
                continue;
            }
            float pt[7];
#pragma unroll
            for (int a = 0; a < 7; a++) pt[a] = (float)((double)p[a] + delta[a]);
            if (!(pt[4] > 0.05f) || !(pt[5] > 0.05f)) {
                lam *= 10.0;
                if (lam > 1e10) { fl = 0; it++; break; }
                continue;
            }
            float c2t = evaluate(pt, false);
            if (c2t < chi2) {
                float rel = (chi2 - c2t) / chi2;
#pragma unroll
                for (int a = 0; a < 7; a++) p[a] = pt[a];
                chi2 = c2t;
                lam *= 0.1;
                // FP32 chi^2 resolves ~1e-7: the relative-decrease test of the
                // FP64 rule (1e-8) is taken at 1e-6 here
                if (rel < 1e-6f) { fl = 0; it++; break; }
                evaluate(p, true);
            } else {
                lam *= 10.0;
                if (lam > 1e10) { fl = 0; it++; break; }
            }
        }
        if (nsing > 0 && fl) fl |= IPP_FLAG_FIT_SINGULAR;
        if (!(p[4] > 0.05f) || !(p[5] > 0.05f)) fl |= IPP_FLAG_FIT_BAD_SIGMA;
        if (p[4] < p[5]) { float t = p[4]; p[4] = p[5]; p[5] = t; p[6] += 0.5f * F_PI; }
        p[6] = p[6] - F_PI * floorf((p[6] + 0.5f * F_PI) / F_PI);
        if (lg == 0) {
#pragma unroll
            for (int a = 0; a < 7; a++) J.params[st * 7 + a] = p[a];
            J.chi2[st] = chi2;
            if (J.iters) J.iters[st] = it;
            if (J.flags) J.flags[st] = fl;
        }
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

int ipp_launch_psf_fit(const FitJob& J, cudaStream_t s) {
    const int NP = J.S * J.S;
    int blocks;
    if (NP <= 8 * 32) {
        constexpr int G = 8;
        int64_t groups = J.N;
        blocks = (int)std::min<int64_t>((groups * G + F_THREADS - 1) / F_THREADS, (int64_t)sm_count() * 16);
        k_psf_fit<G, 32><<<blocks, F_THREADS, 0, s>>>(J);
    } else if (NP <= 32 * 32) {
        constexpr int G = 32;
        int64_t groups = J.N;
        blocks = (int)std::min<int64_t>((groups * G + F_THREADS - 1) / F_THREADS, (int64_t)sm_count() * 16);
        k_psf_fit<G, 32><<<blocks, F_THREADS, 0, s>>>(J);
    } else {
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "stamp size %d above 32", J.S);
    }
    return ipp_check_launch("k_psf_fit");
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
