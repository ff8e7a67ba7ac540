// gray.cu -- gray-scale maps of Sec. 2.2.6: value-to-gray functions and
// histogram equalisation.  Readings:
//   xn = clip((x - lo) / (hi - lo), 0, 1), non-finite x -> 0;
//   linear xn; log log10(a xn + 1) / log10(a + 1); power xn^a;
//   exp (a^xn - 1) / (a - 1);
//   equalisation: nbins bins of width (max - min) / nbins over the finite values;
//   the bin of x is floor((x - min) s), s = nbins / (max - min), in single
//   precision (it decides an integer, and both sides round it the same way); the
//   gray value is the cumulative distribution interpolated between bin centres at
//   t = (x - min) s - 1/2, clamped to the first and last bin.
// Every pass streams the frame in groups of four pixels (one 128-bit load where
// the row pitch and base allow); the histogram is privatised per block in
// shared memory and merged with one atomic per non-empty bin.
#include <math.h>

#include <algorithm>

#include "jobs.cuh"

namespace ipp {

constexpr int GR_T = 256;

__device__ __forceinline__ float gray_map(float x, int kind, float lo, float inv, float a, float ka) {
    if (!isfinite(x)) return 0.f;
    float xn = __fmul_rn(__fsub_rn(x, lo), inv);
    xn = fminf(fmaxf(xn, 0.f), 1.f);
    switch (kind) {
        // log1p / expm1 keep full relative accuracy for a near 0 (log) or 1 (exp)
        case IPP_GRAY_LOG: return log1pf(a * xn) * ka;     // ka = 1 / ln(a + 1)
        case IPP_GRAY_POWER: return xn > 0.f ? powf(xn, a) : 0.f;
        case IPP_GRAY_EXP: return expm1f(xn * a) * ka;     // a = ln(base), ka = 1 / (base - 1)
        default: return xn;
    }
}

// Group q of four pixels of a W x H frame: row y, first column x0, and the
// values (0 beyond the row's end).  I is the index type (32-bit when the
// number of groups allows).
template <class I>
__device__ __forceinline__ void load4(const float* __restrict__ img, I q, I qpr, int64_t W, int64_t pitch, bool vec,
                                      int64_t& y, int64_t& x0, float v[4]) {
    const I yy = q / qpr;
    y = (int64_t)yy;
    x0 = (int64_t)(q - yy * qpr) * 4;
    const float* row = img + y * pitch;
    if (vec && x0 + 4 <= W) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(row + x0));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++) v[c] = x0 + c < W ? __ldg(row + x0 + c) : 0.f;
    }
}

__device__ __forceinline__ void store4(float* __restrict__ out, int64_t y, int64_t x0, int64_t W, int64_t opitch,
                                       bool vec, const float v[4]) {
    float* row = out + y * opitch;
    if (vec && x0 + 4 <= W) {
        *reinterpret_cast<float4*>(row + x0) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++)
            if (x0 + c < W) row[x0 + c] = v[c];
    }
}

__device__ __forceinline__ bool vec_ok(const void* p, int64_t pitch) {
    return (pitch % 4 == 0) && (((uintptr_t)p & 15) == 0);
}

template <class I>
__global__ void __launch_bounds__(GR_T) k_gray(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                               int kind, float lo, float inv, float a, float ka,
                                               float* __restrict__ out, int64_t opitch) {
    const I qpr = (I)((W + 3) >> 2), nq = qpr * (I)H;
    const bool vin = vec_ok(img, pitch), vout = vec_ok(out, opitch);
    for (I q = (I)blockIdx.x * GR_T + threadIdx.x; q < nq; q += (I)gridDim.x * GR_T) {
        int64_t y, x0;
        float v[4];
        load4<I>(img, q, qpr, W, pitch, vin, y, x0, v);
#pragma unroll
        for (int c = 0; c < 4; c++) v[c] = gray_map(v[c], kind, lo, inv, a, ka);
        store4(out, y, x0, W, opitch, vout, v);
    }
}

struct GrayWs {
    uint32_t* kmin;   // fkey of the smallest finite value
    uint32_t* kmax;   // fkey of the largest
    unsigned long long* nfin;
    uint32_t* cnt;    // [nbins]
    float* cdf;       // [nbins]
};

template <class I>
__global__ void __launch_bounds__(GR_T) k_minmax(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                                 GrayWs w) {
    const I qpr = (I)((W + 3) >> 2), nq = qpr * (I)H;
    const bool vin = vec_ok(img, pitch);
    uint32_t kmn = 0xffffffffu, kmx = 0u, nf = 0;
    for (I q = (I)blockIdx.x * GR_T + threadIdx.x; q < nq; q += (I)gridDim.x * GR_T) {
        int64_t y, x0;
        float v[4];
        load4<I>(img, q, qpr, W, pitch, vin, y, x0, v);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (x0 + c >= W || !isfinite(v[c])) continue;
            const uint32_t k = fkey(v[c]);
            kmn = min(kmn, k);
            kmx = max(kmx, k);
            nf++;
        }
    }
    kmn = __reduce_min_sync(0xffffffffu, kmn);
    kmx = __reduce_max_sync(0xffffffffu, kmx);
    nf = __reduce_add_sync(0xffffffffu, nf);   // a warp's share of the frame: far below 2^32 pixels
    if ((threadIdx.x & 31) == 0 && nf) {
        atomicMin(w.kmin, kmn);
        atomicMax(w.kmax, kmx);
        atomicAdd(w.nfin, (unsigned long long)nf);
    }
}

template <class I>
__global__ void __launch_bounds__(GR_T) k_hist(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                               int nbins, GrayWs w) {
    extern __shared__ uint32_t hsm[];
    for (int b = threadIdx.x; b < nbins; b += GR_T) hsm[b] = 0u;
    __syncthreads();
    const float mn = fkey_inv(*w.kmin), mx = fkey_inv(*w.kmax);
    if (*w.nfin > 0 && mx > mn) {
        const float sc = __fdiv_rn((float)nbins, __fsub_rn(mx, mn));
        const I qpr = (I)((W + 3) >> 2), nq = qpr * (I)H;
        const bool vin = vec_ok(img, pitch);
        for (I q = (I)blockIdx.x * GR_T + threadIdx.x; q < nq; q += (I)gridDim.x * GR_T) {
            int64_t y, x0;
            float v[4];
            load4<I>(img, q, qpr, W, pitch, vin, y, x0, v);
#pragma unroll
            for (int c = 0; c < 4; c++) {
                if (x0 + c >= W || !isfinite(v[c])) continue;
                int b = (int)floorf(__fmul_rn(__fsub_rn(v[c], mn), sc));
                b = min(max(b, 0), nbins - 1);
                atomicAdd(&hsm[b], 1u);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += GR_T)
        if (hsm[b]) atomicAdd(&w.cnt[b], hsm[b]);
}

// Cumulative distribution of the counts: one block of 1024 threads, each owning
// a contiguous run of bins; warp and block exclusive scans of the run totals.
__global__ void __launch_bounds__(1024) k_cdf(int nbins, GrayWs w) {
    __shared__ unsigned long long wsum[32];
    const int per = (nbins + 1023) / 1024;
    const int s0 = min(nbins, (int)threadIdx.x * per), s1 = min(nbins, s0 + per);
    unsigned long long acc = 0;
    for (int b = s0; b < s1; b++) acc += w.cnt[b];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    unsigned long long x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[wi] = x;
    __syncthreads();
    if (wi == 0) {
        unsigned long long z = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += t;
        }
        wsum[lane] = z;
    }
    __syncthreads();
    unsigned long long run = (x - acc) + (wi > 0 ? wsum[wi - 1] : 0ull);
    const unsigned long long nf = *w.nfin;
    for (int b = s0; b < s1; b++) {
        run += w.cnt[b];
        w.cdf[b] = (float)((double)run / (double)(nf ? nf : 1ull));
    }
}

template <class I>
__global__ void __launch_bounds__(GR_T) k_equalize(const float* __restrict__ img, int64_t W, int64_t H,
                                                   int64_t pitch, int nbins, GrayWs w, float* __restrict__ out,
                                                   int64_t opitch) {
    const float mn = fkey_inv(*w.kmin), mx = fkey_inv(*w.kmax);
    const bool flat = !(*w.nfin > 0 && mx > mn);
    const float sc = flat ? 0.f : __fdiv_rn((float)nbins, __fsub_rn(mx, mn));
    const float cfirst = __ldg(w.cdf), clast = __ldg(w.cdf + nbins - 1);
    const I qpr = (I)((W + 3) >> 2), nq = qpr * (I)H;
    const bool vin = vec_ok(img, pitch), vout = vec_ok(out, opitch);
    for (I q = (I)blockIdx.x * GR_T + threadIdx.x; q < nq; q += (I)gridDim.x * GR_T) {
        int64_t y, x0;
        float v[4];
        load4<I>(img, q, qpr, W, pitch, vin, y, x0, v);
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const float x = v[c];
            float g = 0.f;
            if (!flat && isfinite(x)) {
                const float t = __fsub_rn(__fmul_rn(__fsub_rn(x, mn), sc), 0.5f);
                if (!(t > 0.f)) {
                    g = cfirst;
                } else {
                    const int b = (int)floorf(t);
                    if (b >= nbins - 1) {
                        g = clast;
                    } else {
                        const float c0 = __ldg(w.cdf + b), c1 = __ldg(w.cdf + b + 1);
                        g = fmaf(t - (float)b, c1 - c0, c0);
                    }
                }
            }
            v[c] = g;
        }
        store4(out, y, x0, W, opitch, vout, v);
    }
}

}  // namespace ipp

using namespace ipp;

static unsigned gr_grid(int64_t W, int64_t H, int per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nq = ((W + 3) >> 2) * H;
    const int64_t need = (nq + GR_T - 1) / GR_T, cap = (int64_t)(sms > 0 ? sms : 152) * per_sm;
    return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

static bool gr_small(int64_t W, int64_t H) {
    // 32-bit group indices: q plus the grid's stride stays below 2^32
    return ((W + 3) >> 2) * H < (int64_t(1) << 31);
}

int ipp_launch_gray(const float* img, int64_t W, int64_t H, int64_t pitch, int kind, float lo, float hi, float a,
                    float* out, int64_t opitch, cudaStream_t s) {
    const float inv = (float)(1.0 / ((double)hi - (double)lo));
    float ap = a, ka = 1.f;
    if (kind == IPP_GRAY_LOG) ka = (float)(1.0 / log1p((double)a));
    if (kind == IPP_GRAY_EXP) {
        ap = (float)log((double)a);
        ka = (float)(1.0 / ((double)a - 1.0));
    }
    const unsigned g = gr_grid(W, H, 8);
    if (gr_small(W, H))
        k_gray<uint32_t><<<g, GR_T, 0, s>>>(img, W, H, pitch, kind, lo, inv, ap, ka, out, opitch);
    else
        k_gray<uint64_t><<<g, GR_T, 0, s>>>(img, W, H, pitch, kind, lo, inv, ap, ka, out, opitch);
    return ipp_check_launch("k_gray");
}

size_t ipp_equalize_ws_bytes(int nbins) {
    return 256 + (((size_t)nbins * 4 + 255) & ~(size_t)255) * 2;
}

int ipp_launch_equalize(const float* img, int64_t W, int64_t H, int64_t pitch, int nbins, float* out,
                        int64_t opitch, void* ws, cudaStream_t s) {
    GrayWs w;
    char* b = (char*)ws;
    const size_t nb = ((size_t)nbins * 4 + 255) & ~(size_t)255;
    w.kmin = (uint32_t*)b;
    w.kmax = (uint32_t*)(b + 4);
    w.nfin = (unsigned long long*)(b + 8);
    w.cnt = (uint32_t*)(b + 256);
    w.cdf = (float*)(b + 256 + nb);
    if (cudaMemsetAsync(b, 0xff, 4, s) != cudaSuccess || cudaMemsetAsync(b + 4, 0, 12, s) != cudaSuccess ||
        cudaMemsetAsync(w.cnt, 0, (size_t)nbins * 4, s) != cudaSuccess)
        return ipp_check_launch("equalize workspace memset");
    const bool sm = gr_small(W, H);
    const unsigned g = gr_grid(W, H, 8), gh = gr_grid(W, H, 4);
    const size_t hs = (size_t)nbins * 4;
    if (sm) {
        k_minmax<uint32_t><<<g, GR_T, 0, s>>>(img, W, H, pitch, w);
        cudaFuncSetAttribute(k_hist<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs);
        k_hist<uint32_t><<<gh, GR_T, hs, s>>>(img, W, H, pitch, nbins, w);
    } else {
        k_minmax<uint64_t><<<g, GR_T, 0, s>>>(img, W, H, pitch, w);
        cudaFuncSetAttribute(k_hist<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs);
        k_hist<uint64_t><<<gh, GR_T, hs, s>>>(img, W, H, pitch, nbins, w);
    }
    if (int e = ipp_check_launch("k_minmax/k_hist")) return e;
    k_cdf<<<1, 1024, 0, s>>>(nbins, w);
    if (int e = ipp_check_launch("k_cdf")) return e;
    if (sm)
        k_equalize<uint32_t><<<g, GR_T, 0, s>>>(img, W, H, pitch, nbins, w, out, opitch);
    else
        k_equalize<uint64_t><<<g, GR_T, 0, s>>>(img, W, H, pitch, nbins, w, out, opitch);
    return ipp_check_launch("k_equalize");
}
