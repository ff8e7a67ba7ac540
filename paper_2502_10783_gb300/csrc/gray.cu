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
// the row pitch and base allow), two groups in flight per thread; a frame whose
// rows are contiguous is streamed as one flat row (no row arithmetic).  The
// histogram is privatised per block in shared memory and merged with one atomic
// per non-empty bin.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "jobs.cuh"

namespace ipp {

constexpr int GR_T = 256;

// Internal forms of the four functions.  The fast forms use the hardware
// base-2 logarithm and exponential (absolute error near 2^-22 in log2, relative
// near 2^-22 in exp2); they are taken where that error, carried to the gray
// value, stays below a few 1e-7: log for a >= 1 (the error is divided by
// log2(1 + a) >= 1), exp for base >= 2, power always (the exponent error a 2^-22
// is relative in xn^a).  log1p / expm1 keep full relative accuracy for a < 1
// (log) or a base below 2 (exp), where 1 + a xn or a^xn - 1 would cancel.
enum GrForm { GR_LINEAR = 0, GR_LOG_FAST, GR_POWER_FAST, GR_EXP_FAST, GR_LOG1P, GR_EXPM1 };

template <int FORM>
__device__ __forceinline__ float gray_map(float x, float lo, float inv, float a, float ka) {
    if (!isfinite(x)) return 0.f;
    float xn = __fmul_rn(__fsub_rn(x, lo), inv);
    xn = fminf(fmaxf(xn, 0.f), 1.f);
    if (FORM == GR_LOG_FAST) return __log2f(fmaf(a, xn, 1.f)) * ka;            // ka = 1 / log2(1 + a)
    if (FORM == GR_POWER_FAST) return xn > 0.f ? exp2f(a * __log2f(xn)) : 0.f;
    if (FORM == GR_EXP_FAST) return (exp2f(xn * a) - 1.f) * ka;                 // a = log2(base)
    if (FORM == GR_LOG1P) return log1pf(a * xn) * ka;                           // ka = 1 / ln(1 + a)
    if (FORM == GR_EXPM1) return expm1f(xn * a) * ka;                           // a = ln(base)
    return xn;                                                                   // ka = 1 / (base - 1)
}

// Index modes of the streaming loops: 0 a flat row with 32-bit group indices,
// 1 rows with 32-bit group indices, 2 rows with 64-bit group indices.
template <int MODE>
using GrIdx = typename std::conditional<MODE == 2, uint64_t, uint32_t>::type;

// Group q of four pixels: row y, first column x0, and the values (0 beyond the
// row's end).
template <int MODE>
__device__ __forceinline__ void load4(const float* __restrict__ img, GrIdx<MODE> q, GrIdx<MODE> qpr, int64_t W,
                                      int64_t pitch, bool vec, int64_t& y, int64_t& x0, float v[4]) {
    if (MODE == 0) {
        y = 0;
        x0 = (int64_t)q * 4;
    } else {
        const GrIdx<MODE> yy = q / qpr;
        y = (int64_t)yy;
        x0 = (int64_t)(q - yy * qpr) * 4;
    }
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

// Grid-stride visit of all groups, the loads of two groups issued before either
// is processed: fn(v, y, x0) per group.
template <int MODE, class Fn>
__device__ __forceinline__ void stream_groups(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                              bool vin, Fn&& fn) {
    using I = GrIdx<MODE>;
    const I qpr = (I)((W + 3) >> 2), nq = qpr * (I)H, stride = (I)gridDim.x * GR_T;
    for (I q = (I)blockIdx.x * GR_T + threadIdx.x; q < nq; q += 2 * stride) {
        const I q2 = q + stride;
        const bool two = q2 < nq;
        int64_t y0, x0, y1 = 0, x1 = 0;
        float a[4], b[4] = {0.f, 0.f, 0.f, 0.f};
        load4<MODE>(img, q, qpr, W, pitch, vin, y0, x0, a);
        if (two) load4<MODE>(img, q2, qpr, W, pitch, vin, y1, x1, b);
        fn(a, y0, x0);
        if (two) fn(b, y1, x1);
    }
}

template <int MODE, int FORM>
__global__ void __launch_bounds__(GR_T, 8) k_gray(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                               bool vin, float lo, float inv, float a, float ka,
                                               float* __restrict__ out, int64_t opitch, bool vout) {
    stream_groups<MODE>(img, W, H, pitch, vin, [&](float v[4], int64_t y, int64_t x0) {
#pragma unroll
        for (int c = 0; c < 4; c++) v[c] = gray_map<FORM>(v[c], lo, inv, a, ka);
        store4(out, y, x0, W, opitch, vout, v);
    });
}

// Workspace: a 256-byte header (the three reduction words on separate 64-byte
// lines, all zero-initialised by one memset together with the counts), the
// counts and the cumulative distribution.
struct GrayWs {
    uint32_t* kminc;  // complement of the fkey of the smallest finite value (max of complements)
    uint32_t* kmax;   // fkey of the largest finite value
    unsigned long long* nfin;
    uint32_t* cnt;    // [nbins]
    float* cdf;       // [nbins]
    float2* seg;      // [nbins]: (C(b), C(b + 1) - C(b)), one gather per interpolation
};

__device__ __forceinline__ float gr_min(const GrayWs& w) { return fkey_inv(~*w.kminc); }
__device__ __forceinline__ float gr_max(const GrayWs& w) { return fkey_inv(*w.kmax); }

template <int MODE>
__global__ void __launch_bounds__(GR_T, 8) k_minmax(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                                 bool vin, GrayWs w) {
    uint32_t kmn = 0xffffffffu, kmx = 0u, nf = 0;
    stream_groups<MODE>(img, W, H, pitch, vin, [&](float v[4], int64_t, int64_t x0) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if (x0 + c >= W || !isfinite(v[c])) continue;
            const uint32_t k = fkey(v[c]);
            kmn = min(kmn, k);
            kmx = max(kmx, k);
            nf++;
        }
    });
    // warp, then block reduction: one set of atomics per block
    __shared__ uint32_t r_mn[GR_T / 32], r_mx[GR_T / 32], r_nf[GR_T / 32];
    kmn = __reduce_min_sync(0xffffffffu, kmn);
    kmx = __reduce_max_sync(0xffffffffu, kmx);
    nf = __reduce_add_sync(0xffffffffu, nf);   // a block's share of the frame: far below 2^32 pixels
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    if (lane == 0) {
        r_mn[wi] = kmn;
        r_mx[wi] = kmx;
        r_nf[wi] = nf;
    }
    __syncthreads();
    if (wi == 0) {
        kmn = lane < GR_T / 32 ? r_mn[lane] : 0xffffffffu;
        kmx = lane < GR_T / 32 ? r_mx[lane] : 0u;
        nf = lane < GR_T / 32 ? r_nf[lane] : 0u;
        kmn = __reduce_min_sync(0xffffffffu, kmn);
        kmx = __reduce_max_sync(0xffffffffu, kmx);
        nf = __reduce_add_sync(0xffffffffu, nf);
        if (lane == 0 && nf) {
            atomicMax(w.kminc, ~kmn);
            atomicMax(w.kmax, kmx);
            atomicAdd(w.nfin, (unsigned long long)nf);
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(GR_T, 8) k_hist(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                               bool vin, int nbins, GrayWs w) {
    extern __shared__ uint32_t hsm[];
    for (int b = threadIdx.x; b < nbins; b += GR_T) hsm[b] = 0u;
    __syncthreads();
    const float mn = gr_min(w), mx = gr_max(w);
    if (*w.nfin > 0 && mx > mn) {
        const float sc = __fdiv_rn((float)nbins, __fsub_rn(mx, mn));
        stream_groups<MODE>(img, W, H, pitch, vin, [&](float v[4], int64_t, int64_t x0) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                if (x0 + c >= W || !isfinite(v[c])) continue;
                int b = (int)floorf(__fmul_rn(__fsub_rn(v[c], mn), sc));
                b = min(max(b, 0), nbins - 1);
                atomicAdd(&hsm[b], 1u);
            }
        });
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += GR_T)
        if (hsm[b]) atomicAdd(&w.cnt[b], hsm[b]);
}

// Cumulative distribution of the counts, spread over nbins / 256 blocks (the
// FP64 division per bin is the costly step): block k adds up the counts before
// its slice, scans its 256 bins and divides one bin per thread.
__global__ void __launch_bounds__(GR_T) k_cdf(int nbins, GrayWs w) {
    __shared__ unsigned long long part[GR_T / 32];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int s0 = blockIdx.x * GR_T, b = s0 + threadIdx.x;
    unsigned long long before = 0;
    for (int j = threadIdx.x; j < s0; j += GR_T) before += w.cnt[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(0xffffffffu, before, o);
    if (lane == 0) part[wi] = before;
    __syncthreads();
    before = 0;
#pragma unroll
    for (int k = 0; k < GR_T / 32; k++) before += part[k];
    __syncthreads();
    const unsigned long long c = b < nbins ? w.cnt[b] : 0ull;
    unsigned long long x = c;   // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) part[wi] = x;
    __syncthreads();
    for (int k = 0; k < wi; k++) x += part[k];
    const unsigned long long nf = *w.nfin;
    const double dn = (double)(nf ? nf : 1ull);
    if (b < nbins) {
        const unsigned long long run = before + x;
        const float c0 = (float)((double)run / dn);
        // C(b + 1) from the same integer sum the next bin's thread divides
        const float c1 = b + 1 < nbins ? (float)((double)(run + w.cnt[b + 1]) / dn) : c0;
        w.cdf[b] = c0;
        w.seg[b] = make_float2(c0, c1 - c0);
    }
}

template <int MODE>
__global__ void __launch_bounds__(GR_T, 8) k_equalize(const float* __restrict__ img, int64_t W, int64_t H,
                                                   int64_t pitch, bool vin, int nbins, GrayWs w,
                                                   float* __restrict__ out, int64_t opitch, bool vout) {
    const float mn = gr_min(w), mx = gr_max(w);
    const bool flat = !(*w.nfin > 0 && mx > mn);
    const float sc = flat ? 0.f : __fdiv_rn((float)nbins, __fsub_rn(mx, mn));
    const float cfirst = __ldg(w.cdf), clast = __ldg(w.cdf + nbins - 1);
    stream_groups<MODE>(img, W, H, pitch, vin, [&](float v[4], int64_t y, int64_t x0) {
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
                        const float2 cd = __ldg(w.seg + b);
                        g = fmaf(t - (float)b, cd.y, cd.x);
                    }
                }
            }
            v[c] = g;
        }
        store4(out, y, x0, W, opitch, vout, v);
    });
}

}  // namespace ipp

using namespace ipp;

namespace {

// A frame as the streaming loops see it: contiguous rows (in and, where there
// is one, out) collapse to one flat row.
struct GrView {
    int64_t W, H, pitch, opitch;
    bool vin, vout;
    int mode;
    unsigned grid(int per_sm) const {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t nq = ((W + 3) >> 2) * H;
        const int64_t need = (nq + GR_T - 1) / GR_T, cap = (int64_t)(sms > 0 ? sms : 152) * per_sm;
        return (unsigned)std::max<int64_t>(1, std::min(need, cap));
    }
};

GrView gr_view(const float* img, int64_t W, int64_t H, int64_t pitch, const float* out, int64_t opitch) {
    GrView v{W, H, pitch, opitch, false, false, 1};
    if (pitch == W && (!out || opitch == W)) {
        v.W = W * H;
        v.H = 1;
        v.pitch = v.opitch = v.W;
    }
    v.vin = ((uintptr_t)img & 15) == 0 && (v.H == 1 || v.pitch % 4 == 0);
    v.vout = out && ((uintptr_t)out & 15) == 0 && (v.H == 1 || v.opitch % 4 == 0);
    // 32-bit group indices while q plus twice the grid's stride stays below 2^32
    const bool small = ((v.W + 3) >> 2) * v.H < (int64_t(1) << 31);
    v.mode = !small ? 2 : (v.H == 1 ? 0 : 1);
    return v;
}

template <int MODE, int FORM>
int launch_gray_f(const float* img, const GrView& v, float lo, float inv, float a, float ka, float* out,
                  cudaStream_t s) {
    k_gray<MODE, FORM><<<v.grid(8), GR_T, 0, s>>>(img, v.W, v.H, v.pitch, v.vin, lo, inv, a, ka, out, v.opitch,
                                                   v.vout);
    return ipp_check_launch("k_gray");
}

template <int MODE>
int launch_gray_m(const float* img, const GrView& v, int form, float lo, float inv, float a, float ka, float* out,
                  cudaStream_t s) {
    switch (form) {
        case GR_LOG_FAST: return launch_gray_f<MODE, GR_LOG_FAST>(img, v, lo, inv, a, ka, out, s);
        case GR_POWER_FAST: return launch_gray_f<MODE, GR_POWER_FAST>(img, v, lo, inv, a, ka, out, s);
        case GR_EXP_FAST: return launch_gray_f<MODE, GR_EXP_FAST>(img, v, lo, inv, a, ka, out, s);
        case GR_LOG1P: return launch_gray_f<MODE, GR_LOG1P>(img, v, lo, inv, a, ka, out, s);
        case GR_EXPM1: return launch_gray_f<MODE, GR_EXPM1>(img, v, lo, inv, a, ka, out, s);
        default: return launch_gray_f<MODE, GR_LINEAR>(img, v, lo, inv, a, ka, out, s);
    }
}

template <int MODE>
int launch_equalize_m(const float* img, const GrView& v, int nbins, GrayWs w, float* out, cudaStream_t s) {
    const size_t hs = (size_t)nbins * 4;
    // 8 resident blocks per SM while their histograms fit beside each other
    const int per_sm = hs <= 24 * 1024 ? 8 : (hs <= 48 * 1024 ? 4 : 3);
    k_minmax<MODE><<<v.grid(8), GR_T, 0, s>>>(img, v.W, v.H, v.pitch, v.vin, w);
    if (int e = ipp_check_launch("k_minmax")) return e;
    cudaFuncSetAttribute(k_hist<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hs);
    k_hist<MODE><<<v.grid(per_sm), GR_T, hs, s>>>(img, v.W, v.H, v.pitch, v.vin, nbins, w);
    if (int e = ipp_check_launch("k_hist")) return e;
    k_cdf<<<(unsigned)((nbins + GR_T - 1) / GR_T), GR_T, 0, s>>>(nbins, w);
    if (int e = ipp_check_launch("k_cdf")) return e;
    k_equalize<MODE><<<v.grid(8), GR_T, 0, s>>>(img, v.W, v.H, v.pitch, v.vin, nbins, w, out, v.opitch, v.vout);
    return ipp_check_launch("k_equalize");
}

}  // namespace

int ipp_launch_gray(const float* img, int64_t W, int64_t H, int64_t pitch, int kind, float lo, float hi, float a,
                    float* out, int64_t opitch, cudaStream_t s) {
    const float inv = (float)(1.0 / ((double)hi - (double)lo));
    float ap = a, ka = 1.f;
    int form = GR_LINEAR;
    if (kind == IPP_GRAY_LOG) {
        form = a >= 1.f ? GR_LOG_FAST : GR_LOG1P;
        ka = (float)(form == GR_LOG_FAST ? 1.0 / log2(1.0 + (double)a) : 1.0 / log1p((double)a));
    } else if (kind == IPP_GRAY_POWER) {
        form = GR_POWER_FAST;
    } else if (kind == IPP_GRAY_EXP) {
        form = a >= 2.f ? GR_EXP_FAST : GR_EXPM1;
        ap = (float)(form == GR_EXP_FAST ? log2((double)a) : log((double)a));
        ka = (float)(1.0 / ((double)a - 1.0));
    }
    const GrView v = gr_view(img, W, H, pitch, out, opitch);
    if (v.mode == 0) return launch_gray_m<0>(img, v, form, lo, inv, ap, ka, out, s);
    if (v.mode == 1) return launch_gray_m<1>(img, v, form, lo, inv, ap, ka, out, s);
    return launch_gray_m<2>(img, v, form, lo, inv, ap, ka, out, s);
}

size_t ipp_equalize_ws_bytes(int nbins) {
    const size_t nb = ((size_t)nbins * 4 + 255) & ~(size_t)255;
    return 256 + nb * 4;   // header, counts, C, (C, dC) pairs
}

int ipp_launch_equalize(const float* img, int64_t W, int64_t H, int64_t pitch, int nbins, float* out,
                        int64_t opitch, void* ws, cudaStream_t s) {
    GrayWs w;
    char* b = (char*)ws;
    const size_t nb = ((size_t)nbins * 4 + 255) & ~(size_t)255;
    w.kminc = (uint32_t*)b;
    w.kmax = (uint32_t*)(b + 64);
    w.nfin = (unsigned long long*)(b + 128);
    w.cnt = (uint32_t*)(b + 256);
    w.cdf = (float*)(b + 256 + nb);
    w.seg = (float2*)(b + 256 + 2 * nb);
    if (cudaMemsetAsync(b, 0, 256 + (size_t)nbins * 4, s) != cudaSuccess)
        return ipp_check_launch("equalize workspace memset");
    const GrView v = gr_view(img, W, H, pitch, out, opitch);
    if (v.mode == 0) return launch_equalize_m<0>(img, v, nbins, w, out, s);
    if (v.mode == 1) return launch_equalize_m<1>(img, v, nbins, w, out, s);
    return launch_equalize_m<2>(img, v, nbins, w, out, s);
}

// ---- zscale display limits -----------------------------------------------------------
// Reading after the published IRAF algorithm (Sec. 2.2.6 names SAOimage's zscale):
// up to n_samples pixels at a flat stride, non-finite ones dropped, sorted; an
// iterated least-squares line of the sorted samples against their index with
// krej-sigma rejection grown by h samples on each side; the limits from the line's
// slope over the contrast, about the median, clipped to the sample range.  One
// block: the samples are sorted in shared memory (bitonic network), each thread
// keeps the residuals of its four samples in registers, and every sum is a block
// reduction in a fixed order, so the result does not depend on scheduling.
namespace ipp {

constexpr int ZS_T = 1024, ZS_MAX = 4096, ZS_PER = ZS_MAX / ZS_T;

// sum of NV doubles over the block, the same value in every thread
template <int NV>
__device__ __forceinline__ void zs_sum(double v[NV], double (*red)[ZS_T / 32]) {
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
        for (int k = 0; k < ZS_T / 32; k++) s += red[c][k];
        v[c] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(ZS_T) k_zscale(const float* __restrict__ img, int64_t W, int64_t H, int64_t pitch,
                                                 int ns, double contrast, double krej, int max_iter,
                                                 double* __restrict__ z, int32_t* __restrict__ counts) {
    __shared__ float s[ZS_MAX];
    __shared__ unsigned char good[ZS_MAX], bad[ZS_MAX];
    __shared__ int pre[ZS_MAX + 1];
    __shared__ int tsum[ZS_T];
    __shared__ double red[5][ZS_T / 32];
    __shared__ int npix_sh;
    const int tid = threadIdx.x;
    const int64_t N = W * H;
    const int64_t stride = max((int64_t)1, N / ns);
    // samples; absent or non-finite ones become +inf and sort to the end
    for (int k = tid; k < ZS_MAX; k += ZS_T) {
        float v = INFINITY;
        if (k < ns && (int64_t)k * stride < N) {
            const int64_t idx = (int64_t)k * stride, r = idx / W;
            const float q = __ldg(img + r * pitch + (idx - r * W));
            if (isfinite(q)) v = q;
        }
        s[k] = v;
    }
    if (tid == 0) npix_sh = 0;
    __syncthreads();
    // bitonic sort, ascending
    for (int size = 2; size <= ZS_MAX; size <<= 1) {
        for (int st = size >> 1; st > 0; st >>= 1) {
            for (int t = tid; t < ZS_MAX / 2; t += ZS_T) {
                const int lo = 2 * t - (t & (st - 1)), hi = lo + st;
                const bool asc = (lo & size) == 0;
                const float a = s[lo], b = s[hi];
                if ((a > b) == asc) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int k = tid; k < ZS_MAX; k += ZS_T)
        if (s[k] < INFINITY && (k + 1 == ZS_MAX || !(s[k + 1] < INFINITY))) npix_sh = k + 1;
    __syncthreads();
    const int npix = npix_sh;
    if (npix == 0) {
        if (tid == 0) {
            z[0] = z[1] = NAN;
            if (counts) counts[0] = counts[1] = 0;
        }
        return;
    }
    const double zmin = s[0], zmax = s[npix - 1];
    const int c = (npix - 1) / 2;
    const double median = (npix & 1) ? (double)s[c] : 0.5 * ((double)s[c] + (double)s[c + 1]);
    const int minpix = max(5, (int)(0.5 * (double)npix));
    const int h = max(1, (int)(0.01 * (double)npix)) / 2;
    for (int k = tid; k < ZS_MAX; k += ZS_T) good[k] = k < npix;
    __syncthreads();
    int ngood = npix, last = npix + 1;
    double slope = 0.0;
    for (int it = 0; it < max_iter; it++) {
        if (ngood >= last || ngood < minpix) break;
        // least-squares line over the good samples, x = k - c
        double v5[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < ZS_PER; j++) {
            const int k = tid + j * ZS_T;
            if (k < npix && good[k]) {
                const double x = (double)(k - c), y = (double)s[k];
                v5[0] += 1.0;
                v5[1] += x;
                v5[2] += y;
                v5[3] = __dadd_rn(v5[3], __dmul_rn(x, x));
                v5[4] = __dadd_rn(v5[4], __dmul_rn(x, y));
            }
        }
        zs_sum<5>(v5, red);
        const double n = v5[0];
        const double den = __dsub_rn(__dmul_rn(n, v5[3]), __dmul_rn(v5[1], v5[1]));
        slope = den != 0.0 ? __dsub_rn(__dmul_rn(n, v5[4]), __dmul_rn(v5[1], v5[2])) / den : 0.0;
        const double icpt = __dsub_rn(v5[2], __dmul_rn(slope, v5[1])) / n;
        double fl[ZS_PER];
        double m1[1] = {0.0};
#pragma unroll
        for (int j = 0; j < ZS_PER; j++) {
            const int k = tid + j * ZS_T;
            fl[j] = __dsub_rn((double)s[k], __dadd_rn(__dmul_rn(slope, (double)(k - c)), icpt));
            if (k < npix && good[k]) m1[0] += fl[j];
        }
        zs_sum<1>(m1, red);
        const double m = m1[0] / n;
        double v1[1] = {0.0};
#pragma unroll
        for (int j = 0; j < ZS_PER; j++) {
            const int k = tid + j * ZS_T;
            if (k < npix && good[k]) {
                const double d = __dsub_rn(fl[j], m);
                v1[0] = __dadd_rn(v1[0], __dmul_rn(d, d));
            }
        }
        zs_sum<1>(v1, red);
        const double thr = krej * sqrt(v1[0] / n);
#pragma unroll
        for (int j = 0; j < ZS_PER; j++) {
            const int k = tid + j * ZS_T;
            bad[k] = k < npix && (fl[j] < -thr || fl[j] > thr);
        }
        __syncthreads();
        // prefix counts of rejected samples: thread t owns samples 4t .. 4t + 3
        int loc = 0;
#pragma unroll
        for (int j = 0; j < ZS_PER; j++) loc += bad[tid * ZS_PER + j];
        tsum[tid] = loc;
        __syncthreads();
        for (int o = 1; o < ZS_T; o <<= 1) {   // inclusive scan of the thread totals
            const int add = tid >= o ? tsum[tid - o] : 0;
            __syncthreads();
            tsum[tid] += add;
            __syncthreads();
        }
        int run = tsum[tid] - loc;
        if (tid == 0) pre[0] = 0;
#pragma unroll
        for (int j = 0; j < ZS_PER; j++) {
            run += bad[tid * ZS_PER + j];
            pre[tid * ZS_PER + j + 1] = run;
        }
        __syncthreads();
        // good: no rejected sample within h
        int g = 0;
#pragma unroll
        for (int j = 0; j < ZS_PER; j++) {
            const int k = tid + j * ZS_T;
            const bool ok = k < npix && pre[min(k + h + 1, npix)] - pre[max(k - h, 0)] == 0;
            good[k] = ok;
            g += ok;
        }
        double gs[1] = {(double)g};
        zs_sum<1>(gs, red);
        last = ngood;
        ngood = (int)gs[0];
    }
    if (tid == 0) {
        if (ngood >= minpix) {
            const double sl = slope / contrast;
            const double a = __dsub_rn(median, __dmul_rn((double)(c - 1), sl));
            const double b = __dadd_rn(median, __dmul_rn((double)(npix - c), sl));
            z[0] = a > zmin ? a : zmin;
            z[1] = b < zmax ? b : zmax;
        } else {
            z[0] = zmin;
            z[1] = zmax;
        }
        if (counts) {
            counts[0] = npix;
            counts[1] = ngood;
        }
    }
}

}  // namespace ipp

int ipp_launch_zscale(const float* img, int64_t W, int64_t H, int64_t pitch, int ns, double contrast, double krej,
                      int max_iter, double* z, int32_t* counts, cudaStream_t s) {
    ipp::k_zscale<<<1, ipp::ZS_T, 0, s>>>(img, W, H, pitch, ns, contrast, krej, max_iter, z, counts);
    return ipp_check_launch("k_zscale");
}
