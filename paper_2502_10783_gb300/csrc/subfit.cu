// subfit.cu -- the fit of image subtraction (Sec. 2.2.4, Eqs. 8-10): stamp
// selection, the normal equations of the basis-kernel model and their Cholesky
// solve.  Readings (the same as the difference-image kernels of subtract.cu):
//   stamps: the frame is cut into nsx x nsy regions; in each, the median and
//     1.4826 MAD of the template's finite pixels; the candidate is the brightest
//     template pixel (first in raster order among equals) whose fit footprint
//     (2 fh + 1)^2 and convolution support (2 (fh + hw) + 1)^2 lie inside the
//     frame and are finite in I and R, kept when it exceeds the median by nsig
//     robust sigmas;
//   model: I + B = R (x) K, K = sum_n a_n K_n, a_n = sum_s c_{n,s} P_s taken at
//     the candidate's centre, B = sum_b d_b P_b at each pixel; unweighted least
//     squares over every footprint pixel of every candidate; the design row of a
//     pixel is [C_n P_s for n, s] then [-P_b for b], C_n = R (x) K_n, target I.
//
// Precision.  The normal matrix is badly conditioned (after a diagonal scaling
// its condition number is ~1e11 on a survey frame), so it is formed in FP64: a
// relative error of 1e-6 in its entries moves the fitted model by ~2%.  The
// convolutions use the separability of the basis, K_n(u, v) = h_{k,i}(u)
// h_{k,j}(v) with h_{k,p}(t) = exp(-t^2 / (2 sig_k^2)) t^p: a row pass with the
// sum(deg_k + 1) one-dimensional filters, then a column pass per basis function
// (725 k FP64 multiply-adds per 21 x 21 footprint instead of 9.5 M).  The stamp
// selection is exact: order statistics by radix selection on the values' bit
// patterns, the MAD on the FP64 differences the definition takes.
#include <math.h>

#include <algorithm>

#include "jobs.cuh"

namespace ipp {

// ---- stamp selection: one block per region ------------------------------------
constexpr int SS_T = 1024, SS_W = SS_T / 32;

struct StampRegion {
    const float* I;
    const float* R;
    int64_t pitch, W, H;
    int x0, y0, rw, rh;   // the region [x0, x0 + rw) x [y0, y0 + rh)
    int n;                // rw * rh
};

__device__ __forceinline__ float reg_r(const StampRegion& g, int t, int* x, int* y) {
    const int yy = t / g.rw;
    *y = g.y0 + yy;
    *x = g.x0 + (t - yy * g.rw);
    return __ldg(g.R + (int64_t)*y * g.pitch + *x);
}

// block sums / extrema (all threads call; result to all)
__device__ long long block_sum_ll(long long v, long long* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long s = 0;
    for (int w = 0; w < SS_W; w++) s += red[w];
    __syncthreads();
    return s;
}

__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* red) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long m = 0;
    for (int w = 0; w < SS_W; w++) m = red[w] > m ? red[w] : m;
    __syncthreads();
    return m;
}

__device__ unsigned long long block_min_u64(unsigned long long v, unsigned long long* red) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t < v ? t : v;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long m = ~0ull;
    for (int w = 0; w < SS_W; w++) m = red[w] < m ? red[w] : m;
    __syncthreads();
    return m;
}

// Keys of a region's finite values for the order statistics, as unsigned
// 64-bit integers ordered like the quantities they stand for:
//   mode 0: the value, fkey(v);
//   mode 1: |v - med| exactly, as the integer |v 2^-e0 - med 2^-e0| -- every value
//     and med are multiples of 2^e0 (e0: one below the smallest ulp in the
//     region), so the difference is exact and its FP64 rounding is the FP64
//     subtraction's, without the narrow FP64 pipe in the per-element work;
//   mode 2: the bit pattern of the FP64 |v - med| (when the region's range does
//     not fit 62 bits at scale 2^e0).
struct KeySpec {
    int mode;
    int e0;
    double med;
    long long imed;
};

__device__ __forceinline__ bool stamp_key(const StampRegion& g, int t, const KeySpec& ks, unsigned long long* k) {
    int x, y;
    const float v = reg_r(g, t, &x, &y);
    if (!isfinite(v)) return false;
    if (ks.mode == 0) {
        *k = fkey(v);
    } else if (ks.mode == 1) {
        const long long d = __float2ll_rz(ldexpf(v, -ks.e0)) - ks.imed;
        *k = (unsigned long long)(d < 0 ? -d : d);
    } else {
        *k = (unsigned long long)__double_as_longlong(fabs((double)v - ks.med));
    }
    return true;
}

// The k-th smallest key (0-based) of the region: radix selection, 8 bits a
// pass from bit top + 7 down, every key sharing the bits above top with
// prefix0; per-warp histograms in shared memory (hist: SS_W x 256 counters),
// fed by per-thread run lengths of equal digits.
__device__ unsigned long long block_select(const StampRegion& g, const KeySpec& ks, long long k, int top,
                                           unsigned long long prefix0, unsigned int* hist, int* sdig,
                                           long long* sbelow) {
    unsigned long long prefix = prefix0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int shift = top; shift >= 0; shift -= 8) {
        for (int t = threadIdx.x; t < SS_W * 256; t += SS_T) hist[t] = 0;
        __syncthreads();
        // each thread counts runs of equal digits over its elements (the region's
        // keys mostly share their high digits) and adds a run to its warp's
        // histogram when the digit changes
        unsigned cur = 256u, run = 0u;
        for (int t = threadIdx.x; t < g.n; t += SS_T) {
            unsigned long long key = 0;
            bool ok = stamp_key(g, t, ks, &key);
            if (ok && shift + 8 < 64) ok = (key >> (shift + 8)) == prefix;
            if (!ok) continue;
            const unsigned dig = (unsigned)((key >> shift) & 255u);
            if (dig == cur) {
                run++;
            } else {
                if (run) atomicAdd(&hist[warp * 256 + cur], run);
                cur = dig;
                run = 1u;
            }
        }
        if (run) atomicAdd(&hist[warp * 256 + cur], run);
        __syncthreads();
        // totals per digit (thread b < 256), then warp 0 finds the digit of rank k
        if (threadIdx.x < 256) {
            unsigned s = 0;
            for (int w = 0; w < SS_W; w++) s += hist[w * 256 + threadIdx.x];
            hist[threadIdx.x] = s;   // row 0 is no longer needed per warp
        }
        __syncthreads();
        if (warp == 0) {
            long long c8 = 0;
            for (int b = 0; b < 8; b++) c8 += hist[lane * 8 + b];
            long long inc = c8;
            for (int o = 1; o < 32; o <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            const long long exc = inc - c8;
            const unsigned hit = __ballot_sync(0xffffffffu, exc <= k && k < inc);
            if (hit && lane == __ffs(hit) - 1) {
                long long c = exc;
                int d = lane * 8;
                for (int b = 0; b < 8; b++) {
                    const long long nb = c + hist[lane * 8 + b];
                    if (k < nb) { d = lane * 8 + b; break; }
                    c = nb;
                }
                *sdig = d;
                *sbelow = c;
            }
        }
        __syncthreads();
        prefix = (prefix << 8) | (unsigned long long)*sdig;
        k -= *sbelow;
        __syncthreads();
    }
    return prefix;
}

// (count of keys <= kk, smallest key > kk) over the region
__device__ void block_count_next(const StampRegion& g, const KeySpec& ks, unsigned long long kk, long long* cnt,
                                 unsigned long long* next, long long* red, unsigned long long* redu) {
    long long c = 0;
    unsigned long long nx = ~0ull;
    for (int t = threadIdx.x; t < g.n; t += SS_T) {
        unsigned long long key;
        if (!stamp_key(g, t, ks, &key)) continue;
        if (key <= kk) c++;
        else if (key < nx) nx = key;
    }
    *cnt = block_sum_ll(c, red);
    *next = block_min_u64(nx, redu);
}

// the two middle order statistics (k0 = (n - 1) / 2, k1 = n / 2) as keys, for
// keys in [kmin, kmax]: the radix passes start at the highest byte where kmin
// and kmax differ
__device__ void block_middle(const StampRegion& g, const KeySpec& ks, long long n, unsigned long long kmin,
                             unsigned long long kmax, unsigned int* hist, long long* red, unsigned long long* redu,
                             int* sdig, long long* sbelow, unsigned long long* a, unsigned long long* b) {
    const long long k0 = (n - 1) / 2, k1 = n / 2;
    const unsigned long long dif = kmin ^ kmax;
    const int top = dif ? ((63 - __clzll((long long)dif)) & ~7) : 0;
    const unsigned long long prefix0 = top + 8 < 64 ? kmin >> (top + 8) : 0ull;
    *a = block_select(g, ks, k0, top, prefix0, hist, sdig, sbelow);
    if (k1 == k0) { *b = *a; return; }
    long long cle;
    unsigned long long nx;
    block_count_next(g, ks, *a, &cle, &nx, red, redu);
    *b = cle > k1 ? *a : nx;
}

// Is every pixel of the (2 m + 1)^2 box of A around (x, y) finite?  (block-wide)
__device__ bool block_box_finite(const float* A, int64_t pitch, int x, int y, int m) {
    const int s = 2 * m + 1;
    bool bad = false;
    for (int t = threadIdx.x; t < s * s; t += SS_T) {
        const int dy = t / s, dx = t - dy * s;
        if (!isfinite(__ldg(A + (int64_t)(y - m + dy) * pitch + (x - m + dx)))) bad = true;
    }
    return !__syncthreads_or(bad);
}

// One block per region: the candidate's pixel or -1.
__global__ void __launch_bounds__(SS_T) k_sub_stamps(const float* I, const float* R, int64_t W, int64_t H,
                                                     int64_t pitch, int nsx, int nsy, int hw, int fh, double nsig,
                                                     int2* reg_out) {
    __shared__ unsigned int hist[SS_W * 256];
    __shared__ long long red[SS_W];
    __shared__ unsigned long long redu[SS_W];
    __shared__ int sdig;
    __shared__ long long sbelow;
    const int sx = blockIdx.x % nsx, sy = blockIdx.x / nsx;
    StampRegion g;
    g.I = I; g.R = R; g.pitch = pitch; g.W = W; g.H = H;
    g.x0 = (int)(sx * W / nsx);
    g.y0 = (int)(sy * H / nsy);
    g.rw = (int)((sx + 1) * W / nsx) - g.x0;
    g.rh = (int)((sy + 1) * H / nsy) - g.y0;
    g.n = g.rw * g.rh;
    // the finite values: count, key range, smallest ulp exponent, largest |v|
    long long c = 0;
    unsigned long long kmin = ~0ull, kmax = 0, emin = ~0ull, amax = 0;
    for (int t = threadIdx.x; t < g.n; t += SS_T) {
        int x, y;
        const float v = reg_r(g, t, &x, &y);
        if (!isfinite(v)) continue;
        c++;
        const unsigned long long k = fkey(v);
        kmin = k < kmin ? k : kmin;
        kmax = k > kmax ? k : kmax;
        const uint32_t bits = __float_as_uint(v) & 0x7fffffffu, be = bits >> 23;
        const unsigned long long ue = be ? be : 1u;      // ulp 2^(be - 150), denormals as be = 1
        emin = ue < emin ? ue : emin;
        amax = bits > amax ? bits : amax;
    }
    const long long n = block_sum_ll(c, red);
    if (n == 0) {
        if (threadIdx.x == 0) reg_out[blockIdx.x] = make_int2(-1, -1);
        return;
    }
    kmin = block_min_u64(kmin, redu);
    kmax = block_max_u64(kmax, redu);
    emin = block_min_u64(emin, redu);
    amax = block_max_u64(amax, redu);
    // median (Eq. 1's even-count mean of the middle pair)
    KeySpec ks{0, 0, 0.0, 0};
    unsigned long long ka, kb;
    block_middle(g, ks, n, kmin, kmax, hist, red, redu, &sdig, &sbelow, &ka, &kb);
    const double va = (double)fkey_inv((uint32_t)ka), vb = (double)fkey_inv((uint32_t)kb);
    const double med = (n & 1) ? vb : __dmul_rn(0.5, __dadd_rn(va, vb));
    // MAD: exact integer differences at scale 2^e0 when they fit 62 bits
    ks.med = med;
    ks.e0 = (int)emin - 150 - 1;
    const double span = ldexp((double)__uint_as_float((uint32_t)amax) + fabs(med), -ks.e0);
    double mad;
    if (span < 4.6e18) {
        ks.mode = 1;
        ks.imed = __double2ll_rz(ldexp(med, -ks.e0));
        const unsigned long long top =
            (unsigned long long)ldexp((double)__uint_as_float((uint32_t)amax) + fabs(med), -ks.e0) + 1ull;
        block_middle(g, ks, n, 0ull, top, hist, red, redu, &sdig, &sbelow, &ka, &kb);
        const double da = ldexp((double)ka, ks.e0), db = ldexp((double)kb, ks.e0);
        mad = (n & 1) ? db : __dmul_rn(0.5, __dadd_rn(da, db));
    } else {
        ks.mode = 2;
        block_middle(g, ks, n, 0ull, ~0ull, hist, red, redu, &sdig, &sbelow, &ka, &kb);
        const double da = __longlong_as_double((long long)ka), db = __longlong_as_double((long long)kb);
        mad = (n & 1) ? db : __dmul_rn(0.5, __dadd_rn(da, db));
    }
    const double sgm = __dmul_rn(1.4826, mad);
    const double thr = __dadd_rn(med, __dmul_rn(nsig, sgm));
    // the brightest eligible pixel: arg-max rounds over the keys below the last
    // rejected one (fkey(v) << 32 | ~raster index: ties to the first pixel)
    const int m = fh + hw;
    unsigned long long bound = ~0ull;
    int bx = -1, by = -1;
    float best = 0.f;
    for (;;) {
        unsigned long long mk = 0;
        for (int t = threadIdx.x; t < g.n; t += SS_T) {
            int x, y;
            const float v = reg_r(g, t, &x, &y);
            if (!isfinite(v) || x < m || y < m || x > W - 1 - m || y > H - 1 - m) continue;
            const unsigned long long key =
                ((unsigned long long)fkey(v) << 32) | (unsigned long long)(~(uint32_t)((int64_t)y * W + x));
            if (key < bound && key > mk) mk = key;
        }
        mk = block_max_u64(mk, redu);
        if (mk == 0) break;                              // no eligible pixel left
        const uint32_t idx = ~(uint32_t)(mk & 0xffffffffu);
        const int x = (int)(idx % (uint32_t)W), y = (int)(idx / (uint32_t)W);
        if (block_box_finite(R, pitch, x, y, m) && block_box_finite(I, pitch, x, y, fh)) {
            bx = x; by = y;
            best = fkey_inv((uint32_t)(mk >> 32));
            break;
        }
        bound = mk;
    }
    if (threadIdx.x == 0)
        reg_out[blockIdx.x] = (bx >= 0 && (double)best > thr) ? make_int2(bx, by) : make_int2(-1, -1);
}

// Candidates in region order (row-major over the regions) and their count.
__global__ void __launch_bounds__(1024) k_sub_compact(const int2* reg, int nreg, int32_t* cx, int32_t* cy,
                                                      int32_t* n_dev) {
    __shared__ int red[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nreg; base += 1024) {
        const int r = base + threadIdx.x;
        const int2 v = r < nreg ? reg[r] : make_int2(-1, -1);
        const int f = v.x >= 0 ? 1 : 0;
        int inc = f;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) red[warp] = inc;
        __syncthreads();
        int before = carry;
        for (int w = 0; w < warp; w++) before += red[w];
        if (f) { cx[before + inc - 1] = v.x; cy[before + inc - 1] = v.y; }
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_dev = carry;
}

// ---- normal equations ---------------------------------------------------------
struct SubFitJob {
    const float* I;
    const float* R;
    int64_t pitch, W, H;
    const int32_t* cx;
    const int32_t* cy;
    const int32_t* n_dev;
    int max_c;
    int hw, fh, nk, nf;          // nf = sum (deg_k + 1) one-dimensional filters
    double sig[8];
    int fo[9];                   // first filter of Gaussian k
    int sord, bord, nb, ns, ng, np;
    int deg[8];
    double* C;                   // [max_c][nb][nfp]
    double* G;                   // [max_c][nb][nb] (m <= n)
    double* X;                   // [max_c][nb][ng]
    double* Y;                   // [max_c][nb]
    double* BB;                  // [max_c][ng][ng]
    double* BI;                  // [max_c][ng]
    double* Ps;                  // [max_c][ns]
    double* AtA;                 // [np][np]
    double* Atb;                 // [np]
};

// Spatial terms x^p y^q (p outer, q inner, p + q <= order) of the normalised
// coordinates xs = 2x / (W - 1) - 1, ys = 2y / (H - 1) - 1 (0 for one column / row).
__device__ void sub_terms_dev(double x, double y, int64_t W, int64_t H, int order, double* t) {
    const double xs = W > 1 ? __dsub_rn(__ddiv_rn(2.0 * x, (double)(W - 1)), 1.0) : 0.0;
    const double ys = H > 1 ? __dsub_rn(__ddiv_rn(2.0 * y, (double)(H - 1)), 1.0) : 0.0;
    int n = 0;
    double xp = 1.0;
    for (int p = 0; p <= order; p++) {
        double yq = 1.0;
        for (int q = 0; q <= order - p; q++) {
            t[n++] = __dmul_rn(xp, yq);
            yq = __dmul_rn(yq, ys);
        }
        xp = __dmul_rn(xp, xs);
    }
}

// one block per candidate: the footprint's C_n = R (x) K_n, separably
__global__ void __launch_bounds__(256) k_sub_conv(SubFitJob J) {
    extern __shared__ double sm[];
    if ((int)blockIdx.x >= min(*J.n_dev, J.max_c)) return;
    const int c = blockIdx.x;
    const int S = 2 * J.hw + 1, m = J.hw + J.fh, WS = 2 * m + 1, FW = 2 * J.fh + 1, nfp = FW * FW;
    double* h = sm;                    // [nf][S] one-dimensional filters
    double* Rw = h + J.nf * S;         // [WS][WS] the template around the candidate
    double* T = Rw + WS * WS;          // [nf][WS][FW] row-filtered template
    int2* bf = reinterpret_cast<int2*>(T + (size_t)J.nf * WS * FW);   // [nb] row and column filter of basis n
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < J.nk; k++)
            for (int i = 0; i <= J.deg[k]; i++)
                for (int j = 0; j <= J.deg[k] - i; j++) bf[n++] = make_int2(J.fo[k] + i, J.fo[k] + j);
    }
    for (int t = threadIdx.x; t < J.nf * S; t += 256) {
        const int f = t / S, u = t - f * S - J.hw;
        int k = 0;
        while (k + 1 < J.nk && f >= J.fo[k + 1]) k++;
        const int p = f - J.fo[k];
        double v = exp(-(double)(u * u) / (2.0 * J.sig[k] * J.sig[k]));
        for (int q = 0; q < p; q++) v *= (double)u;
        h[t] = v;
    }
    const int x0 = J.cx[c] - m, y0 = J.cy[c] - m;
    // a candidate whose support leaves the frame contributes nothing
    const bool inb = x0 >= 0 && y0 >= 0 && x0 + WS <= J.W && y0 + WS <= J.H;
    for (int t = threadIdx.x; t < WS * WS; t += 256) {
        const int r = t / WS, q = t - r * WS;
        Rw[t] = inb ? (double)__ldg(J.R + (int64_t)(y0 + r) * J.pitch + (x0 + q)) : 0.0;
    }
    __syncthreads();
    // rows: T[f][r][q] = sum_u h_f(u) R(x - u, row r), x = footprint column q
    for (int t = threadIdx.x; t < J.nf * WS * FW; t += 256) {
        const int f = t / (WS * FW), rq = t - f * WS * FW, r = rq / FW, q = rq - r * FW;
        const double* hf = h + f * S;
        const double* rr = Rw + r * WS + q + 2 * J.hw;   // R at column offset u = -hw .. hw: rr[-(u + hw)]
        double s = 0.0;
        for (int u = 0; u < S; u++) s = fma(hf[u], rr[-u], s);
        T[t] = s;
    }
    __syncthreads();
    // columns: C_n(p) = sum_v h_{k,j}(v) T_{k,i}(x, y - v)
    double* C = J.C + (size_t)c * J.nb * nfp;
    for (int t = threadIdx.x; t < J.nb * nfp; t += 256) {
        const int n = t / nfp, p = t - n * nfp, pr = p / FW, pq = p - pr * FW;
        const int fi = bf[n].x, fj = bf[n].y;
        const double* hv = h + fj * S;
        const double* tc = T + (size_t)fi * WS * FW + (pr + 2 * J.hw) * FW + pq;
        double s = 0.0;
        for (int v = 0; v < S; v++) s = fma(hv[v], tc[-v * FW], s);
        C[t] = s;
    }
}

// one block per candidate: its Gram matrix of the C_n, the cross terms with the
// background terms and the target, and the candidate's spatial terms
__global__ void __launch_bounds__(256) k_sub_gram(SubFitJob J) {
    extern __shared__ double sm[];
    if ((int)blockIdx.x >= min(*J.n_dev, J.max_c)) return;
    const int c = blockIdx.x;
    const int FW = 2 * J.fh + 1, nfp = FW * FW, nb = J.nb, ng = J.ng;
    double* Cs = sm;                   // [nb][nfp]
    double* Is = Cs + nb * nfp;        // [nfp]
    double* Pb = Is + nfp;             // [ng][nfp]
    const double* C = J.C + (size_t)c * nb * nfp;
    for (int t = threadIdx.x; t < nb * nfp; t += 256) Cs[t] = C[t];
    const int cx = J.cx[c], cy = J.cy[c], m = J.hw + J.fh;
    const bool inb = cx >= m && cy >= m && cx + m < J.W && cy + m < J.H;   // else every part is 0
    for (int p = threadIdx.x; p < nfp; p += 256) {
        const int pr = p / FW, pq = p - pr * FW;
        const int x = cx - J.fh + pq, y = cy - J.fh + pr;
        Is[p] = inb ? (double)__ldg(J.I + (int64_t)y * J.pitch + x) : 0.0;
        if (ng) {
            double tb[64];
            sub_terms_dev((double)x, (double)y, J.W, J.H, J.bord, tb);
            for (int b = 0; b < ng; b++) Pb[b * nfp + p] = inb ? tb[b] : 0.0;
        }
    }
    if (threadIdx.x == 0) {
        double ts[64];
        sub_terms_dev((double)cx, (double)cy, J.W, J.H, J.sord, ts);
        for (int s = 0; s < J.ns; s++) J.Ps[(size_t)c * J.ns + s] = ts[s];
    }
    __syncthreads();
    const int ntri = nb * (nb + 1) / 2;
    const int ntask = ntri + nb * ng + nb + ng * ng + ng;
    for (int t = threadIdx.x; t < ntask; t += 256) {
        const double *a, *b;
        double* out;
        if (t < ntri) {                                   // G[n][m], m <= n
            int n = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
            while (n * (n + 1) / 2 > t) n--;
            while ((n + 1) * (n + 2) / 2 <= t) n++;
            const int mm = t - n * (n + 1) / 2;
            a = Cs + n * nfp; b = Cs + mm * nfp;
            out = J.G + ((size_t)c * nb + n) * nb + mm;
        } else if (t < ntri + nb * ng) {                  // X[n][b] = sum C_n P_b
            const int u = t - ntri, n = u / ng, g = u - n * ng;
            a = Cs + n * nfp; b = Pb + g * nfp;
            out = J.X + ((size_t)c * nb + n) * ng + g;
        } else if (t < ntri + nb * ng + nb) {             // Y[n] = sum C_n I
            const int n = t - ntri - nb * ng;
            a = Cs + n * nfp; b = Is;
            out = J.Y + (size_t)c * nb + n;
        } else if (t < ntri + nb * ng + nb + ng * ng) {   // BB[g][h] = sum P_g P_h
            const int u = t - ntri - nb * ng - nb, g = u / ng, hh = u - g * ng;
            a = Pb + g * nfp; b = Pb + hh * nfp;
            out = J.BB + ((size_t)c * ng + g) * ng + hh;
        } else {                                          // BI[g] = sum P_g I
            const int g = t - ntri - nb * ng - nb - ng * ng;
            a = Pb + g * nfp; b = Is;
            out = J.BI + (size_t)c * ng + g;
        }
        double s = 0.0;
        for (int p = 0; p < nfp; p++) s = fma(a[p], b[p], s);
        *out = s;
    }
}

// AtA and Atb from the candidates' parts, summed in candidate order: one thread
// per entry of the lower triangle (both halves written)
__global__ void __launch_bounds__(256) k_sub_assemble(SubFitJob J) {
    const int nc = min(*J.n_dev, J.max_c);
    const int np = J.np, nk = J.nb * J.ns, ns = J.ns, nb = J.nb, ng = J.ng;
    const int ntri = np * (np + 1) / 2;
    for (int t = blockIdx.x * 256 + threadIdx.x; t < ntri + np; t += gridDim.x * 256) {
        if (t >= ntri) {                                   // Atb
            const int a = t - ntri;
            double s = 0.0;
            if (a < nk) {
                const int n = a / ns, sa = a - n * ns;
                for (int c = 0; c < nc; c++) s += J.Ps[(size_t)c * ns + sa] * J.Y[(size_t)c * nb + n];
            } else {
                const int g = a - nk;
                for (int c = 0; c < nc; c++) s -= J.BI[(size_t)c * ng + g];
            }
            J.Atb[a] = s;
            continue;
        }
        int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
        while (a * (a + 1) / 2 > t) a--;
        while ((a + 1) * (a + 2) / 2 <= t) a++;
        const int b = t - a * (a + 1) / 2;                 // b <= a
        double s = 0.0;
        if (a < nk) {                                      // both kernel unknowns
            const int n = a / ns, sa = a - n * ns, mm = b / ns, sb = b - mm * ns;
            const int hi = max(n, mm), lo = min(n, mm);
            for (int c = 0; c < nc; c++)
                s += J.Ps[(size_t)c * ns + sa] * J.Ps[(size_t)c * ns + sb] * J.G[((size_t)c * nb + hi) * nb + lo];
        } else if (b < nk) {                               // background row a, kernel column b
            const int g = a - nk, mm = b / ns, sb = b - mm * ns;
            for (int c = 0; c < nc; c++) s -= J.Ps[(size_t)c * ns + sb] * J.X[((size_t)c * nb + mm) * ng + g];
        } else {                                           // both background
            const int g = a - nk, hh = b - nk;
            for (int c = 0; c < nc; c++) s += J.BB[((size_t)c * ng + g) * ng + hh];
        }
        J.AtA[(size_t)a * np + b] = s;
        J.AtA[(size_t)b * np + a] = s;
    }
}

// Cholesky solve of AtA x = Atb in place, blocked and right-looking: for each
// panel of CB columns, the diagonal block is factored in shared memory
// (k_chol_diag), the rows below it are solved against it (k_chol_trsm, a warp
// per row), and the trailing lower triangle takes the panel's rank-CB update
// (k_chol_syrk, a 32 x 32 tile per block).  Then the two triangular solves,
// CB rows at a time (k_chol_solve).  FP64 throughout.  A pivot that is not
// positive sets *status = 1; the later kernels then leave everything as is.
constexpr int CB = 32;

__global__ void k_chol_init(int32_t* status) { *status = 0; }

__global__ void __launch_bounds__(256) k_chol_diag(double* A, int n, int k0, int32_t* status) {
    __shared__ double D[CB][CB + 1];
    __shared__ double rinv;
    __shared__ int fail;
    if (__ldcg(status)) return;
    const int b = min(CB, n - k0);
    for (int t = threadIdx.x; t < b * b; t += 256) {
        const int i = t / b, j = t - i * b;
        D[i][j] = A[(size_t)(k0 + i) * n + k0 + j];
    }
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < b; j++) {
        if (threadIdx.x == 0) {
            const double d = D[j][j];
            if (!(d > 0.0)) fail = 1;
            const double r = d > 0.0 ? sqrt(d) : 1.0;
            D[j][j] = r;
            rinv = 1.0 / r;
        }
        __syncthreads();
        if (fail) break;
        for (int i = j + 1 + threadIdx.x; i < b; i += 256) D[i][j] *= rinv;
        __syncthreads();
        for (int t = threadIdx.x; t < b * b; t += 256) {          // trailing update inside the block
            const int i = t / b, c = t - i * b;
            if (i > j && c > j && c <= i) D[i][c] -= D[i][j] * D[c][j];
        }
        __syncthreads();
    }
    if (fail) {
        if (threadIdx.x == 0) *status = 1;
        return;
    }
    for (int t = threadIdx.x; t < b * b; t += 256) {
        const int i = t / b, j = t - i * b;
        if (j <= i) A[(size_t)(k0 + i) * n + k0 + j] = D[i][j];
    }
}

// rows i >= k0 + CB: L21[i] = A21[i] L11^-T, one warp per row (lane j holds column j)
__global__ void __launch_bounds__(256) k_chol_trsm(double* A, int n, int k0, const int32_t* status) {
    __shared__ double L[CB][CB + 1];
    if (__ldcg(status)) return;
    const int b = min(CB, n - k0);
    for (int t = threadIdx.x; t < b * b; t += 256) {
        const int i = t / b, j = t - i * b;
        L[i][j] = j <= i ? A[(size_t)(k0 + i) * n + k0 + j] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = k0 + b + blockIdx.x * 8 + warp; i < n; i += gridDim.x * 8) {
        double a = lane < b ? A[(size_t)i * n + k0 + lane] : 0.0;
        double x = 0.0;
        for (int j = 0; j < b; j++) {
            const double xj = __shfl_sync(0xffffffffu, lane == j ? a / L[j][j] : 0.0, j);
            if (lane == j) x = xj;
            if (lane > j) a -= xj * L[lane][j];
        }
        if (lane < b) A[(size_t)i * n + k0 + lane] = x;
    }
}

// trailing update of the lower triangle from row / column k0 + CB on: tile
// (ti, tc), ti >= tc, of 32 x 32, A[i][c] -= sum_m L[i][k0 + m] L[c][k0 + m]
__global__ void __launch_bounds__(256) k_chol_syrk(double* A, int n, int k0, const int32_t* status) {
    __shared__ double Li[32][CB + 1], Lc[32][CB + 1];
    if (__ldcg(status)) return;
    const int r0 = k0 + CB;
    const int t = blockIdx.x;
    int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while (ti * (ti + 1) / 2 > t) ti--;
    while ((ti + 1) * (ti + 2) / 2 <= t) ti++;
    const int tc = t - ti * (ti + 1) / 2;
    const int i0 = r0 + ti * 32, c0 = r0 + tc * 32;
    for (int q = threadIdx.x; q < 32 * CB; q += 256) {
        const int r = q / CB, m = q - r * CB;
        Li[r][m] = i0 + r < n ? A[(size_t)(i0 + r) * n + k0 + m] : 0.0;
        Lc[r][m] = c0 + r < n ? A[(size_t)(c0 + r) * n + k0 + m] : 0.0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 32 * 32; q += 256) {
        const int r = q >> 5, c = q & 31;
        const int i = i0 + r, cc = c0 + c;
        if (i >= n || cc >= n || cc > i) continue;
        double acc = 0.0;
        for (int m = 0; m < CB; m++) acc = fma(Li[r][m], Lc[c][m], acc);
        A[(size_t)i * n + cc] -= acc;
    }
}

// L y = b, then L' x = y, CB rows at a time: the block's warps first take the
// dot products with the part already solved (a warp per row), then warp 0
// solves the CB x CB triangle.  The solution goes to b (and x64 / x32).
// the CB x CB diagonal block of L at r0 (bsz rows) in shared memory, and the
// reciprocals of its diagonal, for the sequential part of a solve step
__device__ __forceinline__ void chol_stage_block(const double* A, int n, int r0, int bsz, double (*Ld)[CB + 1],
                                                 double* rd) {
    for (int t = threadIdx.x; t < bsz * bsz; t += 1024) {
        const int i = t / bsz, j = t - i * bsz;
        Ld[i][j] = A[(size_t)(r0 + i) * n + r0 + j];
    }
    if (threadIdx.x < bsz) rd[threadIdx.x] = 1.0 / A[(size_t)(r0 + threadIdx.x) * n + r0 + threadIdx.x];
}

__global__ void __launch_bounds__(1024) k_chol_solve(const double* A, double* b, int n, double* x64, float* x32,
                                                     const int32_t* status) {
    __shared__ double part[CB], rd[CB];
    __shared__ double Ld[CB][CB + 1];
    if (__ldcg(status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r0 = 0; r0 < n; r0 += CB) {                 // forward
        const int bsz = min(CB, n - r0);
        chol_stage_block(A, n, r0, bsz, Ld, rd);
        if (warp < bsz) {
            const int i = r0 + warp;
            double s = 0.0;
            for (int k = lane; k < r0; k += 32) s = fma(A[(size_t)i * n + k], b[k], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) part[warp] = b[i] - s;
        }
        __syncthreads();
        if (warp == 0) {
            double y = lane < bsz ? part[lane] : 0.0, x = 0.0;
            for (int j = 0; j < bsz; j++) {
                const double xj = __shfl_sync(0xffffffffu, y * rd[j], j);
                if (lane == j) x = xj;
                if (lane > j && lane < bsz) y -= Ld[lane][j] * xj;
            }
            if (lane < bsz) b[r0 + lane] = x;
        }
        __syncthreads();
    }
    const int nblk = (n + CB - 1) / CB;
    for (int blk = nblk - 1; blk >= 0; blk--) {          // backward with L'
        const int r0 = blk * CB, bsz = min(CB, n - r0);
        chol_stage_block(A, n, r0, bsz, Ld, rd);
        if (warp < bsz) {
            const int i = r0 + warp;
            double s = 0.0;
            for (int k = r0 + bsz + lane; k < n; k += 32) s = fma(A[(size_t)k * n + i], b[k], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) part[warp] = b[i] - s;
        }
        __syncthreads();
        if (warp == 0) {
            double y = lane < bsz ? part[lane] : 0.0, x = 0.0;
            for (int j = bsz - 1; j >= 0; j--) {
                const double xj = __shfl_sync(0xffffffffu, y * rd[j], j);
                if (lane == j) x = xj;
                if (lane < j) y -= Ld[j][lane] * xj;
            }
            if (lane < bsz) b[r0 + lane] = x;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += 1024) {
        if (x64) x64[i] = b[i];
        if (x32) x32[i] = (float)b[i];
    }
}

}  // namespace ipp

using namespace ipp;

namespace {
size_t a256s(size_t x) { return (x + 255) & ~(size_t)255; }

struct SubDims {
    int nb, ns, ng, np, nf, nfp, WS, S;
    size_t conv_smem, gram_smem;
};

SubDims sub_dims(int hw, int fh, int nk, const int32_t* deg, int sord, int bord) {
    SubDims d{};
    for (int k = 0; k < nk; k++) { d.nb += (deg[k] + 1) * (deg[k] + 2) / 2; d.nf += deg[k] + 1; }
    d.ns = (sord + 1) * (sord + 2) / 2;
    d.ng = bord >= 0 ? (bord + 1) * (bord + 2) / 2 : 0;
    d.np = d.nb * d.ns + d.ng;
    d.S = 2 * hw + 1;
    d.WS = 2 * (hw + fh) + 1;
    const int FW = 2 * fh + 1;
    d.nfp = FW * FW;
    d.conv_smem = sizeof(double) * ((size_t)d.nf * d.S + (size_t)d.WS * d.WS + (size_t)d.nf * d.WS * FW) +
                  sizeof(int2) * (size_t)d.nb;
    d.gram_smem = sizeof(double) * ((size_t)d.nb * d.nfp + d.nfp + (size_t)d.ng * d.nfp);
    return d;
}

// workspace: region results, then the per-candidate parts, the normal
// equations and the candidate list of ipp_sub_fit
size_t sub_carve(const SubDims& d, int max_c, int nreg, void* base, SubFitJob* J, int2** reg, int32_t** cxy) {
    const size_t mc = (size_t)std::max(max_c, 1);
    const size_t sz[] = {(size_t)std::max(nreg, 1) * sizeof(int2), mc * d.nb * d.nfp * 8, mc * d.nb * d.nb * 8,
                         mc * d.nb * std::max(d.ng, 1) * 8, mc * d.nb * 8, mc * std::max(d.ng * d.ng, 1) * 8,
                         mc * std::max(d.ng, 1) * 8, mc * d.ns * 8, (size_t)d.np * d.np * 8, (size_t)d.np * 8,
                         (2 * mc + 1) * sizeof(int32_t)};
    constexpr int NA = sizeof(sz) / sizeof(sz[0]);
    size_t off[NA], o = 0;
    for (int k = 0; k < NA; k++) { off[k] = o; o += a256s(sz[k]); }
    if (base) {
        unsigned char* b = static_cast<unsigned char*>(base);
        if (reg) *reg = reinterpret_cast<int2*>(b + off[0]);
        if (J) {
            J->C = reinterpret_cast<double*>(b + off[1]);
            J->G = reinterpret_cast<double*>(b + off[2]);
            J->X = reinterpret_cast<double*>(b + off[3]);
            J->Y = reinterpret_cast<double*>(b + off[4]);
            J->BB = reinterpret_cast<double*>(b + off[5]);
            J->BI = reinterpret_cast<double*>(b + off[6]);
            J->Ps = reinterpret_cast<double*>(b + off[7]);
            J->AtA = reinterpret_cast<double*>(b + off[8]);
            J->Atb = reinterpret_cast<double*>(b + off[9]);
        }
        if (cxy) *cxy = reinterpret_cast<int32_t*>(b + off[10]);
    }
    return o;
}
}  // namespace

size_t ipp_subfit_ws_bytes(int max_c, int nreg, int hw, int fh, int nk, const int32_t* deg, int sord, int bord) {
    return sub_carve(sub_dims(hw, fh, nk, deg, sord, bord), max_c, nreg, nullptr, nullptr, nullptr, nullptr);
}

size_t ipp_subfit_smem(int hw, int fh, int nk, const int32_t* deg, int sord, int bord) {
    const SubDims d = sub_dims(hw, fh, nk, deg, sord, bord);
    return std::max(d.conv_smem, d.gram_smem);
}

int ipp_launch_sub_stamps(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int nsx, int nsy,
                          int hw, int fh, double nsig, int32_t* cx, int32_t* cy, int32_t* n_dev, void* ws,
                          cudaStream_t s) {
    int2* reg = static_cast<int2*>(ws);   // the first array of the workspace
    k_sub_stamps<<<(unsigned)(nsx * nsy), SS_T, 0, s>>>(I, R, W, H, pitch, nsx, nsy, hw, fh, nsig, reg);
    if (int e = ipp_check_launch("k_sub_stamps")) return e;
    k_sub_compact<<<1, 1024, 0, s>>>(reg, nsx * nsy, cx, cy, n_dev);
    return ipp_check_launch("k_sub_compact");
}

int ipp_launch_sub_normal(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, const int32_t* cx,
                          const int32_t* cy, const int32_t* n_dev, int max_c, int nreg, int hw, int fh, int nk,
                          const double* sig, const int32_t* deg, int sord, int bord, double* AtA, double* Atb,
                          void* ws, cudaStream_t s) {
    const SubDims d = sub_dims(hw, fh, nk, deg, sord, bord);
    SubFitJob J{};
    sub_carve(d, max_c, nreg, ws, &J, nullptr, nullptr);
    J.I = I; J.R = R; J.pitch = pitch; J.W = W; J.H = H;
    J.cx = cx; J.cy = cy; J.n_dev = n_dev; J.max_c = max_c;
    J.hw = hw; J.fh = fh; J.nk = nk; J.nf = d.nf;
    J.fo[0] = 0;
    for (int k = 0; k < nk; k++) { J.sig[k] = sig[k]; J.deg[k] = deg[k]; J.fo[k + 1] = J.fo[k] + deg[k] + 1; }
    J.sord = sord; J.bord = bord; J.nb = d.nb; J.ns = d.ns; J.ng = d.ng; J.np = d.np;
    if (AtA) J.AtA = AtA;
    if (Atb) J.Atb = Atb;
    if (max_c < 1) return IPP_OK;
    cudaFuncSetAttribute(k_sub_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.conv_smem);
    cudaFuncSetAttribute(k_sub_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.gram_smem);
    k_sub_conv<<<(unsigned)max_c, 256, d.conv_smem, s>>>(J);
    if (int e = ipp_check_launch("k_sub_conv")) return e;
    k_sub_gram<<<(unsigned)max_c, 256, d.gram_smem, s>>>(J);
    if (int e = ipp_check_launch("k_sub_gram")) return e;
    const int nt = d.np * (d.np + 1) / 2 + d.np;
    k_sub_assemble<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(J);
    return ipp_check_launch("k_sub_assemble");
}

int ipp_launch_sub_solve(double* AtA, double* Atb, int np, double* coef64, float* coef, int32_t* status,
                         cudaStream_t s) {
    k_chol_init<<<1, 1, 0, s>>>(status);
    if (int e = ipp_check_launch("k_chol_init")) return e;
    for (int k0 = 0; k0 < np; k0 += CB) {
        k_chol_diag<<<1, 256, 0, s>>>(AtA, np, k0, status);
        if (int e = ipp_check_launch("k_chol_diag")) return e;
        const int rest = np - k0 - CB;
        if (rest <= 0) break;
        k_chol_trsm<<<(unsigned)std::min((rest + 7) / 8, 152), 256, 0, s>>>(AtA, np, k0, status);
        if (int e = ipp_check_launch("k_chol_trsm")) return e;
        const int nt = (rest + 31) / 32;
        k_chol_syrk<<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(AtA, np, k0, status);
        if (int e = ipp_check_launch("k_chol_syrk")) return e;
    }
    k_chol_solve<<<1, 1024, 0, s>>>(AtA, Atb, np, coef64, coef, status);
    return ipp_check_launch("k_chol_solve");
}

int ipp_launch_sub_fit(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int nsx, int nsy,
                       double nsig, int hw, int fh, int nk, const double* sig, const int32_t* deg, int sord, int bord,
                       double* coef64, float* coef, int32_t* cx_out, int32_t* cy_out, int32_t* n_out,
                       int32_t* status, void* ws, cudaStream_t s) {
    const SubDims d = sub_dims(hw, fh, nk, deg, sord, bord);
    const int nreg = nsx * nsy;
    SubFitJob J{};
    int32_t* cxy = nullptr;
    sub_carve(d, nreg, nreg, ws, &J, nullptr, &cxy);
    int32_t* cx = cx_out ? cx_out : cxy;
    int32_t* cy = cy_out ? cy_out : cxy + nreg;
    int32_t* nd = n_out ? n_out : cxy + 2 * nreg;
    if (int e = ipp_launch_sub_stamps(I, R, W, H, pitch, nsx, nsy, hw, fh, nsig, cx, cy, nd, ws, s)) return e;
    if (int e = ipp_launch_sub_normal(I, R, W, H, pitch, cx, cy, nd, nreg, nreg, hw, fh, nk, sig, deg, sord, bord,
                                      nullptr, nullptr, ws, s))
        return e;
    return ipp_launch_sub_solve(J.AtA, J.Atb, d.np, coef64, coef, status, s);
}
