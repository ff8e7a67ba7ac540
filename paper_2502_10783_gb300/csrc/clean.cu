// clean.cu -- cleaning of the deblended objects (Sec. 2.2.5: each object is
// tested against its neighbours, and one that does not stand out from them is
// merged into them).  The reading, after SExtractor's cleaning:
//   per object, from its pixels: the peak (largest value, first in raster order
//   on ties), the barycentre and second moments weighted by the positive
//   values (1/12 added to x2 and y2 when x2 y2 - xy^2 < 1/144; no positive
//   pixel: the unweighted centre, x2 = y2 = 1/12, xy = 0);
//   the model of object j at a pixel: peak_j (1 + r^2 / a^2)^-beta, r^2 the
//   moments' elliptical radius (y2 dx^2 - 2 xy dx dy + x2 dy^2) / det, with
//   a^2 = 2 ln 2 / (2^(1/beta) - 1) (the FWHM of the Gaussian of those moments);
//   object i is spurious when its peak less the models of every brighter object
//   (larger peak; equal peaks: smaller label) at its peak pixel is below the
//   detection threshold there; it merges into the brighter object whose model
//   is largest there (ties: the smaller label), merges followed to a kept
//   object; kept objects are renumbered 1.. in label order (a label with no
//   pixel is no object and takes no number).
//
// Kernels: per-pixel statistics with atomics (the peak as one 64-bit key; the
// weighted sums as exact integer pairs, so the barycentres do not depend on the
// order of the adds), per-object moments, a bitonic sort of the objects by
// brightness (so that the objects brighter than one are a prefix), the test
// tiled over (object, chunk of brighter objects) blocks with compensated
// partial sums combined in chunk order, merge targets followed to their roots,
// a label-order scan and the relabelled map.
#include "jobs.cuh"

namespace ipp {

constexpr int CL_T = 256;

// one chunk's share of the test of one object: compensated sum of the models,
// the largest model and its label
struct __align__(16) CleanPart { float s_hi, s_lo, best; int bj; };

// per-object workspace (arrays of max_obj + 1 entries; index = label)
struct CleanWs {
    unsigned long long* pkey;   // fkey(peak) << 32 | ~raster index (max = largest, then first)
    long long* sw;              // [2 (n+1)] sum f over positive f (pairs in 2^-8 and 2^-40 units)
    long long* swx;             // [2 (n+1)] sum f x (pairs in 2^-8 and 2^-32 units)
    long long* swy;             // [2 (n+1)] sum f y
    long long* cnt;             // pixel count, sum x, sum y (unweighted) [3 (n+1)]
    long long* mom;             // [6 (n+1)] sum f dx^2, f dy^2, f dx dy about the barycentre (pairs)
    float4* geo;                // cx, cy, peak, valid
    float2* blo;                // the barycentre's remainders: cx + lo.x, cy + lo.y to ~2^-48
    float4* ell;                // y2 / (det a^2), -2 xy / (det a^2), x2 / (det a^2), threshold at the peak
    int32_t* into;              // merge target
    int32_t* num;               // the kept object a label's merges lead to
    int32_t* tcount;            // kept objects per tile of 1024 labels
    unsigned long long* skey;   // [P] brightness sort keys
    CleanPart* part;            // [nchunk][P] per-chunk partials of the test
    int P;                      // sort size (a power of two >= max_obj, >= 2048)
};

// where the detection threshold comes from: a map (pitch W), else the mesh rms
// (k rms, floored at thresh_abs), else thresh_abs alone
struct CleanThr {
    const float* map;
    const float* mesh_rms;
    int nx, ny;
    float mesh_w, mesh_h, k, thresh_abs;
    int64_t W;
};

__device__ __forceinline__ int clean_n(const int32_t* n_dev, int32_t max_obj) {
    return max(0, min(__ldg(n_dev), max_obj));
}

__global__ void __launch_bounds__(CL_T) k_clean_pix_a(const float* sub, int64_t pitch, const int32_t* labels,
                                                      int64_t W, int64_t H, const int32_t* n_dev, int32_t max_obj,
                                                      CleanWs ws) {
    const int n = clean_n(n_dev, max_obj);
    for (int64_t p = (int64_t)blockIdx.x * CL_T + threadIdx.x; p < W * H; p += (int64_t)gridDim.x * CL_T) {
        const int l = __ldg(labels + p);
        if (l <= 0 || l > n) continue;
        const int64_t y = p / W, x = p - y * W;
        const float f = __ldg(sub + y * pitch + x);
        const unsigned long long key = ((unsigned long long)fkey(f) << 32) | (unsigned long long)(~(uint32_t)p);
        atomicMax(ws.pkey + l, key);
        atomicAdd(reinterpret_cast<unsigned long long*>(ws.cnt + 3 * l), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(ws.cnt + 3 * l + 1), (unsigned long long)x);
        atomicAdd(reinterpret_cast<unsigned long long*>(ws.cnt + 3 * l + 2), (unsigned long long)y);
        if (f > 0.f) {
            long long t[2];
            fx_split(f, t);
            // the coordinate-weighted residuals in 2^-32 units: |t1 >> 8| < 2^23,
            // so x < 2^16 keeps 2^24 pixels of one object inside 64 bits
            const long long r32 = t[1] >> 8;
            atomicAdd(reinterpret_cast<unsigned long long*>(ws.sw + 2 * l), (unsigned long long)t[0]);
            atomicAdd(reinterpret_cast<unsigned long long*>(ws.sw + 2 * l + 1), (unsigned long long)t[1]);
            atomicAdd(reinterpret_cast<unsigned long long*>(ws.swx + 2 * l), (unsigned long long)(t[0] * x));
            atomicAdd(reinterpret_cast<unsigned long long*>(ws.swx + 2 * l + 1), (unsigned long long)(r32 * x));
            atomicAdd(reinterpret_cast<unsigned long long*>(ws.swy + 2 * l), (unsigned long long)(t[0] * y));
            atomicAdd(reinterpret_cast<unsigned long long*>(ws.swy + 2 * l + 1), (unsigned long long)(r32 * y));
        }
    }
}

__device__ __forceinline__ df pair32_value(const long long* p) {
    const df a = df_from_i64(__ldcg(p)), b = df_from_i64(__ldcg(p + 1));
    return df_add(df_scale(a, 1.0f / 256.0f), df_scale(b, 1.0f / 4294967296.0f));
}

// barycentres (exact sums, double-float quotient)
__global__ void __launch_bounds__(CL_T) k_clean_obj_a(const int32_t* n_dev, int32_t max_obj, CleanWs ws) {
    const int n = clean_n(n_dev, max_obj);
    for (int l = blockIdx.x * CL_T + threadIdx.x; l <= n; l += gridDim.x * CL_T) {
        if (l == 0) continue;
        const long long c = ws.cnt[3 * l];
        float cx = 0.f, cy = 0.f, lx = 0.f, ly = 0.f;
        const df sw = fx_value(ws.sw + 2 * l);
        if (sw.hi > 0.f) {
            const df bx = df_div(pair32_value(ws.swx + 2 * l), sw), by = df_div(pair32_value(ws.swy + 2 * l), sw);
            cx = __fadd_rn(bx.hi, bx.lo);
            cy = __fadd_rn(by.hi, by.lo);
            lx = (bx.hi - cx) + bx.lo;
            ly = (by.hi - cy) + by.lo;
        } else if (c > 0) {
            const df sx = df_from_i64(ws.cnt[3 * l + 1]), sy = df_from_i64(ws.cnt[3 * l + 2]), n = df_from_i64(c);
            const df bx = df_div(sx, n), by = df_div(sy, n);
            cx = __fadd_rn(bx.hi, bx.lo);
            cy = __fadd_rn(by.hi, by.lo);
            lx = (bx.hi - cx) + bx.lo;
            ly = (by.hi - cy) + by.lo;
        }
        ws.blo[l] = make_float2(lx, ly);
        const unsigned long long k = ws.pkey[l];
        const float pk = c > 0 ? fkey_inv((uint32_t)(k >> 32)) : -INFINITY;
        ws.geo[l] = make_float4(cx, cy, pk, c > 0 ? 1.f : 0.f);
    }
}

__global__ void __launch_bounds__(CL_T) k_clean_pix_b(const float* sub, int64_t pitch, const int32_t* labels,
                                                      int64_t W, int64_t H, const int32_t* n_dev, int32_t max_obj,
                                                      CleanWs ws) {
    const int n = clean_n(n_dev, max_obj);
    for (int64_t p = (int64_t)blockIdx.x * CL_T + threadIdx.x; p < W * H; p += (int64_t)gridDim.x * CL_T) {
        const int l = __ldg(labels + p);
        if (l <= 0 || l > n) continue;
        const int64_t y = p / W, x = p - y * W;
        const float f = __ldg(sub + y * pitch + x);
        if (!(f > 0.f)) continue;
        const float4 g = ws.geo[l];
        const float2 lo = ws.blo[l];
        const float dx = ((float)x - g.x) - lo.x, dy = ((float)y - g.y) - lo.y;
        // exact sums of the FP32 terms: the moments do not depend on the order
        fx_atomic_add(ws.mom + 6 * l, f * dx * dx);
        fx_atomic_add(ws.mom + 6 * l + 2, f * dy * dy);
        fx_atomic_add(ws.mom + 6 * l + 4, f * dx * dy);
    }
}

// the detection threshold at pixel (x, y): max(k rms(x, y), thresh_abs), rms the
// Keys interpolation of the mesh rms (nodes clamped at the grid's edges)
__device__ float clean_thr_at(const CleanThr& T, int64_t x, int64_t y) {
    if (T.map) return __ldg(T.map + y * T.W + x);
    if (!T.mesh_rms) return T.thresh_abs;
    const float u = ((float)x + 0.5f) / T.mesh_w - 0.5f, v = ((float)y + 0.5f) / T.mesh_h - 0.5f;
    const float qf = floorf(u), pf = floorf(v);
    float wx[4], wy[4];
    keys_weights(u - qf, wx);
    keys_weights(v - pf, wy);
    const int q0 = (int)qf, p0 = (int)pf;
    float acc = 0.f;
    for (int a = 0; a < 4; a++) {
        const int p = clampi(p0 - 1 + a, 0, T.ny - 1);
        float r = 0.f;
        for (int b = 0; b < 4; b++) r = fmaf(wx[b], __ldg(T.mesh_rms + p * T.nx + clampi(q0 - 1 + b, 0, T.nx - 1)), r);
        acc = fmaf(wy[a], r, acc);
    }
    return fmaxf(T.k * acc, T.thresh_abs);
}

// moments, the model's inverse shape, and the threshold at the peak pixel
__global__ void __launch_bounds__(CL_T) k_clean_obj_b(const int32_t* n_dev, int32_t max_obj, CleanWs ws,
                                                      CleanThr T, float inv_a2) {
    const int n = clean_n(n_dev, max_obj);
    for (int l = blockIdx.x * CL_T + threadIdx.x; l <= n; l += gridDim.x * CL_T) {
        if (l == 0) continue;
        const df sw = fx_value(ws.sw + 2 * l);
        float x2 = 1.0f / 12.0f, y2 = 1.0f / 12.0f, xy = 0.f;
        if (sw.hi > 0.f) {
            const df m0 = df_div(fx_value(ws.mom + 6 * l), sw), m1 = df_div(fx_value(ws.mom + 6 * l + 2), sw),
                     m2 = df_div(fx_value(ws.mom + 6 * l + 4), sw);
            x2 = __fadd_rn(m0.hi, m0.lo);
            y2 = __fadd_rn(m1.hi, m1.lo);
            xy = __fadd_rn(m2.hi, m2.lo);
            if (x2 * y2 - xy * xy < 1.0f / 144.0f) { x2 += 1.0f / 12.0f; y2 += 1.0f / 12.0f; }
        }
        const float det = x2 * y2 - xy * xy;
        const float k = inv_a2 / det;
        float thr = T.thresh_abs;
        if (ws.geo[l].w > 0.f) {
            const uint32_t pix = ~(uint32_t)(ws.pkey[l] & 0xffffffffu);
            thr = clean_thr_at(T, pix % (uint32_t)T.W, pix / (uint32_t)T.W);
        }
        ws.ell[l] = make_float4(y2 * k, -2.0f * xy * k, x2 * k, thr);
    }
}

// ---- brightness order ------------------------------------------------------
// Sort key of label l: (~fkey(peak) << 32) | l, so that ascending keys run from
// the brightest object down, equal peaks by label -- the "brighter" relation of
// the test.  Empty labels and padding take the largest key and sort last.
// Bitonic sort of P = 2^m keys: 2048-key blocks in shared memory, the strides
// of 2048 and more in global passes.
constexpr int BS_T = 1024, BS_N = 2 * BS_T;

__global__ void __launch_bounds__(CL_T) k_clean_keys(const int32_t* n_dev, int32_t max_obj, CleanWs ws, int P) {
    const int n = clean_n(n_dev, max_obj);
    for (int r = blockIdx.x * CL_T + threadIdx.x; r < P; r += gridDim.x * CL_T) {
        const int l = r + 1;
        unsigned long long k = ~0ull;
        if (l <= n && ws.geo[l].w > 0.f)
            k = ((unsigned long long)(~fkey(ws.geo[l].z)) << 32) | (unsigned long long)(uint32_t)l;
        ws.skey[r] = k;
    }
}

__device__ __forceinline__ void bitonic_cas(unsigned long long& a, unsigned long long& b, bool up) {
    if ((a > b) == up) { const unsigned long long t = a; a = b; b = t; }
}

// k in [k_lo, k_hi] (powers of two), strides below BS_N only; k_lo = 2 sorts the
// block from scratch, k_lo = k_hi finishes one merge of size k
__global__ void __launch_bounds__(BS_T) k_bitonic_local(unsigned long long* keys, int k_lo, int k_hi) {
    __shared__ unsigned long long sk[BS_N];
    const int base = blockIdx.x * BS_N;
    sk[threadIdx.x] = keys[base + threadIdx.x];
    sk[threadIdx.x + BS_T] = keys[base + threadIdx.x + BS_T];
    __syncthreads();
    for (int k = k_lo; k <= k_hi; k <<= 1) {
        for (int j = min(k >> 1, BS_N >> 1); j > 0; j >>= 1) {
            const int t = threadIdx.x;
            const int i = 2 * t - (t & (j - 1));   // the lower element of this thread's pair
            const bool up = ((base + i) & k) == 0;
            bitonic_cas(sk[i], sk[i + j], up);
            __syncthreads();
        }
    }
    keys[base + threadIdx.x] = sk[threadIdx.x];
    keys[base + threadIdx.x + BS_T] = sk[threadIdx.x + BS_T];
}

__global__ void __launch_bounds__(CL_T) k_bitonic_global(unsigned long long* keys, int P, int k, int j) {
    const int t = blockIdx.x * CL_T + threadIdx.x;
    if (t >= P / 2) return;
    const int i = 2 * t - (t & (j - 1));
    const bool up = (i & k) == 0;
    unsigned long long a = keys[i], b = keys[i + j];
    if ((a > b) == up) { keys[i] = b; keys[i + j] = a; }
}

// ---- the test ----------------------------------------------------------------
// In brightness order the objects brighter than the one of rank r are the ranks
// 0..r-1.  Block (bi, bc): ranks [256 bi, 256 bi + 256) against the ranks of chunk
// bc ([CL_JC bc, CL_JC (bc + 1))), staged through shared memory 256 at a time.
// Each thread sums its models in rank order with a compensated (Kahan) FP32
// accumulator and keeps the largest model (ties: the smaller label); the chunks'
// partials are combined in chunk order by k_clean_decide, so the result does not
// depend on the scheduling.
constexpr int CL_JC = 4096;


__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float t = hi + v;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (v - bp);
    hi = t;
}

// Kahan-compensated accumulation: the total is s - c (error bound 2 eps of the
// sum of magnitudes, whatever the order of the terms)
__device__ __forceinline__ void kahan_acc(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

template <bool UNIT>
__global__ void __launch_bounds__(CL_T) k_clean_pairs(const int32_t* n_dev, int32_t max_obj, CleanWs ws, int64_t W,
                                                      float beta) {
    __shared__ float4 sa[CL_T], sq[CL_T];   // (cx, cy, peak, lo.x), (y2', -2 xy', x2', lo.y) of object rank t
    __shared__ int sb[CL_T];                // its label
    const int n = clean_n(n_dev, max_obj);
    const int r0 = blockIdx.x * CL_T, c0 = blockIdx.y * CL_JC;
    if (r0 >= n || c0 >= min(n, r0 + CL_T)) return;     // nothing brighter here
    const int r = r0 + threadIdx.x;
    const unsigned long long key = r < n ? ws.skey[r] : ~0ull;
    const bool valid = key != ~0ull;
    const int li = valid ? (int)(uint32_t)key : 0;
    float px = 0.f, py = 0.f;
    if (valid) {
        const uint32_t pix = ~(uint32_t)(ws.pkey[li] & 0xffffffffu);
        const uint32_t yy = pix / (uint32_t)W;
        py = (float)yy;
        px = (float)(pix - yy * (uint32_t)W);
    }
    float sum = 0.f, comp = 0.f, best = -1.f;
    int bj = -1;
    const int c1 = min(min(c0 + CL_JC, n), r0 + CL_T);
    const int lim = valid ? min(c1, r) : c0;              // ranks c0..lim-1 are brighter than r
    for (int t0 = c0; t0 < c1; t0 += CL_T) {
        __syncthreads();
        const int jr = t0 + threadIdx.x;
        if (jr < c1) {
            const unsigned long long kj = ws.skey[jr];
            const int lj = kj != ~0ull ? (int)(uint32_t)kj : 0;
            sb[threadIdx.x] = lj;
            if (lj > 0) {
                const float4 g = ws.geo[lj], e = ws.ell[lj];
                const float2 o = ws.blo[lj];
                sa[threadIdx.x] = make_float4(g.x, g.y, g.z, o.x);
                sq[threadIdx.x] = make_float4(e.x, e.y, e.z, o.y);
            }
        }
        __syncthreads();
        const int m = min(CL_T, lim - t0);
        for (int t = 0; t < m; t++) {
            const float4 a = sa[t], e = sq[t];
            const float dx = (px - a.x) - a.w, dy = (py - a.y) - e.w;
            // r^2 / a^2 = dx (y2' dx - 2 xy' dy) + x2' dy^2
            const float q = fmaf(dx, fmaf(e.x, dx, e.y * dy), e.z * dy * dy);
            const float mv = UNIT ? __fdividef(a.z, 1.0f + q) : a.z * expf(-beta * log1pf(q));
            kahan_acc(sum, comp, mv);
            if (mv >= best) {                              // ties to the smaller label (rare)
                const int lj = sb[t];
                if (mv > best || lj < bj) { best = mv; bj = lj; }
            }
        }
    }
    if (r < n) ws.part[(size_t)blockIdx.y * ws.P + r] = CleanPart{sum, -comp, best, bj};
}

// per rank: the chunks' partials in chunk order, the decision and the target
__global__ void __launch_bounds__(CL_T) k_clean_decide(const int32_t* n_dev, int32_t max_obj, CleanWs ws) {
    const int n = clean_n(n_dev, max_obj);
    for (int r = blockIdx.x * CL_T + threadIdx.x; r < n; r += gridDim.x * CL_T) {
        const unsigned long long key = ws.skey[r];
        if (key == ~0ull) continue;
        const int li = (int)(uint32_t)key;
        float hi = 0.f, lo = 0.f, best = -1.f;
        int bj = -1;
        for (int c = 0; c * CL_JC < r; c++) {
            const CleanPart p = ws.part[(size_t)c * ws.P + r];
            two_sum_acc(hi, lo, p.s_hi);
            lo += p.s_lo;
            if (p.bj > 0 && (p.best > best || (p.best == best && p.bj < bj))) { best = p.best; bj = p.bj; }
        }
        const float sum = hi + lo;
        const float4 g = ws.geo[li];
        ws.into[li] = (bj > 0 && g.z - sum < ws.ell[li].w) ? bj : li;
    }
}

__global__ void __launch_bounds__(CL_T) k_clean_into_init(const int32_t* n_dev, int32_t max_obj, CleanWs ws) {
    const int n = clean_n(n_dev, max_obj);
    for (int l = blockIdx.x * CL_T + threadIdx.x; l <= n; l += gridDim.x * CL_T) ws.into[l] = l;
}

// merge targets followed to a kept object (each target is strictly brighter, so
// a chain has at most n steps): num[i] = that object
__global__ void __launch_bounds__(CL_T) k_clean_root(const int32_t* n_dev, int32_t max_obj, CleanWs ws) {
    const int n = clean_n(n_dev, max_obj);
    for (int i = blockIdx.x * CL_T + threadIdx.x + 1; i <= n; i += gridDim.x * CL_T) {
        int r = i;
        for (int s = 0; s <= n && ws.into[r] != r; s++) r = ws.into[r];
        ws.num[i] = r;
    }
}

// kept objects (their own root, holding pixels) per tile of 1024 labels
__global__ void __launch_bounds__(1024) k_clean_count(const int32_t* n_dev, int32_t max_obj, CleanWs ws) {
    const int n = clean_n(n_dev, max_obj);
    const int i = blockIdx.x * 1024 + threadIdx.x + 1;
    const int kept = (i <= n && ws.num[i] == i && ws.geo[i].w > 0.f) ? 1 : 0;
    const int c = __syncthreads_count(kept);
    if (threadIdx.x == 0) ws.tcount[blockIdx.x] = c;
}

// new numbers 1.. in label order: a tile's offset is the sum of the counts
// before it; a block scan inside.  The number of a kept object replaces its
// (self) target in into[]; the count goes to n_out.
__global__ void __launch_bounds__(1024) k_clean_assign(const int32_t* n_dev, int32_t max_obj, CleanWs ws,
                                                       int32_t* n_out) {
    __shared__ int red[32];
    const int n = clean_n(n_dev, max_obj);
    const int tile = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (tile * 1024 >= max(n, 1)) return;
    int off = 0;
    for (int t = threadIdx.x; t < tile; t += 1024) off += ws.tcount[t];
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if (lane == 0) red[warp] = off;
    __syncthreads();
    off = 0;
    for (int w = 0; w < 32; w++) off += red[w];
    __syncthreads();
    const int i = tile * 1024 + threadIdx.x + 1;
    const int kept = (i <= n && ws.num[i] == i && ws.geo[i].w > 0.f) ? 1 : 0;
    int inc = kept;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) red[warp] = inc;
    __syncthreads();
    int before = off;
    for (int w = 0; w < warp; w++) before += red[w];
    if (kept) ws.into[i] = before + inc;
    // the tile holding label n (or tile 0 when there is none) reports the count
    if (threadIdx.x == 1023 && tile == (n > 0 ? (n - 1) / 1024 : 0)) *n_out = before + inc;
}

__global__ void __launch_bounds__(CL_T) k_clean_relabel(const int32_t* labels, int64_t npx, const int32_t* n_dev,
                                                        int32_t max_obj, CleanWs ws, int32_t* out) {
    const int n = clean_n(n_dev, max_obj);
    for (int64_t p = (int64_t)blockIdx.x * CL_T + threadIdx.x; p < npx; p += (int64_t)gridDim.x * CL_T) {
        const int l = __ldg(labels + p);
        out[p] = (l <= 0 || l > n) ? 0 : ws.into[ws.num[l]];   // the number of the object's kept root
    }
}

}  // namespace ipp

using namespace ipp;

static size_t a256c(size_t x) { return (x + 255) & ~(size_t)255; }

static int clean_sort_size(int32_t max_obj) {
    int P = BS_N;
    while (P < max_obj) P <<= 1;
    return P;
}

static size_t ipp_clean_ws_carve(int32_t max_obj, void* base, CleanWs* w) {
    const size_t n = (size_t)max_obj + 1;
    const int P = clean_sort_size(max_obj);
    const size_t nchunk = ((size_t)P + CL_JC - 1) / CL_JC;
    const size_t sz[] = {n * 8, n * 16, n * 16, n * 16, n * 24, n * 48, n * 16, n * 8, n * 16, n * 4, n * 4,
                         (size_t)P * 8, nchunk * P * sizeof(CleanPart), (n / 1024 + 1) * 4};
    constexpr int NA = sizeof(sz) / sizeof(sz[0]);
    size_t off[NA], o = 0;
    for (int k = 0; k < NA; k++) { off[k] = o; o += a256c(sz[k]); }
    if (base && w) {
        unsigned char* b = static_cast<unsigned char*>(base);
        w->pkey = (unsigned long long*)(b + off[0]);
        w->sw = (long long*)(b + off[1]);
        w->swx = (long long*)(b + off[2]);
        w->swy = (long long*)(b + off[3]);
        w->cnt = (long long*)(b + off[4]);
        w->mom = (long long*)(b + off[5]);
        w->geo = (float4*)(b + off[6]);
        w->blo = (float2*)(b + off[7]);
        w->ell = (float4*)(b + off[8]);
        w->into = (int32_t*)(b + off[9]);
        w->num = (int32_t*)(b + off[10]);
        w->skey = (unsigned long long*)(b + off[11]);
        w->part = (CleanPart*)(b + off[12]);
        w->tcount = (int32_t*)(b + off[13]);
        w->P = P;
    }
    return o;
}

size_t ipp_clean_ws_bytes(int32_t max_obj) { return ipp_clean_ws_carve(max_obj, nullptr, nullptr); }

int ipp_launch_clean(const float* sub, int64_t pitch, const int32_t* labels, int64_t W, int64_t H,
                     const int32_t* n_dev, int32_t max_obj, const float* thr_map, const float* mesh_rms, int nx,
                     int ny, float mesh_w, float mesh_h, float k, float thresh_abs, float beta, int32_t* out,
                     int32_t* n_out, void* ws, cudaStream_t s) {
    CleanWs w;
    ipp_clean_ws_carve(max_obj, ws, &w);
    // the accumulators start at zero (peak keys, sums, counts, moments)
    const size_t acc = (size_t)((unsigned char*)w.geo - (unsigned char*)ws);
    if (cudaMemsetAsync(ws, 0, acc, s) != cudaSuccess) return ipp_check_launch("clean memset");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t npx = W * H;
    const unsigned pg = (unsigned)std::min<int64_t>((npx + CL_T - 1) / CL_T, (int64_t)std::max(sms, 1) * 16);
    const unsigned og = (unsigned)std::max<int64_t>(1, ((int64_t)max_obj + CL_T) / CL_T);
    const float a2 = (float)(2.0 * std::log(2.0) / (std::pow(2.0, 1.0 / beta) - 1.0));
    k_clean_pix_a<<<pg, CL_T, 0, s>>>(sub, pitch, labels, W, H, n_dev, max_obj, w);
    if (int e = ipp_check_launch("k_clean_pix_a")) return e;
    k_clean_obj_a<<<og, CL_T, 0, s>>>(n_dev, max_obj, w);
    if (int e = ipp_check_launch("k_clean_obj_a")) return e;
    k_clean_pix_b<<<pg, CL_T, 0, s>>>(sub, pitch, labels, W, H, n_dev, max_obj, w);
    if (int e = ipp_check_launch("k_clean_pix_b")) return e;
    const CleanThr T{thr_map, mesh_rms, nx, ny, mesh_w, mesh_h, k, thresh_abs, W};
    k_clean_obj_b<<<og, CL_T, 0, s>>>(n_dev, max_obj, w, T, 1.0f / a2);
    if (int e = ipp_check_launch("k_clean_obj_b")) return e;
    k_clean_into_init<<<og, CL_T, 0, s>>>(n_dev, max_obj, w);
    if (int e = ipp_check_launch("k_clean_into_init")) return e;
    // brightness order: keys, 2048-key blocks sorted in shared memory, then the
    // merges of 4096 keys and more
    const int P = w.P;
    k_clean_keys<<<(unsigned)(P / CL_T), CL_T, 0, s>>>(n_dev, max_obj, w, P);
    if (int e = ipp_check_launch("k_clean_keys")) return e;
    k_bitonic_local<<<(unsigned)(P / BS_N), BS_T, 0, s>>>(w.skey, 2, BS_N);
    if (int e = ipp_check_launch("k_bitonic_local")) return e;
    for (int kk = 2 * BS_N; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j >= BS_N; j >>= 1) {
            k_bitonic_global<<<(unsigned)(P / 2 / CL_T), CL_T, 0, s>>>(w.skey, P, kk, j);
            if (int e = ipp_check_launch("k_bitonic_global")) return e;
        }
        k_bitonic_local<<<(unsigned)(P / BS_N), BS_T, 0, s>>>(w.skey, kk, kk);
        if (int e = ipp_check_launch("k_bitonic_local")) return e;
    }
    const int nchunk = (P + CL_JC - 1) / CL_JC;
    const dim3 pg2((unsigned)(P / CL_T), (unsigned)nchunk);
    if (beta == 1.0f) k_clean_pairs<true><<<pg2, CL_T, 0, s>>>(n_dev, max_obj, w, W, beta);
    else k_clean_pairs<false><<<pg2, CL_T, 0, s>>>(n_dev, max_obj, w, W, beta);
    if (int e = ipp_check_launch("k_clean_pairs")) return e;
    k_clean_decide<<<og, CL_T, 0, s>>>(n_dev, max_obj, w);
    if (int e = ipp_check_launch("k_clean_decide")) return e;
    k_clean_root<<<og, CL_T, 0, s>>>(n_dev, max_obj, w);
    if (int e = ipp_check_launch("k_clean_root")) return e;
    const unsigned ntile = (unsigned)(max_obj / 1024 + 1);
    k_clean_count<<<ntile, 1024, 0, s>>>(n_dev, max_obj, w);
    if (int e = ipp_check_launch("k_clean_count")) return e;
    k_clean_assign<<<ntile, 1024, 0, s>>>(n_dev, max_obj, w, n_out);
    if (int e = ipp_check_launch("k_clean_assign")) return e;
    k_clean_relabel<<<pg, CL_T, 0, s>>>(labels, npx, n_dev, max_obj, w, out);
    return ipp_check_launch("k_clean_relabel");
}
