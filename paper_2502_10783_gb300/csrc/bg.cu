// bg.cu -- mesh background (Sec. 2.2.2, Eqs. 1-4): per-mesh iterative sigma
// clip, invalid-mesh fill and mesh median filter, interpolation + subtraction.
//
// k_mesh_stats: one 128-thread CTA per mesh with ~31 KB of shared memory, so
// seven meshes run on each SM and a 4096^2 frame of 128 px meshes is a single
// wave.  The mesh is not held on chip.  Warp 0 first sorts a 256-value sample
// to place a histogram window (bins of ~1/64-1/128 robust sigma, outliers in
// two end bins).  Read 1 (HBM, float4) builds the histogram and the exact sums
// of the whole set relative to the window centre -- in-window values as int64
// fixed point (a power-of-two scale no coarser than their own spacing), the
// few outside the window in double-float.  A window that missed or is too
// coarse is re-placed with one more read.  The last read (L2) keeps, bin-sorted
// in shared memory, only the values a clip pass can touch: the tails beyond ~2
// robust sigma, where the bounds fall, and a band of bins around the median
// (sorted in parallel before the passes start).  A pass then touches only the
// values it removes and the median bins, so it costs O(removed + median bin),
// and its statistics are formed in double-float on one lane (the FP64 pipe of
// this GPU is narrow).  A pass that needs a bin that was not stored (bounds
// inside the core, a median outside the band) reads the mesh again for that
// pass: same result, more traffic.
#include <math.h>

#include "jobs.cuh"

namespace ipp {

constexpr int MS_THREADS = 128;
constexpr int MS_WARPS = MS_THREADS / kWarp;
constexpr int MS_NB = 1024;          // window bins 1..MS_NB; 0 = below, MS_NB+1 = above
constexpr int MS_NBT = MS_NB + 2;
constexpr int MS_SCALE_BITS = 14;    // fixed point: d_int = (v - c*) * 2^(14 - e), bw = 2^e
constexpr int MS_STORE = 2880;       // stored values: tails + median band
constexpr int MS_GCAP = 512;         // gathered values of unstored median bins
constexpr int MS_BAND = 8;           // median band half-width in bins (at most)
constexpr int MS_CHUNK = 8;          // loads in flight per thread
constexpr int MS_WARPSORT_MAX = 256;
constexpr int MS_WARP_SCAN = 192;   // removal ranges up to this length are scanned by warp 0 alone

// slots of MeshShared::bc_i
enum { BI_STATE = 0, BI_MODE, BI_KBL, BI_KBH, BI_GL, BI_GH, BI_GCNT, BI_NEED, BI_RB0, BI_RR0, BI_RB1, BI_RR1,
       BI_DIGIT, BI_REM, BI_N0, BI_REFINE, BI_E, BI_CL, BI_ML, BI_MH, BI_CH, BI_SBAD, BI_COUNT };
enum { ST_STOP = 0, ST_SCAN = 1, ST_GATHER = 2, ST_RADIX = 3 };

struct MeshShared {
    uint32_t hbuf[2 * MS_NBT];      // counts | scatter cursors; radix histogram after the scatter
    uint32_t hstart[MS_NBT + 1];    // exclusive prefix of the counts
    uint32_t sstart[MS_NBT + 1];    // exclusive prefix of the stored counts
    uint32_t sorted_bits[(MS_NBT + 31) / 32];  // stored bins whose slice is already sorted
    float store[MS_STORE];
    float gbuf[MS_GCAP];
    long long redl[MS_WARPS * 2];
    float4 redo[MS_WARPS];
    int redi[MS_WARPS * 3];
    float redf[MS_WARPS * 3];
    long long ks_i[2];   // running sums of the kept set (clip loop, warp 0 lane 0)
    df ks_o[2];
    df st[3];            // median, mean, sigma of the kept set
    float bc_f[8];
    int bc_i[BI_COUNT];
};

// Bin of a value: monotone in v (FP subtraction and the power-of-two scaling
// are monotone), clamped to [0, MS_NB+1].
__device__ __forceinline__ int bin_of(float v, float cstar, float inv_bw) {
    float t = floorf((v - cstar) * inv_bw);
    t = fmaxf(fminf(t, (float)(MS_NB / 2)), (float)(-MS_NB / 2 - 1));
    return (int)t + MS_NB / 2 + 1;
}

// Where a mesh lives and how its values are formed (calibrated when raw u16).
struct MeshGeom {
    const void* img;
    int dtype;
    int64_t pitch, W;
    const uint8_t* mask;
    const float* bias_map;
    float bias;
    const float* inv_flat;
    int64_t x0, y0;
    int mw, we, he, slots;
    bool vec;  // f32, unmasked, 16-byte aligned rows, we % 4 == 0: float4 reads
};

// Value of mesh pixel (r, c) (inside the mesh's frame region); false when the
// pixel is masked or not finite.
__device__ __forceinline__ bool mesh_value_at(const MeshGeom& G, int r, int c, float* out) {
    const int64_t yy = G.y0 + r, xx = G.x0 + c;
    float x;
    if (G.dtype == IPP_F32) {
        x = __ldg(reinterpret_cast<const float*>(G.img) + yy * G.pitch + xx);
    } else {
        const float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(G.img) + yy * G.pitch + xx);
        const float b = G.bias_map ? __ldg(G.bias_map + yy * G.W + xx) : G.bias;
        x = (raw - b) * __ldg(G.inv_flat + yy * G.W + xx);
    }
    *out = x;
    return !(G.mask && G.mask[yy * G.W + xx]) && isfinite(x);
}

// Calls f(v) for every usable value of the mesh that this thread owns.  Vector
// path: float4 quads of the mesh's frame region, quad e4 = threadIdx.x + k *
// MS_THREADS; scalar path: element e = threadIdx.x + k * MS_THREADS of the
// mw x mh slots (row e / mw, column e % mw).  A chunk of loads is issued before
// any is used: addresses are clamped into the mesh and slots beyond it are
// skipped afterwards.  Every call forms the values with the same arithmetic, so
// re-reads see identical values.
template <int T = MS_THREADS, class F>
__device__ __forceinline__ void mesh_for_each(const MeshGeom& G, F&& f) {
    if (G.vec) {
        constexpr int VCH = 4;
        const int qpr = G.we >> 2, nq = G.he * qpr;
        const float4* base = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(G.img) + G.y0 * G.pitch +
                                                             G.x0);
        const int64_t p4 = G.pitch >> 2;
        const int dr = T / qpr, dc = T - dr * qpr;
        int r = threadIdx.x / qpr, c = threadIdx.x - r * qpr;
        for (int e0 = threadIdx.x; e0 < nq; e0 += VCH * T) {
            float4 q[VCH];
#pragma unroll
            for (int j = 0; j < VCH; j++) {
                q[j] = __ldg(base + (int64_t)min(r, G.he - 1) * p4 + c);
                r += dr;
                c += dc;
                if (c >= qpr) { c -= qpr; r++; }
            }
#pragma unroll
            for (int j = 0; j < VCH; j++) {
                if (e0 + j * T >= nq) continue;
                if (isfinite(q[j].x)) f(q[j].x);
                if (isfinite(q[j].y)) f(q[j].y);
                if (isfinite(q[j].z)) f(q[j].z);
                if (isfinite(q[j].w)) f(q[j].w);
            }
        }
        return;
    }
    const int dr = T / G.mw, dc = T - dr * G.mw;
    int r = threadIdx.x / G.mw, c = threadIdx.x - r * G.mw;
    for (int e0 = threadIdx.x; e0 < G.slots; e0 += MS_CHUNK * T) {
        float v[MS_CHUNK];
        bool ok[MS_CHUNK];
#pragma unroll
        for (int j = 0; j < MS_CHUNK; j++) {
            const bool in = e0 + j * T < G.slots && r < G.he && c < G.we;
            ok[j] = mesh_value_at(G, min(r, G.he - 1), min(c, G.we - 1), &v[j]) && in;
            r += dr;
            c += dc;
            if (c >= G.mw) { c -= G.mw; r++; }
        }
#pragma unroll
        for (int j = 0; j < MS_CHUNK; j++)
            if (ok[j]) f(v[j]);
    }
}

// Sums of a set of values relative to c*: in-window values in int64 fixed
// point (scale 2^-fx, exact for values no finer than that), the values of the two
// end bins (outliers) in double-float (pairs of FP32, ~48-bit mantissa) so that
// no FP64 instruction is needed per element.
struct Sums {
    long long i1, i2;
    df o1, o2;
};

__device__ __forceinline__ void sums_add(Sums& a, float v, int b, float cstar, float fxs) {
    if (b >= 1 && b <= MS_NB) {
        const int d = __float2int_rn((v - cstar) * fxs);
        a.i1 += d;
        a.i2 += (long long)d * d;
    } else {
        const df d = two_sum(v, -cstar);
        df q = sq_exact(d.hi);
        q = df_add_f(q, __fmul_rn(2.0f * d.hi, d.lo));
        a.o1 = df_add(a.o1, d);
        a.o2 = df_add(a.o2, q);
    }
}

// Read-1 accumulation of one value: its bin's count, and the sums of sums_add
// with the in-window part in per-thread registers (a1: at most 128 values of
// |d| <= 2^23 per thread, so int32 holds it).  The same bins and fixed-point
// values as bin_of and sums_add.
__device__ __forceinline__ void hist_acc(uint32_t* hist, float x, float cstar, float inv_bw, int& a1, long long& a2,
                                         Sums& o) {
    const float t = (x - cstar) * inv_bw;
    const int f = min(max(__float2int_rd(t), -MS_NB / 2 - 1), MS_NB / 2);
    atomicAdd(&hist[f + MS_NB / 2 + 1], 1u);
    if (f >= -MS_NB / 2 && f < MS_NB / 2) {
        const int d = __float2int_rn(t * (float)(1 << MS_SCALE_BITS));
        a1 += d;
        a2 += (long long)d * d;
    } else {
        const df dd = two_sum(x, -cstar);
        df q = sq_exact(dd.hi);
        q = df_add_f(q, __fmul_rn(2.0f * dd.hi, dd.lo));
        o.o1 = df_add(o.o1, dd);
        o.o2 = df_add(o.o2, q);
    }
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-warp partial of (Sums, three counts) into shared slot `warp`; warps with
// nothing to add (the common case in late clip passes) skip the shuffles.
__device__ __forceinline__ void warp_partial(MeshShared& S, const Sums& s, const int c[3], int lane, int warp) {
    const bool anyi = __any_sync(0xffffffffu, s.i1 != 0 || s.i2 != 0);
    const bool anyo = __any_sync(0xffffffffu, s.o1.hi != 0.f || s.o2.hi != 0.f);
    const long long a = anyi ? warp_sum_ll(s.i1) : 0, b = anyi ? warp_sum_ll(s.i2) : 0;
    const df x = anyo ? warp_sum_df(s.o1) : df{0.f, 0.f};
    const df y = anyo ? warp_sum_df(s.o2) : df{0.f, 0.f};
    const bool anyc = __any_sync(0xffffffffu, (c[0] | c[1] | c[2]) != 0);
    const int c0 = anyc ? warp_sum_i(c[0]) : 0, c1 = anyc ? warp_sum_i(c[1]) : 0, c2 = anyc ? warp_sum_i(c[2]) : 0;
    if (lane == 0) {
        S.redl[warp] = a; S.redl[MS_WARPS + warp] = b;
        S.redo[warp] = make_float4(x.hi, x.lo, y.hi, y.lo);
        S.redi[warp] = c0; S.redi[MS_WARPS + warp] = c1; S.redi[2 * MS_WARPS + warp] = c2;
    }
}

// Warp 0 only, after a barrier: totals of the per-warp partials (lanes
// 0..MS_WARPS-1 hold one each; lane 0 ends with the totals).  Counts are
// broadcast to every lane; the sums (int64, outlier sums as double-float) are
// valid in lane 0.
__device__ __forceinline__ void warp0_totals(const MeshShared& S, int lane, int c[3], long long* i1, long long* i2,
                                             df* o1, df* o2) {
    const bool in = lane < MS_WARPS;
    long long a = in ? S.redl[lane] : 0, b = in ? S.redl[MS_WARPS + lane] : 0;
    const float4 o = in ? S.redo[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    df x{o.x, o.y}, y{o.z, o.w};
    int c0 = in ? S.redi[lane] : 0, c1 = in ? S.redi[MS_WARPS + lane] : 0, c2 = in ? S.redi[2 * MS_WARPS + lane] : 0;
#pragma unroll
    for (int off = MS_WARPS / 2; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
        x = df_add(x, df{__shfl_xor_sync(0xffffffffu, x.hi, off), __shfl_xor_sync(0xffffffffu, x.lo, off)});
        y = df_add(y, df{__shfl_xor_sync(0xffffffffu, y.hi, off), __shfl_xor_sync(0xffffffffu, y.lo, off)});
        c0 += __shfl_xor_sync(0xffffffffu, c0, off);
        c1 += __shfl_xor_sync(0xffffffffu, c1, off);
        c2 += __shfl_xor_sync(0xffffffffu, c2, off);
    }
    c[0] = __shfl_sync(0xffffffffu, c0, 0);
    c[1] = __shfl_sync(0xffffffffu, c1, 0);
    c[2] = __shfl_sync(0xffffffffu, c2, 0);
    *i1 = a;
    *i2 = b;
    *o1 = x;
    *o2 = y;
}

// Bitonic sort of 32*E values held E per lane (value index E*lane + j),
// ascending, within one warp.  Padding slots hold +inf.
template <int E>
__device__ __forceinline__ void warp_bitonic(float a[E], int lane) {
    constexpr int N = 32 * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            if (jj >= E) {  // partner in another lane, same slot
                const int lm = jj / E;
#pragma unroll
                for (int j = 0; j < E; j++) {
                    const int i = E * lane + j;
                    const float b = __shfl_xor_sync(0xffffffffu, a[j], lm);
                    const bool lower = (i & jj) == 0, asc = (i & k) == 0;
                    a[j] = (lower == asc) ? fminf(a[j], b) : fmaxf(a[j], b);
                }
            } else {        // partner in this lane
#pragma unroll
                for (int j = 0; j < E; j++) {
                    if (j & jj) continue;
                    const int i = E * lane + j;
                    const bool asc = (i & k) == 0;
                    const float x = a[j], y = a[j + jj];
                    a[j] = asc ? fminf(x, y) : fmaxf(x, y);
                    a[j + jj] = asc ? fmaxf(x, y) : fminf(x, y);
                }
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void warp_sort_slice(float* sval, int s0, int m, int lane) {
    float a[E];
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int i = E * lane + j;
        a[j] = i < m ? sval[s0 + i] : INFINITY;
    }
    warp_bitonic<E>(a, lane);
#pragma unroll
    for (int j = 0; j < E; j++) {
        const int i = E * lane + j;
        if (i < m) sval[s0 + i] = a[j];
    }
    __syncwarp();
}

// Warp 0 only: sort stored bin b's slice in place once (slices up to 256 values).
__device__ void warp_ensure_sorted(MeshShared& S, int b, int lane) {
    if ((S.sorted_bits[b >> 5] >> (b & 31)) & 1u) return;
    const int s0 = S.sstart[b], m = (int)S.sstart[b + 1] - s0;
    if (m <= 32) warp_sort_slice<1>(S.store, s0, m, lane);
    else if (m <= 64) warp_sort_slice<2>(S.store, s0, m, lane);
    else if (m <= 128) warp_sort_slice<4>(S.store, s0, m, lane);
    else warp_sort_slice<8>(S.store, s0, m, lane);
    if (lane == 0) atomicOr(&S.sorted_bits[b >> 5], 1u << (b & 31));
    __syncwarp();
}

// Warp 0 only: r-th smallest of the values of buf[s0, s1) that lie in [lo, hi]
// and, when bsel >= 0, fall in bin bsel: 11/11/10-bit radix passes over the
// order-preserving keys, histogram in S.hbuf (free after the scatter).
__device__ float warp_radix_select(MeshShared& S, const float* buf, int s0, int s1, float lo, float hi, int bsel,
                                   float cstar, float inv_bw, int r, int lane) {
    uint32_t prefix = 0, pmask = 0;
    int rr = r;
    for (int pass = 0; pass < 3; pass++) {
        const int sh = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
        const int nb = pass == 2 ? 1024 : 2048, per = nb / 32;
        for (int k = lane; k < nb; k += 32) S.hbuf[k] = 0;
        __syncwarp();
        for (int k = s0 + lane; k < s1; k += 32) {
            const float v = buf[k];
            if (!(v >= lo && v <= hi)) continue;
            if (bsel >= 0 && bin_of(v, cstar, inv_bw) != bsel) continue;
            const uint32_t key = fkey(v);
            if ((key & pmask) != prefix) continue;
            atomicAdd(&S.hbuf[(key >> sh) & (nb - 1)], 1u);
        }
        __syncwarp();
        int tot = 0;
        for (int d = lane * per; d < (lane + 1) * per; d++) tot += (int)S.hbuf[d];
        int inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        const int before = inc - tot;
        int dsel = 0, rem = 0;
        if (rr >= before && rr < inc) {
            int acc = before, d = lane * per;
            for (; d < (lane + 1) * per; d++) {
                const int c = (int)S.hbuf[d];
                if (rr < acc + c) break;
                acc += c;
            }
            dsel = d;
            rem = rr - acc;
        }
        const unsigned who = __ballot_sync(0xffffffffu, rr >= before && rr < inc);
        const int src = who ? __ffs(who) - 1 : 0;
        dsel = __shfl_sync(0xffffffffu, dsel, src);
        rem = __shfl_sync(0xffffffffu, rem, src);
        prefix |= (uint32_t)dsel << sh;
        pmask |= (uint32_t)(nb - 1) << sh;
        rr = rem;
        __syncwarp();
    }
    return fkey_inv(prefix);
}

// Block-wide: the same selection over the values of the mesh itself (global
// re-reads), for a median bin holding more values than the gather buffer.
__device__ float block_radix_select_global(MeshShared& S, const MeshGeom& G, float lo, float hi, int bsel,
                                           float cstar, float inv_bw, int r) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t prefix = 0, pmask = 0;
    int rr = r;
    for (int pass = 0; pass < 3; pass++) {
        const int sh = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
        const int nb = pass == 2 ? 1024 : 2048, per = nb / 32;
        for (int k = threadIdx.x; k < nb; k += MS_THREADS) S.hbuf[k] = 0;
        __syncthreads();
        mesh_for_each(G, [&](float v) {
            if (!(v >= lo && v <= hi) || bin_of(v, cstar, inv_bw) != bsel) return;
            const uint32_t key = fkey(v);
            if ((key & pmask) == prefix) atomicAdd(&S.hbuf[(key >> sh) & (nb - 1)], 1u);
        });
        __syncthreads();
        if (warp == 0) {
            int tot = 0;
            for (int d = lane * per; d < (lane + 1) * per; d++) tot += (int)S.hbuf[d];
            int inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            const int before = inc - tot;
            if (rr >= before && rr < inc) {
                int acc = before, d = lane * per;
                for (; d < (lane + 1) * per; d++) {
                    const int c = (int)S.hbuf[d];
                    if (rr < acc + c) break;
                    acc += c;
                }
                S.bc_i[BI_DIGIT] = d;
                S.bc_i[BI_REM] = rr - acc;
            }
        }
        __syncthreads();
        prefix |= (uint32_t)S.bc_i[BI_DIGIT] << sh;
        pmask |= (uint32_t)(nb - 1) << sh;
        rr = S.bc_i[BI_REM];
        __syncthreads();
    }
    return fkey_inv(prefix);
}

// State of the kept set [lo, hi] of a clip pass.
struct KeptSet {
    float lo, hi;
    int bl, bh;     // bins of lo and hi
    int nbl, nbh;   // kept elements in bins bl and bh (nbh unused when bl == bh)
    int n;
};

// Warp 0 only: bin and rank (among the kept values of that bin) of the k-th
// smallest kept value.  The bin search probes 32 bins per step (ballot), so
// it takes two or three steps over the 1026 bins.
__device__ __forceinline__ void kept_locate(const MeshShared& S, const KeptSet& K, int k, int lane, int* bin, int* r) {
    const int full = (K.bh > K.bl + 1) ? (int)(S.hstart[K.bh] - S.hstart[K.bl + 1]) : 0;
    const int nbl = (K.bl == K.bh) ? K.n : K.nbl;
    if (k < nbl) {
        *bin = K.bl; *r = k;
    } else if (k - nbl < full) {
        const int kk = k - nbl;
        const uint32_t base = S.hstart[K.bl + 1];
        // largest a in [K.bl + 1, K.bh) with hstart[a] - base <= kk (true at K.bl + 1)
        int a = K.bl + 1, e = K.bh;
        while (e - a > 1) {
            const int step = (e - a + 31) >> 5;
            const int p = a + lane * step;
            const unsigned m = __ballot_sync(0xffffffffu, p < e && (int)(S.hstart[p] - base) <= kk);
            const int na = a + (31 - __clz(m)) * step;
            e = min(na + step, e);
            a = na;
        }
        *bin = a; *r = kk - (int)(S.hstart[a] - base);
    } else {
        *bin = K.bh; *r = k - nbl - full;
    }
}

// Which bins the scatter stored: [0, cl], [ml, mh] and [ch, MS_NB+1].
struct Stored {
    int cl, ml, mh, ch;
    __device__ __forceinline__ bool bin(int b) const { return b <= cl || b >= ch || (b >= ml && b <= mh); }
    __device__ __forceinline__ bool range(int a, int b) const {  // every bin of [a, b]; empty ranges are
        return a > b || b <= cl || a >= ch || (a >= ml && b <= mh);
    }
};

// ---- scalar statistics of the kept set (one thread) --------------------------
// Double-float arithmetic on the FP32 pipe (~48-bit significands, relative
// error ~1e-14): the FP64 pipe of this GPU is narrow and its latency sits on
// the serial path of every clip pass.  Windows so fine or so coarse that the
// scaled sums would leave the FP32 range (|e| > 40) take the FP64 branch.
__device__ __forceinline__ df df_from_d(double d) {
    const float h = __double2float_rn(d);
    return df{h, __double2float_rn(d - (double)h)};
}
// smallest float >= hi + lo, largest float <= hi + lo (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ float df_to_float_ru(df a) { return a.lo > 0.f ? nextafterf(a.hi, INFINITY) : a.hi; }
__device__ __forceinline__ float df_to_float_rd(df a) { return a.lo < 0.f ? nextafterf(a.hi, -INFINITY) : a.hi; }

// mean and population sigma of the kept set from its sums relative to c*:
// s1 = i1 * unit + o1, s2 = i2 * unit^2 + o2, unit = 2^(e - MS_SCALE_BITS)
__device__ __forceinline__ void kept_stats(long long i1, long long i2, df o1, df o2, int n, float cstar, int e,
                                           df* mu, df* sd) {
    if (e >= -40 && e <= 40) {
        const float u = ldexpf(1.0f, e - MS_SCALE_BITS);
        const df s1 = df_add(df_scale(df_from_i64(i1), u), o1);
        const df s2 = df_add(df_scale(df_scale(df_from_i64(i2), u), u), o2);
        const df rn = df_div(df{1.0f, 0.0f}, df{(float)n, 0.0f});
        const df m1 = df_mul(s1, rn);
        *mu = df_add_f(m1, cstar);
        *sd = df_sqrt(df_sub(df_mul(s2, rn), df_mul(m1, m1)));
    } else {
        const double unit = ldexp(1.0, e - MS_SCALE_BITS);
        const double s1 = (double)i1 * unit + df_to_d(o1);
        const double s2 = (double)i2 * unit * unit + df_to_d(o2);
        const double m1 = s1 / n;
        *mu = df_from_d((double)cstar + m1);
        *sd = df_from_d(sqrt(fmax(s2 / n - m1 * m1, 0.0)));
    }
}

// Warp 0 only: exclusive prefix of the histogram counts into S.hstart, and the
// bins holding the order statistics kq[0..2] (broadcast to every lane).
__device__ __forceinline__ void warp_scan_counts(const uint32_t* counts, uint32_t* hstart, int lane, const int kq[3],
                                                 int bq[3]) {
    constexpr int PER = (MS_NBT + 31) / 32;
    const int b0 = lane * PER, b1 = min(b0 + PER, MS_NBT);
    int acc = 0;
    for (int b = b0; b < b1; b++) acc += (int)counts[b];
    int inc = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    int run = inc - acc;
    int loc[3] = {0, 0, 0};
    unsigned hit = 0;
    for (int b = b0; b < b1; b++) {
        const int h = (int)counts[b];
        hstart[b] = (uint32_t)run;
#pragma unroll
        for (int t = 0; t < 3; t++)
            if (kq[t] >= run && kq[t] < run + h) { loc[t] = b; hit |= 1u << t; }
        run += h;
    }
    if (lane == 31) hstart[MS_NBT] = (uint32_t)inc;
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const unsigned who = __ballot_sync(0xffffffffu, (hit >> t) & 1u);
        bq[t] = __shfl_sync(0xffffffffu, loc[t], who ? __ffs(who) - 1 : 0);
    }
    __syncwarp();
}

__device__ __forceinline__ void warp0_scan_counts(MeshShared& S, int lane, const int kq[3], int bq[3]) {
    warp_scan_counts(S.hbuf, S.hstart, lane, kq, bq);
}

// Warp 0 only: value of rank r (among kept values) in bin b, when it is on chip:
// a stored slice (sorted once, or radix-selected when long) or the gathered
// bins [gl, gh].  Returns false when neither holds bin b.
__device__ bool warp_value_of(MeshShared& S, const Stored& St, int b, int r, const KeptSet& K, float cstar,
                              float inv_bw, int lane, float* out) {
    if (St.bin(b)) {
        const int s0 = S.sstart[b], s1 = S.sstart[b + 1];
        const bool sorted = (S.sorted_bits[b >> 5] >> (b & 31)) & 1u;
        if (sorted || s1 - s0 <= MS_WARPSORT_MAX) {
            warp_ensure_sorted(S, b, lane);
            int a = s0;
            if (b == K.bl) {  // first value >= lo in the sorted slice (bins inside the kept range are whole)
                int e = s1;
                while (a < e) { const int m = (a + e) >> 1; if (S.store[m] < K.lo) a = m + 1; else e = m; }
            }
            *out = S.store[min(a + r, s1 - 1)];
        } else {
            *out = warp_radix_select(S, S.store, s0, s1, K.lo, K.hi, -1, cstar, inv_bw, r, lane);
        }
        return true;
    }
    if (b >= S.bc_i[BI_GL] && b <= S.bc_i[BI_GH]) {
        *out = warp_radix_select(S, S.gbuf, 0, min(S.bc_i[BI_GCNT], MS_GCAP), K.lo, K.hi, b, cstar, inv_bw, r,
                                 lane);
        return true;
    }
    return false;
}

// Warp 0 only: statistics of the current kept set from its two middle order
// statistics, and the bounds of the next pass (published for every warp).
// Returns the next state: ST_SCAN, or ST_STOP after the last allowed pass.
__device__ int warp0_finish(MeshShared& S, const MeshJob& J, const Stored& St, const KeptSet& K, float mid0,
                            float mid1, int it, float cstar, int e, float inv_bw, df nsig, int lane, float* plo,
                            float* phi) {
    if (lane == 0) {
        df mu, sd;
        kept_stats(S.ks_i[0], S.ks_i[1], S.ks_o[0], S.ks_o[1], K.n, cstar, e, &mu, &sd);
        const df m2 = two_sum(mid0, mid1);
        S.st[0] = df{0.5f * m2.hi, 0.5f * m2.lo};
        S.st[1] = mu;
        S.st[2] = sd;
    }
    if (it == J.maxiters) return ST_STOP;  // statistics of the set left after maxiters passes
    if (lane == 0) {
        const df ks = df_mul(nsig, S.st[2]);
        *plo = fmaxf(K.lo, df_to_float_ru(df_sub(S.st[0], ks)));
        *phi = fminf(K.hi, df_to_float_rd(df_add(S.st[0], ks)));
    }
    *plo = __shfl_sync(0xffffffffu, *plo, 0);
    *phi = __shfl_sync(0xffffffffu, *phi, 0);
    const int nbl = bin_of(*plo, cstar, inv_bw), nbh = bin_of(*phi, cstar, inv_bw);
    const bool on_chip = St.range(K.bl, nbl) && St.range(max(nbh, nbl + 1), K.bh);
    if (lane == 0) {
        S.bc_f[0] = *plo; S.bc_f[1] = *phi; S.bc_f[2] = K.lo; S.bc_f[3] = K.hi;
        S.bc_i[BI_KBL] = K.bl; S.bc_i[BI_KBH] = K.bh;
        S.bc_i[BI_MODE] = on_chip;
    }
    return ST_SCAN;
}

__device__ __forceinline__ void mesh_stats_body(const MeshJob& J, const int mesh) {
    __shared__ MeshShared S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const int mx = mesh % J.nx, my = mesh / J.nx;
    MeshGeom G;
    G.img = J.img; G.dtype = J.dtype; G.pitch = J.pitch; G.W = J.W; G.mask = J.mask;
    G.bias_map = J.bias_map; G.bias = J.bias; G.inv_flat = J.inv_flat;
    G.x0 = (int64_t)mx * J.mesh_w; G.y0 = (int64_t)my * J.mesh_h;
    G.mw = J.mesh_w;
    G.we = (int)min((int64_t)J.mesh_w, J.W - G.x0);
    G.he = (int)min((int64_t)J.mesh_h, J.H - G.y0);
    G.slots = J.mesh_w * J.mesh_h;
    G.vec = J.dtype == IPP_F32 && !J.mask && (J.pitch & 3) == 0 && (G.we & 3) == 0 &&
            ((reinterpret_cast<uintptr_t>(J.img) + (uintptr_t)((G.y0 * J.pitch + G.x0) * 4)) & 15) == 0;

    // ---- histogram window from a sample: warp 0 sorts 256 values spread over
    // the mesh; bw = 2^e with NB*bw in (8, 16] robust sigma, centre c* a
    // multiple of bw near the sample median.  Values outside the window land in the two
    // end bins, whose slices are handled element by element. ----------------
    if (warp == 0) {
        float a[8];
        int nv = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int k = lane + 32 * j;
            const int r = (int)(((int64_t)k * G.he) >> 8), c = (int)(((int64_t)k * 61 + 7) % G.we);
            float x;
            a[j] = mesh_value_at(G, r, c, &x) ? x : INFINITY;
            nv += a[j] != INFINITY;
        }
        nv = warp_sum_i(nv);
        warp_bitonic<8>(a, lane);
#pragma unroll
        for (int j = 0; j < 8; j++) S.gbuf[8 * lane + j] = a[j];
        __syncwarp();
        if (lane == 0) {
            int e = 0;
            float cs = 0.f;
            if (nv >= 16) {
                const float p16 = S.gbuf[(int)(0.1587f * nv)], p50 = S.gbuf[nv / 2], p84 = S.gbuf[(int)(0.8413f * nv)];
                float span = fmaxf(8.0f * (p84 - p16), (S.gbuf[nv - 1] - S.gbuf[0]) * 1e-6f);
                span = fmaxf(span, fabsf(p50) * 1e-6f + 1e-30f);
                e = max(min((int)floorf(log2f(span / MS_NB)), 100), -110);
                cs = rintf(p50 * ldexpf(1.0f, -e)) * ldexpf(1.0f, e);
            }
            S.bc_i[BI_SBAD] = nv < 16;  // too few usable samples: the window is re-placed after read 1
            S.bc_i[BI_E] = e;
            S.bc_f[4] = cs;
        }
    }
    for (int k = threadIdx.x; k < MS_NBT; k += MS_THREADS) S.hbuf[k] = 0;
    __syncthreads();
    int e = S.bc_i[BI_E];
    float cstar = S.bc_f[4], bw = ldexpf(1.0f, e), inv_bw = ldexpf(1.0f, -e);

    // ---- read 1 (HBM): histogram in that window, exact sums relative to its
    // centre, count, min, max ----------------------------------------------------
    Sums tot{0, 0, df{0.f, 0.f}, df{0.f, 0.f}};
    {
        int n_loc = 0, a1 = 0;
        long long a2 = 0;
        float vmin = INFINITY, vmax = -INFINITY;
        mesh_for_each(G, [&](float x) {
            hist_acc(S.hbuf, x, cstar, inv_bw, a1, a2, tot);
            n_loc++;
            vmin = fminf(vmin, x);
            vmax = fmaxf(vmax, x);
        });
        tot.i1 = a1;
        tot.i2 = a2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
            vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        }
        const int cn[3] = {n_loc, 0, 0};
        warp_partial(S, tot, cn, lane, warp);
        if (lane == 0) { S.redf[warp] = vmin; S.redf[MS_WARPS + warp] = vmax; }
    }
    __syncthreads();
    float mu0 = 0.f, sd0 = 0.f;  // mean and sigma of the mesh (warp 0; used only to re-place a missed window)
    if (warp == 0) {
        int c[3];
        long long i1, i2;
        df o1, o2;
        warp0_totals(S, lane, c, &i1, &i2, &o1, &o2);
        if (lane == 0) {
            float a = INFINITY, b = -INFINITY;
            for (int w = 0; w < MS_WARPS; w++) { a = fminf(a, S.redf[w]); b = fmaxf(b, S.redf[MS_WARPS + w]); }
            S.bc_i[BI_N0] = c[0];
            S.bc_f[2] = a;
            S.bc_f[3] = b;
            if (c[0] > 0) {
                const double unit0 = ldexp(1.0, e - MS_SCALE_BITS);
                const double m1 = ((double)i1 * unit0 + df_to_d(o1)) / c[0];
                const double var = ((double)i2 * unit0 * unit0 + df_to_d(o2)) / c[0] - m1 * m1;
                mu0 = (float)((double)cstar + m1);
                sd0 = (float)sqrt(fmax(var, 0.0));
            }
        }
    }
    __syncthreads();
    const int n0 = S.bc_i[BI_N0];
    const float vmin = S.bc_f[2], vmax = S.bc_f[3];

    if (n0 < J.min_valid || n0 == 0) {
        if (threadIdx.x == 0) { J.raw_bkg[mesh] = 0.f; J.raw_rms[mesh] = -1.f; }
        return;
    }
    if (vmin == vmax) {  // constant mesh: every statistic is that value, sigma 0
        if (threadIdx.x == 0) {
            const double c = (double)vmin;
            double bk;
            switch (J.estimator) {
                case IPP_EST_MEDIAN: case IPP_EST_MEAN: bk = c; break;
                case IPP_EST_FACTORS: bk = J.mf * c - J.mnf * c; break;
                default: bk = 2.5 * c - 1.5 * c; break;
            }
            J.raw_bkg[mesh] = (float)bk;
            J.raw_rms[mesh] = 0.f;
        }
        return;
    }

    // ---- check the window: when the median bin is crowded it is narrowed
    // around the median (window of ~8 robust sigma from the 15.87 / 84.13
    // percentile bins); when the window missed the bulk of the values (median
    // in an end bin, or the end bins holding over 1/8 of them) it is re-placed
    // from the mean and sigma of read 1.  Each change costs one more read (L2).
    const int kq[3] = {(int)(0.1587f * n0), n0 / 2, (int)(0.8413f * n0)};
    int bq[3];
    for (int round = 0; round < 3; round++) {
        if (warp == 0) {
            warp0_scan_counts(S, lane, kq, bq);
            if (lane == 0) {
                int redo = 0;
                float nc = cstar;
                int ne = e;
                const int b16 = bq[0], b50 = bq[1], b84 = bq[2];
                const int ends = (int)(S.hbuf[0] + S.hbuf[MS_NB + 1]);
                if (round < 2 && ((round == 0 && S.bc_i[BI_SBAD]) || b50 == 0 || b50 == MS_NB + 1 || ends > n0 / 8)) {
                    float span = fmaxf(8.0f * sd0, (vmax - vmin) * 1e-6f);
                    span = fmaxf(span, fabsf(mu0) * 1e-6f + 1e-30f);
                    const int e2 = max(min((int)floorf(log2f(span / MS_NB)), 100), -110);
                    const float c2 = rintf(mu0 * ldexpf(1.0f, -e2)) * ldexpf(1.0f, e2);
                    if (e2 != e || c2 != cstar) { redo = 1; ne = e2; nc = c2; }
                } else if (round < 2 && S.hbuf[b50] > 192) {
                    // window of about +-4 sigma_r: the median bins then hold ~n/100 values
                    const float sr = fmaxf(0.5f * (float)(b84 - b16 + 1) * bw, bw * 0.5f);
                    const int e2 = max((int)floorf(log2f(8.0f * sr / MS_NB)), -110);
                    if (e2 < e) {
                        redo = 1;
                        ne = e2;
                        const float centre = cstar + ((float)(b50 - MS_NB / 2 - 1) + 0.5f) * bw;
                        nc = rintf(centre * ldexpf(1.0f, -e2)) * ldexpf(1.0f, e2);
                    }
                }
                S.bc_i[BI_REFINE] = redo;
                S.bc_i[BI_E] = ne;
                S.bc_f[4] = nc;
            }
        }
        __syncthreads();
        if (!S.bc_i[BI_REFINE]) break;
        e = S.bc_i[BI_E];
        cstar = S.bc_f[4];
        bw = ldexpf(1.0f, e);
        inv_bw = ldexpf(1.0f, -e);
        for (int k = threadIdx.x; k < MS_NBT; k += MS_THREADS) S.hbuf[k] = 0;
        __syncthreads();
        tot = Sums{0, 0, df{0.f, 0.f}, df{0.f, 0.f}};
        int a1 = 0;
        long long a2 = 0;
        mesh_for_each(G, [&](float x) { hist_acc(S.hbuf, x, cstar, inv_bw, a1, a2, tot); });  // re-read (L2)
        tot.i1 = a1;
        tot.i2 = a2;
        __syncthreads();
    }

    // ---- what to keep on chip: tails beyond ~2 robust sigma and a band
    // around the median bin, within MS_STORE values ------------------------
    if (warp == 0) {
        if (lane == 0) {
            const int b50 = bq[1];
            const int srb = max(1, bq[1] - bq[0]);  // robust sigma in bins, from the side stars do not inflate
            const int ntot = (int)S.hstart[MS_NBT];
            // tails [0, cl] and [ch, MS_NB+1]: the end bins (outliers) always, when
            // they fit; a tail of -1 / MS_NBT stores nothing on that side
            auto tails = [&](int cl, int ch) {
                return (cl >= 0 ? (int)S.hstart[cl + 1] : 0) + (ch <= MS_NBT - 1 ? ntot - (int)S.hstart[ch] : 0);
            };
            auto band = [&](int D) {
                if (D < 0) return 0;
                const int a = max(b50 - D, 0), b = min(b50 + D, MS_NBT - 1);
                return (int)(S.hstart[b + 1] - S.hstart[a]);
            };
            int T = 2 * srb, D = MS_BAND;
            auto cl_of = [&](int t) { return max(b50 - t, 0); };
            auto ch_of = [&](int t) { return min(b50 + t, MS_NBT - 1); };
            while (D > 2 && tails(cl_of(T), ch_of(T)) + band(D) > MS_STORE) D--;
            while (tails(cl_of(T), ch_of(T)) + band(D) > MS_STORE && (cl_of(T) > 0 || ch_of(T) < MS_NBT - 1))
                T += max(1, srb / 2);
            int cl = cl_of(T), ch = ch_of(T);
            while (D >= 0 && tails(cl, ch) + band(D) > MS_STORE) D--;
            if (tails(cl, ch) > MS_STORE) {  // even the end bins do not fit: keep the smaller one, if any
                const int lo_n = tails(0, MS_NBT), hi_n = tails(-1, MS_NBT - 1);
                if (lo_n <= hi_n) { ch = MS_NBT; if (lo_n > MS_STORE) cl = -1; }
                else { cl = -1; if (hi_n > MS_STORE) ch = MS_NBT; }
            }
            // three disjoint, ordered intervals [0, cl] < [ml, mh] < [ch, NBT-1]: a
            // band touching a tail joins it; tails that meet store everything
            int ml = D >= 0 ? max(b50 - D, 0) : 1, mh = D >= 0 ? min(b50 + D, MS_NBT - 1) : 0;
            if (ml <= mh && ml <= cl + 1) { cl = max(cl, mh); ml = 1; mh = 0; }
            if (ml <= mh && mh >= ch - 1) { ch = min(ch, ml); ml = 1; mh = 0; }
            if (cl >= ch - 1) { cl = MS_NBT - 1; ch = MS_NBT; ml = 1; mh = 0; }
            S.bc_i[BI_CL] = cl;
            S.bc_i[BI_CH] = ch;
            S.bc_i[BI_ML] = ml;
            S.bc_i[BI_MH] = mh;
        }
    }
    for (int k = threadIdx.x; k < (MS_NBT + 31) / 32; k += MS_THREADS) S.sorted_bits[k] = 0;
    __syncthreads();
    const Stored St{S.bc_i[BI_CL], S.bc_i[BI_ML], S.bc_i[BI_MH], S.bc_i[BI_CH]};
    // prefix of the stored counts (closed form over the three intervals) and the scatter cursors
    for (int b = threadIdx.x; b <= MS_NBT; b += MS_THREADS) {
        uint32_t v = S.hstart[min(b, St.cl + 1)];
        if (St.ml <= St.mh && b > St.ml) v += S.hstart[min(b, St.mh + 1)] - S.hstart[St.ml];
        if (St.ch <= MS_NBT - 1 && b > St.ch) v += S.hstart[b] - S.hstart[St.ch];
        S.sstart[b] = v;
        if (b < MS_NBT) S.hbuf[MS_NBT + b] = v;
    }
    __syncthreads();

    // ---- last read (L2): scatter the stored bins in bin order ------------------
    const float fxs = ldexpf(1.0f, MS_SCALE_BITS - e);           // fixed-point scale
    const df nsig = df_from_d(J.nsigma);
    {
        uint32_t* cursor = S.hbuf + MS_NBT;
        mesh_for_each(G, [&](float x) {
            const int b = bin_of(x, cstar, inv_bw);
            if (St.bin(b)) S.store[atomicAdd(&cursor[b], 1u)] = x;
        });
        const int cz[3] = {0, 0, 0};
        warp_partial(S, tot, cz, lane, warp);  // sums of the whole set, from the last histogram read
    }
    __syncthreads();  // scatter and partials complete; S.hbuf is free from here on
    // (the band's bins are sorted when a pass first needs one: typically one or
    // two of them hold a median over all passes)

    // ---- clip passes ----------------------------------------------------------
    // Warp 0 owns the kept set: it selects the median, evaluates Eq. 1-2's
    // statistics and the next bounds, and -- when the values a pass removes are
    // on chip and few -- finds and subtracts them itself and goes on to the
    // next pass without the block.  The block joins (two barriers) only for a
    // long removal range (the first passes over bright stars), a removal that
    // must read the mesh again, or a median bin that must be fetched.
    KeptSet K;
    K.lo = -INFINITY; K.hi = INFINITY; K.bl = 0; K.bh = MS_NB + 1;
    K.nbl = (int)(S.hstart[1] - S.hstart[0]);
    K.nbh = (int)(S.hstart[MS_NBT] - S.hstart[MS_NB + 1]);
    K.n = n0;
    float plo = 0.f, phi = 0.f;   // bounds of the pending pass (warp 0)
    int bm[2] = {0, 0}, rm[2] = {0, 0};  // median bins and ranks of the current set (warp 0)
    int it = 0;                   // passes whose bounds are set (warp 0)
    int pend = 0;                 // removals to apply: 1 in the block partials, 2 in wrem / wc (warp 0)
    int fetched = ST_STOP;        // a median fetch just served by the block (warp 0)
    Sums wrem{0, 0, df{0.f, 0.f}, df{0.f, 0.f}};
    int wc[3] = {0, 0, 0};
    if (warp == 0) {
        int cz[3];
        df o1, o2;
        long long i1, i2;
        warp0_totals(S, lane, cz, &i1, &i2, &o1, &o2);
        if (lane == 0) {
            S.ks_i[0] = i1; S.ks_i[1] = i2; S.ks_o[0] = o1; S.ks_o[1] = o2;
            S.bc_i[BI_GL] = 1; S.bc_i[BI_GH] = 0;   // nothing gathered yet
        }
        __syncwarp();
    }
    // Every round of this loop either ends it, completes a pass, or serves a
    // fetch that the next round's pass consumes: at most 3 (maxiters + 1)
    // rounds.  The cap only guards that bound.
    for (int round = 0; round < 3 * (J.maxiters + 2); round++) {
        if (warp == 0) {
            int state = ST_STOP;
            for (int guard = 0; guard <= J.maxiters + 1; guard++) {
                if (pend) {  // removals of the last pass
                    int c[3];
                    long long i1, i2;
                    df o1, o2;
                    if (pend == 1) {
                        warp0_totals(S, lane, c, &i1, &i2, &o1, &o2);
                    } else {
                        c[0] = wc[0]; c[1] = wc[1]; c[2] = wc[2];
                        i1 = wrem.i1; i2 = wrem.i2; o1 = wrem.o1; o2 = wrem.o2;
                    }
                    pend = 0;
                    // no value dropped: the set is stable (c >= n cannot happen: the
                    // median lies inside [med - k sd, med + k sd])
                    if (c[0] == 0 || c[0] >= K.n) { state = ST_STOP; break; }
                    if (lane == 0) {
                        S.ks_i[0] -= i1; S.ks_i[1] -= i2;
                        S.ks_o[0] = df_sub(S.ks_o[0], o1); S.ks_o[1] = df_sub(S.ks_o[1], o2);
                    }
                    K.bl = bin_of(plo, cstar, inv_bw); K.bh = bin_of(phi, cstar, inv_bw);
                    K.lo = plo; K.hi = phi;
                    K.nbl = c[1]; K.nbh = c[2];
                    K.n -= c[0];
                }
                float mid[2];
                if (fetched != ST_STOP) {  // the median bins the block just fetched
                    const int needm = S.bc_i[BI_NEED];
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        if (fetched == ST_RADIX && ((needm >> q) & 1)) mid[q] = S.bc_f[6 + q];
                        else warp_value_of(S, St, bm[q], rm[q], K, cstar, inv_bw, lane, &mid[q]);
                    }
                    fetched = ST_STOP;
                } else {
                    kept_locate(S, K, (K.n - 1) / 2, lane, &bm[0], &rm[0]);
                    kept_locate(S, K, K.n / 2, lane, &bm[1], &rm[1]);
                    bool have[2];
#pragma unroll
                    for (int q = 0; q < 2; q++)
                        have[q] = warp_value_of(S, St, bm[q], rm[q], K, cstar, inv_bw, lane, &mid[q]);
                    if (!(have[0] && have[1])) {
                        // fetch the median bins that are not stored (both, so that a new
                        // gather never drops one the old gather held): gather them when
                        // they fit, else select from the mesh directly
                        const bool u0 = !St.bin(bm[0]), u1 = !St.bin(bm[1]);
                        const int gl = u0 ? bm[0] : bm[1], gh = u1 ? bm[1] : bm[0];
                        const int need = (int)(S.hstart[gh + 1] - S.hstart[gl]);
                        if (lane == 0) {
                            S.bc_f[2] = K.lo; S.bc_f[3] = K.hi;
                            S.bc_i[BI_NEED] = (!have[0]) | ((!have[1]) << 1);
                            S.bc_i[BI_RB0] = bm[0]; S.bc_i[BI_RR0] = rm[0];
                            S.bc_i[BI_RB1] = bm[1]; S.bc_i[BI_RR1] = rm[1];
                            if (need <= MS_GCAP) {
                                S.bc_i[BI_GL] = gl; S.bc_i[BI_GH] = gh; S.bc_i[BI_GCNT] = 0;
                            }
                        }
                        state = need <= MS_GCAP ? ST_GATHER : ST_RADIX;
                        fetched = state;
                        break;
                    }
                }
                state = warp0_finish(S, J, St, K, mid[0], mid[1], it, cstar, e, inv_bw, nsig, lane, &plo, &phi);
                __syncwarp();   // lane 0's statistics and bounds in shared memory are visible to the warp
                if (state == ST_STOP) break;
                it++;
                // removals on chip (the same decision warp0_finish published, taken from
                // registers every lane holds): scanned here when the range is short
                const int nbl_bin = bin_of(plo, cstar, inv_bw), nbh_bin = bin_of(phi, cstar, inv_bw);
                if (St.range(K.bl, nbl_bin) && St.range(max(nbh_bin, nbl_bin + 1), K.bh)) {
                    const int a0 = S.sstart[K.bl], a1 = S.sstart[nbl_bin + 1];
                    const int ub = max(nbh_bin, nbl_bin + 1);
                    const int b0 = ub <= K.bh ? (int)S.sstart[ub] : 0, b1 = ub <= K.bh ? (int)S.sstart[K.bh + 1] : 0;
                    if ((a1 - a0) + (b1 - b0) <= MS_WARP_SCAN) {
                        Sums rem{0, 0, df{0.f, 0.f}, df{0.f, 0.f}};
                        int c[3] = {0, 0, 0};
                        for (int k = a0 + lane; k < a1; k += kWarp) {
                            const float x = S.store[k];
                            if (!(x >= K.lo && x <= K.hi)) continue;
                            if (x < plo || x > phi) { c[0]++; sums_add(rem, x, bin_of(x, cstar, inv_bw), cstar, fxs); }
                            else if (k >= (int)S.sstart[nbl_bin]) c[1]++;
                        }
                        for (int k = b0 + lane; k < b1; k += kWarp) {
                            const float x = S.store[k];
                            if (!(x >= K.lo && x <= K.hi)) continue;
                            if (x < plo || x > phi) { c[0]++; sums_add(rem, x, bin_of(x, cstar, inv_bw), cstar, fxs); }
                            else if (k < (int)S.sstart[nbh_bin + 1] && nbh_bin != nbl_bin) c[2]++;
                        }
                        wc[0] = warp_sum_i(c[0]); wc[1] = warp_sum_i(c[1]); wc[2] = warp_sum_i(c[2]);
                        const bool anyo = __any_sync(0xffffffffu, rem.o1.hi != 0.f || rem.o2.hi != 0.f);
                        wrem.i1 = warp_sum_ll(rem.i1);
                        wrem.i2 = warp_sum_ll(rem.i2);
                        wrem.o1 = anyo ? warp_sum_df(rem.o1) : df{0.f, 0.f};
                        wrem.o2 = anyo ? warp_sum_df(rem.o2) : df{0.f, 0.f};
                        pend = 2;
                        continue;
                    }
                }
                pend = 1;  // the block scans this pass's removals
                break;
            }
            if (lane == 0) S.bc_i[BI_STATE] = state;
        }
        __syncthreads();
        const int state = S.bc_i[BI_STATE];
        if (state == ST_STOP) break;
        if (state != ST_SCAN) {  // fetch median bins (block-wide); warp 0 then goes on from the fetched values
            const float klo = S.bc_f[2], khi = S.bc_f[3];
            if (state == ST_GATHER) {
                const int gl = S.bc_i[BI_GL], gh = S.bc_i[BI_GH];
                mesh_for_each(G, [&](float x) {
                    const int b = bin_of(x, cstar, inv_bw);
                    if (b >= gl && b <= gh) {
                        const int p = atomicAdd(&S.bc_i[BI_GCNT], 1);
                        if (p < MS_GCAP) S.gbuf[p] = x;
                    }
                });
            } else {
                const int needm = S.bc_i[BI_NEED];
                for (int q = 0; q < 2; q++) {
                    if (!((needm >> q) & 1)) continue;
                    const float v = block_radix_select_global(S, G, klo, khi, S.bc_i[q ? BI_RB1 : BI_RB0], cstar,
                                                              inv_bw, S.bc_i[q ? BI_RR1 : BI_RR0]);
                    if (threadIdx.x == 0) S.bc_f[6 + q] = v;
                }
            }
            __syncthreads();
            continue;
        }
        const float nlo = S.bc_f[0], nhi = S.bc_f[1], klo = S.bc_f[2], khi = S.bc_f[3];
        const int kbl = S.bc_i[BI_KBL], kbh = S.bc_i[BI_KBH];
        const bool on_chip = S.bc_i[BI_MODE];
        const int nbl_bin = bin_of(nlo, cstar, inv_bw), nbh_bin = bin_of(nhi, cstar, inv_bw);
        Sums rem{0, 0, df{0.f, 0.f}, df{0.f, 0.f}};
        int c[3] = {0, 0, 0};  // removed, kept in new bin bl, kept in new bin bh
        if (on_chip) {
            // values removed by this pass lie in bins [bl, nbl_bin] and [nbh_bin, bh]
            const int a0 = S.sstart[kbl], a1 = S.sstart[nbl_bin + 1];
            for (int k = a0 + (int)threadIdx.x; k < a1; k += MS_THREADS) {
                const float x = S.store[k];
                if (!(x >= klo && x <= khi)) continue;
                if (x < nlo || x > nhi) { c[0]++; sums_add(rem, x, bin_of(x, cstar, inv_bw), cstar, fxs); }
                else if (k >= (int)S.sstart[nbl_bin]) c[1]++;
            }
            const int ub = max(nbh_bin, nbl_bin + 1);
            if (ub <= kbh) {
                const int b0 = S.sstart[ub], b1 = S.sstart[kbh + 1];
                for (int k = b0 + (int)threadIdx.x; k < b1; k += MS_THREADS) {
                    const float x = S.store[k];
                    if (!(x >= klo && x <= khi)) continue;
                    if (x < nlo || x > nhi) { c[0]++; sums_add(rem, x, bin_of(x, cstar, inv_bw), cstar, fxs); }
                    else if (k < (int)S.sstart[nbh_bin + 1] && nbh_bin != nbl_bin) c[2]++;
                }
            }
        } else {
            mesh_for_each(G, [&](float x) {
                if (!(x >= klo && x <= khi)) return;
                const int b = bin_of(x, cstar, inv_bw);
                if (x < nlo || x > nhi) { c[0]++; sums_add(rem, x, b, cstar, fxs); }
                else if (b == nbl_bin) c[1]++;
                else if (b == nbh_bin) c[2]++;
            });
        }
        warp_partial(S, rem, c, lane, warp);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const df med = S.st[0], mu = S.st[1], sd = S.st[2];
        df bk;
        switch (J.estimator) {
            case IPP_EST_MEDIAN: bk = med; break;
            case IPP_EST_MEAN: bk = mu; break;
            case IPP_EST_FACTORS: bk = df_sub(df_mul(df_from_d(J.mf), med), df_mul(df_from_d(J.mnf), mu)); break;
            default: bk = df_sub(df_mul_f(med, 2.5f), df_mul_f(mu, 1.5f)); break;
        }
        const float b = __fadd_rn(bk.hi, bk.lo), r = __fadd_rn(sd.hi, sd.lo);
        // values beyond ~1e19 from the window centre overflow the double-float
        // outlier sums: such a mesh is reported invalid (and filled) rather than wrong
        const bool ok = isfinite(b) && isfinite(r);
        J.raw_bkg[mesh] = ok ? b : 0.f;
        J.raw_rms[mesh] = ok ? r : -1.f;
    }
}

__global__ void __launch_bounds__(MS_THREADS, 7) k_mesh_stats(MeshJob J) { mesh_stats_body(J, blockIdx.x); }

// ---------------------------------------------------------------------------
// Invalid-mesh fill and median filter on the mesh grid.  An invalid node takes
// the median of the valid nodes in the smallest (2k+1)^2 neighbourhood holding
// any -- since the smaller neighbourhoods hold none, those are exactly the
// valid nodes on the ring at Chebyshev distance k -- and each node then
// becomes the median of the in-bounds filled nodes of its fw x fh window.
// The fill is computed once per node into the caller's fill arrays (pass 1),
// the window medians read the filled grids (pass 2), each pass a thread per
// node over many blocks.  A grid without any valid node returns at once with
// IPP_ERR_NO_VALID_MESH.
constexpr int MF_THREADS = 64;     // small blocks: a 32 x 32 grid still spreads over 16 SMs

// median (Eq. 1) of the valid nodes on the ring at Chebyshev distance k of
// (p, q) (in-bounds part), by rank counting; cnt = their number (> 0)
__device__ float ring_median(const float* src, const float* raw_rms, int nx, int ny, int p, int q, int k, int cnt) {
    const int k0 = (cnt - 1) / 2, k1 = cnt / 2;
    float a = 0.f, b = 0.f;
    const int p0 = max(p - k, 0), p1 = min(p + k, ny - 1), q0 = max(q - k, 0), q1 = min(q + k, nx - 1);
    for (int pp = p0; pp <= p1; pp++)
        for (int qq = q0; qq <= q1; qq++) {
            if (max(abs(pp - p), abs(qq - q)) != k) continue;
            const int id = pp * nx + qq;
            if (raw_rms[id] < 0.f) continue;
            const float x = src[id];
            int less = 0, leq = 0;
            for (int p2 = p0; p2 <= p1; p2++)
                for (int q2 = q0; q2 <= q1; q2++) {
                    if (max(abs(p2 - p), abs(q2 - q)) != k) continue;
                    const int j = p2 * nx + q2;
                    if (raw_rms[j] < 0.f) continue;
                    const float y = src[j];
                    less += y < x;
                    leq += y <= x;
                }
            if (less <= k0 && k0 < leq) a = x;
            if (less <= k1 && k1 < leq) b = x;
        }
    return (float)(0.5 * ((double)a + (double)b));
}

// fill of node (p, q): its own values when valid, else the ring medians
__device__ __forceinline__ void fill_node(const float* raw_bkg, const float* raw_rms, int nx, int ny, int p, int q,
                                          float* fb, float* fr) {
    const int id = p * nx + q;
    if (raw_rms[id] >= 0.f) { *fb = raw_bkg[id]; *fr = raw_rms[id]; return; }
    for (int k = 1; k < max(nx, ny); k++) {
        const int p0 = max(p - k, 0), p1 = min(p + k, ny - 1), q0 = max(q - k, 0), q1 = min(q + k, nx - 1);
        int cnt = 0;  // valid nodes on ring k: its in-bounds rows p - k, p + k and columns q - k, q + k
        for (int qq = q0; qq <= q1; qq++) {
            if (p - k >= 0) cnt += raw_rms[(p - k) * nx + qq] >= 0.f;
            if (p + k < ny) cnt += raw_rms[(p + k) * nx + qq] >= 0.f;
        }
        for (int pp = max(p - k + 1, 0); pp <= min(p + k - 1, ny - 1); pp++) {
            if (q - k >= 0) cnt += raw_rms[pp * nx + q - k] >= 0.f;
            if (q + k < nx) cnt += raw_rms[pp * nx + q + k] >= 0.f;
        }
        if (cnt > 0) {
            *fb = ring_median(raw_bkg, raw_rms, nx, ny, p, q, k, cnt);
            *fr = ring_median(raw_rms, raw_rms, nx, ny, p, q, k, cnt);
            return;
        }
    }
    *fb = 0.f;  // unreachable when the grid holds a valid node
    *fr = 0.f;
}

// median of the n in-bounds values of a window held in registers (slot i
// used when i < n): rank counting with ties broken by slot, so that every
// index is static and the window stays in registers
template <int N>
__device__ __forceinline__ float reg_median(const float v[N], int n) {
    const int k0 = (n - 1) / 2, k1 = n / 2;
    float a = 0.f, b = 0.f;
#pragma unroll
    for (int i = 0; i < N; i++) {
        int r = 0;
#pragma unroll
        for (int j = 0; j < N; j++) r += (j < n) && (v[j] < v[i] || (v[j] == v[i] && j < i));
        if (i < n && r == k0) a = v[i];
        if (i < n && r == k1) b = v[i];
    }
    return (float)(0.5 * ((double)a + (double)b));
}

// window median of node (p, q) over filled grids fb, fr (row-major, nx wide)
template <int FW, int FH>
__device__ __forceinline__ void window_median(const float* fb, const float* fr, int nx, int ny, int p, int q,
                                              float* ob, float* orr) {
    constexpr int N = FW * FH;
    float wb[N], wr[N];
    int n = 0;
#pragma unroll
    for (int a = 0; a < FH; a++)
#pragma unroll
        for (int c = 0; c < FW; c++) {
            const int pp = p - FH / 2 + a, qq = q - FW / 2 + c;
            const bool in = pp >= 0 && pp < ny && qq >= 0 && qq < nx;
            // in-bounds values packed to the front (n counts them), keeping static indices
            const float vb = in ? fb[pp * nx + qq] : 0.f, vr = in ? fr[pp * nx + qq] : 0.f;
#pragma unroll
            for (int s = 0; s < N; s++)
                if (s == n && in) { wb[s] = vb; wr[s] = vr; }
            n += in;
        }
#pragma unroll
    for (int s = 0; s < N; s++)
        if (s >= n) { wb[s] = 0.f; wr[s] = 0.f; }
    *ob = reg_median<N>(wb, n);
    *orr = reg_median<N>(wr, n);
}

__device__ __forceinline__ void window_median_any(const float* fb, const float* fr, int nx, int ny, int p, int q,
                                                  int fw, int fh, float* ob, float* orr) {
    if (fw == 3 && fh == 3) { window_median<3, 3>(fb, fr, nx, ny, p, q, ob, orr); return; }
    if (fw == 1 && fh == 1) { *ob = fb[p * nx + q]; *orr = fr[p * nx + q]; return; }
    if (fw == 5 && fh == 5) { window_median<5, 5>(fb, fr, nx, ny, p, q, ob, orr); return; }
    // other odd shapes up to 7 x 7: the 7 x 7 window with the rows and columns
    // beyond the requested shape treated as out of bounds
    constexpr int N = 49;
    float wb[N], wr[N];
    int n = 0;
    for (int a = 0; a < fh; a++)
        for (int c = 0; c < fw; c++) {
            const int pp = p - fh / 2 + a, qq = q - fw / 2 + c;
            if (pp < 0 || pp >= ny || qq < 0 || qq >= nx) continue;
            wb[n] = fb[pp * nx + qq];
            wr[n] = fr[pp * nx + qq];
            n++;
        }
    for (int s = n; s < N; s++) { wb[s] = 0.f; wr[s] = 0.f; }
    *ob = reg_median<N>(wb, n);
    *orr = reg_median<N>(wr, n);
}

// pass 1: fills into the caller's arrays.  Each block first checks
// that the grid holds a valid node (a block-wide scan of raw_rms).
__device__ __forceinline__ void mesh_fill_body(const float* raw_bkg, const float* raw_rms, int nx, int ny,
                                               float* fill_bkg, float* fill_rms, int32_t* status_dev, int vb) {
    const int nn = nx * ny;
    int any = 0;
    for (int i = threadIdx.x; i < nn && !any; i += MF_THREADS) any |= raw_rms[i] >= 0.f;
    if (!__syncthreads_or(any)) {
        const int id = vb * MF_THREADS + threadIdx.x;
        if (id < nn) { fill_bkg[id] = 0.f; fill_rms[id] = -1.f; }  // -1: pass 2 writes zeros
        if (id == 0 && status_dev) *status_dev = IPP_ERR_NO_VALID_MESH;
        return;
    }
    const int id = vb * MF_THREADS + threadIdx.x;
    if (id >= nn) return;
    const int p = id / nx, q = id - p * nx;
    fill_node(raw_bkg, raw_rms, nx, ny, p, q, &fill_bkg[id], &fill_rms[id]);
    if (id == 0 && status_dev) *status_dev = IPP_OK;
}

__global__ void __launch_bounds__(MF_THREADS) k_mesh_fill(const float* raw_bkg, const float* raw_rms, int nx, int ny,
                                                          float* fill_bkg, float* fill_rms, int32_t* status_dev) {
    mesh_fill_body(raw_bkg, raw_rms, nx, ny, fill_bkg, fill_rms, status_dev, blockIdx.x);
}

// pass 2: window medians of the filled grids
__device__ __forceinline__ void mesh_median_body(const float* fill_bkg, const float* fill_rms, int nx, int ny, int fw,
                                                 int fh, float* out_bkg, float* out_rms, int vb) {
    const int id = vb * MF_THREADS + threadIdx.x;
    if (id >= nx * ny) return;
    if (fill_rms[0] < 0.f) { out_bkg[id] = 0.f; out_rms[id] = 0.f; return; }  // no valid mesh (pass 1)
    const int p = id / nx, q = id - p * nx;
    window_median_any(fill_bkg, fill_rms, nx, ny, p, q, fw, fh, &out_bkg[id], &out_rms[id]);
}

__global__ void __launch_bounds__(MF_THREADS) k_mesh_median(const float* fill_bkg, const float* fill_rms, int nx,
                                                            int ny, int fw, int fh, float* out_bkg, float* out_rms) {
    mesh_median_body(fill_bkg, fill_rms, nx, ny, fw, fh, out_bkg, out_rms, blockIdx.x);
}

// ---- batched form: the same bodies over a table of frames ------------------
__global__ void __launch_bounds__(MS_THREADS, 7) k_mesh_stats_multi(const MeshJob* J, const int* bs, int nf) {
    const int f = frame_of(bs, nf, blockIdx.x);
    mesh_stats_body(J[f], blockIdx.x - bs[f]);
}

__global__ void __launch_bounds__(MF_THREADS) k_mesh_fill_multi(const MeshFilterJob* J, const int* bs, int nf) {
    const int f = frame_of(bs, nf, blockIdx.x);
    const MeshFilterJob& F = J[f];
    mesh_fill_body(F.raw_bkg, F.raw_rms, F.nx, F.ny, F.fill_bkg, F.fill_rms, F.status_dev, blockIdx.x - bs[f]);
}

__global__ void __launch_bounds__(MF_THREADS) k_mesh_median_multi(const MeshFilterJob* J, const int* bs, int nf) {
    const int f = frame_of(bs, nf, blockIdx.x);
    const MeshFilterJob& F = J[f];
    mesh_median_body(F.fill_bkg, F.fill_rms, F.nx, F.ny, F.fw, F.fh, F.out_bkg, F.out_rms, blockIdx.x - bs[f]);
}

// ---------------------------------------------------------------------------
// Interpolation + subtraction over tiles of BG_TH rows x 128 columns: per row
// the mesh columns are first interpolated vertically (a handful of values in
// shared memory), then each pixel needs only the 4 horizontal Keys weights of
// its column, held in registers.  float4 loads/stores when aligned.
constexpr int BG_TW = 128, BG_TH = 32, BG_THREADS = 256, BG_NQ = 40;


__device__ __forceinline__ float load_pix(const SubJob& J, int64_t y, int64_t x) {
    if (J.dtype == IPP_F32) return __ldg(reinterpret_cast<const float*>(J.img) + y * J.pitch + x);
    float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(J.img) + y * J.pitch + x);
    float b = J.bias_map ? __ldg(J.bias_map + y * J.W + x) : J.bias;
    return (raw - b) * __ldg(J.inv_flat + y * J.W + x);
}

__global__ void __launch_bounds__(BG_THREADS) k_bg_subtract(SubJob J) {
    __shared__ float cv[BG_TH][BG_NQ];
    const int64_t tx0 = (int64_t)blockIdx.x * BG_TW, ty0 = (int64_t)blockIdx.y * BG_TH;
    // node columns used by this tile
    const int qa = (int)floorf(((float)(int)tx0 + 0.5f) / J.mesh_w - 0.5f) - 1;
    const int qz = (int)floorf(((float)((int)tx0 + BG_TW - 1) + 0.5f) / J.mesh_w - 0.5f) + 2;
    const int qbase = max(qa, 0);
    const int nq = min(min(qz, J.nx - 1) - qbase + 1, BG_NQ);  // node columns this tile reads
    // per-row vertical interpolation of the needed node columns
    const float ref = J.mesh[0];
    for (int t = threadIdx.x; t < BG_TH * nq; t += BG_THREADS) {
        int r = t / nq, qq = t - r * nq;
        int q = min(qbase + qq, J.nx - 1);
        float vy = ((float)((int)ty0 + r) + 0.5f) / J.mesh_h - 0.5f;
        float pf = floorf(vy);
        float w[4];
        keys_weights(vy - pf, w);
        int p0 = (int)pf;
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            int p = clampi(p0 - 1 + a, 0, J.ny - 1);
            acc = fmaf(w[a], J.mesh[p * J.nx + q] - ref, acc);
        }
        cv[r][qq] = acc;
    }
    __syncthreads();
    // each thread: 4 consecutive columns, rows warp, warp + 8, ...
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t xc = tx0 + lane * 4;
    float wx[4][4];
    int qi[4][4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        float u = ((float)((int)xc + c) + 0.5f) / J.mesh_w - 0.5f;
        float qf = floorf(u);
        keys_weights(u - qf, wx[c]);
        int q0 = (int)qf;
#pragma unroll
        for (int b = 0; b < 4; b++) qi[c][b] = min(clampi(q0 - 1 + b, 0, J.nx - 1) - qbase, BG_NQ - 1);
    }
    const bool vec = (J.dtype == IPP_F32) && (J.pitch % 4 == 0) && (J.sub_pitch % 4 == 0) &&
                     (((uintptr_t)J.img & 15) == 0) && (((uintptr_t)J.sub & 15) == 0) &&
                     (!J.bkg_map || ((uintptr_t)J.bkg_map & 15) == 0) && (xc + 4 <= J.W);
    constexpr int RPW = BG_TH / (BG_THREADS / 32);  // rows per warp: loads first, then math
    float f[RPW][4];
#pragma unroll
    for (int q = 0; q < RPW; q++) {
        const int r = warp + q * (BG_THREADS / 32);
        const int64_t y = ty0 + r;
#pragma unroll
        for (int c = 0; c < 4; c++) f[q][c] = 0.f;
        if (y >= J.H) continue;
        if (vec) {
            const float4 t4 = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(J.img) + y * J.pitch + xc));
            f[q][0] = t4.x; f[q][1] = t4.y; f[q][2] = t4.z; f[q][3] = t4.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) f[q][c] = (xc + c < J.W) ? load_pix(J, y, xc + c) : 0.f;
        }
    }
#pragma unroll
    for (int q = 0; q < RPW; q++) {
        const int r = warp + q * (BG_THREADS / 32);
        const int64_t y = ty0 + r;
        if (y >= J.H) continue;
        float B[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float acc = 0.f;
#pragma unroll
            for (int b = 0; b < 4; b++) acc = fmaf(wx[c][b], cv[r][qi[c][b]], acc);
            B[c] = ref + acc;
        }
        if (vec) {
            *reinterpret_cast<float4*>(J.sub + y * J.sub_pitch + xc) =
                make_float4(f[q][0] - B[0], f[q][1] - B[1], f[q][2] - B[2], f[q][3] - B[3]);
            if (J.bkg_map) *reinterpret_cast<float4*>(J.bkg_map + y * J.sub_pitch + xc) = make_float4(B[0], B[1], B[2], B[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (xc + c < J.W) {
                    J.sub[y * J.sub_pitch + xc + c] = f[q][c] - B[c];
                    if (J.bkg_map) J.bkg_map[y * J.sub_pitch + xc + c] = B[c];
                }
        }
    }
}

}  // namespace ipp

// ------------------------------------------------------------------ host side
using namespace ipp;

int ipp_launch_mesh_stats(const MeshJob& J, cudaStream_t s) {
    if (J.mesh_w * J.mesh_h > 16384)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "mesh area %d > 16384", J.mesh_w * J.mesh_h);
    // seven 31 KB CTAs per SM need the largest shared-memory carveout; the
    // attribute is per device, so it is set once on each device that launches
    if (int e = ipp_once_per_device(0, [] {
            return cudaFuncSetAttribute(k_mesh_stats, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        cudaSharedmemCarveoutMaxShared);
        }))
        return e;
    k_mesh_stats<<<J.nx * J.ny, MS_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_mesh_stats");
}

int ipp_launch_mesh_filter(const float* raw_bkg, const float* raw_rms, float* fill_bkg, float* fill_rms,
                           int nx, int ny, int fw, int fh, float* out_bkg, float* out_rms,
                           int32_t* status_dev, cudaStream_t s) {
    const int nn = nx * ny;
    if (!fill_bkg || !fill_rms) return ipp_set_error(IPP_ERR_INVALID_ARG, "fill arrays NULL");
    const int blocks = (nn + MF_THREADS - 1) / MF_THREADS;
    k_mesh_fill<<<blocks, MF_THREADS, 0, s>>>(raw_bkg, raw_rms, nx, ny, fill_bkg, fill_rms, status_dev);
    if (int e = ipp_check_launch("k_mesh_fill")) return e;
    k_mesh_median<<<blocks, MF_THREADS, 0, s>>>(fill_bkg, fill_rms, nx, ny, fw, fh, out_bkg, out_rms);
    return ipp_check_launch("k_mesh_median");
}

int ipp_launch_bg_subtract(const SubJob& J, cudaStream_t s) {
    if (J.mesh_w < 4 || J.mesh_h < 4)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "mesh size below 4 px");
    dim3 grid((unsigned)cdiv(J.W, BG_TW), (unsigned)cdiv(J.H, BG_TH));
    k_bg_subtract<<<grid, BG_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_bg_subtract");
}


int ipp_bg_multi_pack(const MeshJob* J, const MeshFilterJob* F, int nf, HostBlob& hb, BgMultiPlan* p) {
    int nb[1024];
    if (nf < 1 || nf > 1024) return ipp_set_error(IPP_ERR_INVALID_ARG, "1..1024 frames");
    for (int f = 0; f < nf; f++) {
        if (J[f].mesh_w * J[f].mesh_h > 16384)
            return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "mesh area %d > 16384", J[f].mesh_w * J[f].mesh_h);
        nb[f] = J[f].nx * J[f].ny;
    }
    p->stats = ipp_put_stage(hb, J, nb, nf);
    for (int f = 0; f < nf; f++) nb[f] = (F[f].nx * F[f].ny + MF_THREADS - 1) / MF_THREADS;
    p->fill = ipp_put_stage(hb, F, nb, nf);
    p->median = p->fill;
    p->nf = nf;
    return hb.ok() ? IPP_OK : ipp_set_error(IPP_ERR_INVALID_ARG, "batch table overflow");
}

int ipp_bg_multi_launch(const BgMultiPlan& p, const unsigned char* t, cudaStream_t s) {
    cudaFuncSetAttribute(k_mesh_stats_multi, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    k_mesh_stats_multi<<<(unsigned)p.stats.total, MS_THREADS, 0, s>>>(
        reinterpret_cast<const MeshJob*>(t + p.stats.jobs), reinterpret_cast<const int*>(t + p.stats.bs), p.nf);
    if (int e = ipp_check_launch("k_mesh_stats_multi")) return e;
    const MeshFilterJob* F = reinterpret_cast<const MeshFilterJob*>(t + p.fill.jobs);
    const int* bs = reinterpret_cast<const int*>(t + p.fill.bs);
    k_mesh_fill_multi<<<(unsigned)p.fill.total, MF_THREADS, 0, s>>>(F, bs, p.nf);
    if (int e = ipp_check_launch("k_mesh_fill_multi")) return e;
    k_mesh_median_multi<<<(unsigned)p.median.total, MF_THREADS, 0, s>>>(F, bs, p.nf);
    return ipp_check_launch("k_mesh_median_multi");
}
