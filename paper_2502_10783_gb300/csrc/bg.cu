// bg.cu -- mesh background (Sec. 2.2.2, Eqs. 1-4): per-mesh iterative sigma
// clip, invalid-mesh fill and mesh median filter, interpolation + subtraction.
//
// k_mesh_stats: one CTA (512 threads) per mesh.  The mesh is read once from HBM
// into registers.  A histogram over a window around the mean (refined around
// the median when outliers made it coarse) turns the mesh into a bin-sorted copy
// in shared memory.  The sums of the whole set are taken once, exactly: values
// inside the window as int64 fixed point (a power-of-two scale no coarser than
// their own spacing), the few outside it in double-float.  Every clip pass then only
// touches the values it removes (the tails, bin by bin) and the bins holding
// the median order statistics, so a pass costs O(removed + median bin), not
// O(mesh), and the bounds agree with an FP64 evaluation to ~1e-13.  Scalar FP64
// work (moments, bounds) runs on one thread: the FP64 pipe is narrow.
#include <math.h>

#include "jobs.cuh"

namespace ipp {

constexpr int MS_THREADS = 512;
constexpr int MS_WARPS = MS_THREADS / kWarp;
constexpr int MS_NB = 1024;          // window bins 1..MS_NB; 0 = below, MS_NB+1 = above
constexpr int MS_NBT = MS_NB + 2;
constexpr int MS_SCALE_BITS = 14;    // fixed point: d_int = (v - c*) * 2^(14 - e), bw = 2^e

struct MeshShared {
    uint32_t hcnt[MS_NBT];
    uint32_t hstart[MS_NBT + 1];
    uint32_t hfill[MS_NBT];   // scatter cursors; reused as radix-select histogram
    uint32_t radix[2048];
    uint32_t sorted_bits[(MS_NBT + 31) / 32];  // bins whose slice is already sorted
    long long redl[MS_WARPS * 2];
    float4 redo[MS_WARPS];
    int redi[MS_WARPS * 3];
    float redf[MS_WARPS * 3];
    double bc_d[8];
    long long bc_l[4];
    long long ks_i[2];   // running sums of the kept set (clip loop, warp 0 lane 0)
    double ks_o[2];
    double st[3];        // median, mean, sigma of the kept set
    int bc_i[8];
    float bc_f[4];
    uint32_t bc_u[2];
};

// Bin of a value: monotone in v (FP subtraction and the power-of-two scaling
// are monotone), clamped to [0, MS_NB+1].
__device__ __forceinline__ int bin_of(float v, float cstar, float inv_bw) {
    float t = floorf((v - cstar) * inv_bw);
    t = fmaxf(fminf(t, (float)(MS_NB / 2)), (float)(-MS_NB / 2 - 1));
    return (int)t + MS_NB / 2 + 1;
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

// Warp 0 only, after a barrier: totals of the per-warp partials.  Counts in
// every lane; sums (int64 and the outlier sums as FP64) valid in lane 0.
__device__ __forceinline__ void warp0_totals(const MeshShared& S, int lane, int c[3], long long* i1, long long* i2,
                                             double* o1, double* o2) {
    const bool in = lane < MS_WARPS;
    *i1 = warp_sum_ll(in ? S.redl[lane] : 0);
    *i2 = warp_sum_ll(in ? S.redl[MS_WARPS + lane] : 0);
    const float4 o = in ? S.redo[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    const df xx = warp_sum_df(df{o.x, o.y}), yy = warp_sum_df(df{o.z, o.w});
    c[0] = warp_sum_i(in ? S.redi[lane] : 0);
    c[1] = warp_sum_i(in ? S.redi[MS_WARPS + lane] : 0);
    c[2] = warp_sum_i(in ? S.redi[2 * MS_WARPS + lane] : 0);
    if (lane == 0) { *o1 = df_to_d(xx); *o2 = df_to_d(yy); }
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

// Warp 0 only: sort bin b's slice in place once (slices up to 256 values).
__device__ void warp_ensure_sorted(MeshShared& S, float* sval, int b, int lane) {
    if ((S.sorted_bits[b >> 5] >> (b & 31)) & 1u) return;
    const int s0 = S.hstart[b], m = (int)S.hstart[b + 1] - s0;
    if (m <= 32) warp_sort_slice<1>(sval, s0, m, lane);
    else if (m <= 64) warp_sort_slice<2>(sval, s0, m, lane);
    else if (m <= 128) warp_sort_slice<4>(sval, s0, m, lane);
    else warp_sort_slice<8>(sval, s0, m, lane);
    if (lane == 0) S.sorted_bits[b >> 5] |= 1u << (b & 31);
    __syncwarp();
}

constexpr int MS_WARPSORT_MAX = 256;

// Warp 0 only: r-th smallest of the elements of slice [s0, s1) within [lo, hi]
// for slices too long to sort: 11/11/10-bit radix passes over the
// order-preserving keys with the histogram in shared memory.
__device__ float warp_radix_select(MeshShared& S, const float* sval, int s0, int s1, float lo, float hi, int r,
                                   int lane) {
    uint32_t prefix = 0, pmask = 0;
    int rr = r;
    for (int pass = 0; pass < 3; pass++) {
        const int sh = pass == 0 ? 21 : (pass == 1 ? 10 : 0);
        const int nb = pass == 2 ? 1024 : 2048, per = nb / 32;
        for (int k = lane; k < nb; k += 32) S.radix[k] = 0;
        __syncwarp();
        for (int k = s0 + lane; k < s1; k += 32) {
            const float v = sval[k];
            if (!(v >= lo && v <= hi)) continue;
            const uint32_t key = fkey(v);
            if ((key & pmask) != prefix) continue;
            atomicAdd(&S.radix[(key >> sh) & (nb - 1)], 1u);
        }
        __syncwarp();
        int tot = 0;
        for (int d = lane * per; d < (lane + 1) * per; d++) tot += (int)S.radix[d];
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
                const int c = (int)S.radix[d];
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

// State of the kept set [lo, hi] of a clip pass.
struct KeptSet {
    float lo, hi;
    int bl, bh;     // bins of lo and hi
    int nbl, nbh;   // kept elements in slices bl and bh (nbh unused when bl == bh)
    int n;
};

// Bin and rank (among the kept values of that bin) of the k-th smallest kept value.
__device__ __forceinline__ void kept_locate(const MeshShared& S, const KeptSet& K, int k, int* bin, int* r) {
    const int full = (K.bh > K.bl + 1) ? (int)(S.hstart[K.bh] - S.hstart[K.bl + 1]) : 0;
    const int nbl = (K.bl == K.bh) ? K.n : K.nbl;
    if (k < nbl) {
        *bin = K.bl; *r = k;
    } else if (k - nbl < full) {
        const int kk = k - nbl;
        const uint32_t base = S.hstart[K.bl + 1];
        int a = K.bl + 1, b = K.bh - 1;
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if ((int)(S.hstart[mid] - base) <= kk) a = mid; else b = mid - 1;
        }
        *bin = a; *r = kk - (int)(S.hstart[a] - base);
    } else {
        *bin = K.bh; *r = k - nbl - full;
    }
}

// Warp 0 only: the two middle order statistics x_k0, x_k1 (k0 = (n-1)/2,
// k1 = n/2) of the kept set; Eq. 1's median is their mean.  Bins of up to
// MS_WARPSORT_MAX values are sorted once per mesh and indexed; longer ones are
// selected by radix passes.
__device__ void kept_middle(MeshShared& S, float* sval, const KeptSet& K, float vals[2], int lane) {
    for (int q = 0; q < 2; q++) {
        const int kq = q == 0 ? (K.n - 1) / 2 : K.n / 2;
        if (q == 1 && kq == (K.n - 1) / 2) { vals[1] = vals[0]; break; }
        int b, r;
        kept_locate(S, K, kq, &b, &r);
        const int s0 = S.hstart[b], s1 = S.hstart[b + 1];
        const bool sorted = (S.sorted_bits[b >> 5] >> (b & 31)) & 1u;
        if (sorted || s1 - s0 <= MS_WARPSORT_MAX) {
            warp_ensure_sorted(S, sval, b, lane);
            int a = s0, e = s1;  // first value >= lo in the sorted slice
            while (a < e) { const int m = (a + e) >> 1; if (sval[m] < K.lo) a = m + 1; else e = m; }
            vals[q] = sval[a + r];
        } else {
            vals[q] = warp_radix_select(S, sval, s0, s1, K.lo, K.hi, r, lane);
        }
    }
}

// Scalar FP64 statistics of the kept set (one thread): mean and population sigma.
struct KeptSums {
    long long i1, i2;
    double o1, o2;
};
__device__ __forceinline__ void kept_stats(const KeptSums& t, int n, float cstar, double unit, double* mu,
                                           double* sd) {
    const double s1 = (double)t.i1 * unit + t.o1;
    const double s2 = (double)t.i2 * unit * unit + t.o2;
    const double m1 = s1 / n;
    *mu = (double)cstar + m1;
    *sd = sqrt(fmax(s2 / n - m1 * m1, 0.0));
}

template <int PPT>
__global__ void __launch_bounds__(MS_THREADS, 2) k_mesh_stats(MeshJob J) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MeshShared& S = *reinterpret_cast<MeshShared*>(smem_raw);
    float* sval = reinterpret_cast<float*>(smem_raw + sizeof(MeshShared));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const int mesh = blockIdx.x;
    const int mx = mesh % J.nx, my = mesh / J.nx;
    const int64_t x0 = (int64_t)mx * J.mesh_w, y0 = (int64_t)my * J.mesh_h;
    const int we = (int)min((int64_t)J.mesh_w, J.W - x0);
    const int he = (int)min((int64_t)J.mesh_h, J.H - y0);
    const int slots = J.mesh_w * J.mesh_h;

    // ---- load (the one HBM read of the mesh); approximate moments ------------
    // element e = threadIdx.x + k * 512 of the mesh sits at (r, c); both advance
    // by fixed steps with k, so no division inside the loop
    float v[PPT];
    const int dr = MS_THREADS / J.mesh_w, dc = MS_THREADS - dr * J.mesh_w;
    const float qnan = __int_as_float(0x7fc00000);  // NaN = not usable
    if (J.dtype == IPP_F32) {
        // every load is issued before any is used: addresses are clamped into
        // the mesh and the out-of-mesh slots are blanked afterwards
        const float* base = reinterpret_cast<const float*>(J.img) + y0 * J.pitch + x0;
        uint32_t inside = 0;
        int r = threadIdx.x / J.mesh_w, c = threadIdx.x - r * J.mesh_w;
        const float* rowp = base + (int64_t)min(r, he - 1) * J.pitch;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int e = threadIdx.x + k * MS_THREADS;
            inside |= (uint32_t)(e < slots && r < he && c < we) << k;
            v[k] = __ldg(rowp + min(c, we - 1));
            const int r0 = r;
            r += dr;
            c += dc;
            if (c >= J.mesh_w) { c -= J.mesh_w; r++; }
            rowp += (int64_t)(min(r, he - 1) - min(r0, he - 1)) * J.pitch;
        }
#pragma unroll
        for (int k = 0; k < PPT; k++)
            if (!((inside >> k) & 1u) || !isfinite(v[k])) v[k] = qnan;
        if (J.mask) {
            r = threadIdx.x / J.mesh_w;
            c = threadIdx.x - r * J.mesh_w;
#pragma unroll
            for (int k = 0; k < PPT; k++) {
                if (v[k] == v[k] && J.mask[(y0 + r) * J.W + x0 + c]) v[k] = qnan;
                r += dr;
                c += dc;
                if (c >= J.mesh_w) { c -= J.mesh_w; r++; }
            }
        }
    } else {
        int r = threadIdx.x / J.mesh_w, c = threadIdx.x - r * J.mesh_w;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int e = threadIdx.x + k * MS_THREADS;
            float x = qnan;
            if (e < slots && r < he && c < we) {
                const int64_t yy = y0 + r, xx = x0 + c;
                const float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(J.img) + yy * J.pitch + xx);
                const float b = J.bias_map ? __ldg(J.bias_map + yy * J.W + xx) : J.bias;
                x = (raw - b) * __ldg(J.inv_flat + yy * J.W + xx);
                if (J.mask && J.mask[yy * J.W + xx]) x = qnan;
                if (!isfinite(x)) x = qnan;
            }
            v[k] = x;
            r += dr;
            c += dc;
            if (c >= J.mesh_w) { c -= J.mesh_w; r++; }
        }
    }
    int n_loc = 0;
    float piv = 0.f, s = 0.f, q = 0.f, vmin = INFINITY, vmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const float x = v[k];
        if (x == x) {
            if (n_loc == 0) piv = x;
            n_loc++;
            const float d = x - piv;
            s += d;
            q = fmaf(d, d, q);
            vmin = fminf(vmin, x);
            vmax = fmaxf(vmax, x);
        }
    }
    // merge (n, mean, M2) across the block (Chan et al.); FP32 is enough here:
    // these moments only place the histogram window
    float mean = n_loc ? piv + s / n_loc : 0.f;
    float m2 = n_loc ? fmaxf(q - s * s / n_loc, 0.f) : 0.f;
    float cnt = (float)n_loc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float nb = __shfl_xor_sync(0xffffffffu, cnt, o);
        const float mb = __shfl_xor_sync(0xffffffffu, mean, o);
        const float qb = __shfl_xor_sync(0xffffffffu, m2, o);
        const float nt = cnt + nb;
        if (nt > 0.f) {
            const float dl = mb - mean;
            mean = mean + dl * (nb / nt);
            m2 = m2 + qb + dl * dl * (cnt * nb / nt);
        }
        cnt = nt;
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if (lane == 0) {
        S.redf[warp] = cnt; S.redf[MS_WARPS + warp] = mean; S.redf[2 * MS_WARPS + warp] = m2;
        S.redi[warp] = __float_as_int(vmin); S.redi[MS_WARPS + warp] = __float_as_int(vmax);
    }
    for (int k = threadIdx.x; k < MS_NBT; k += MS_THREADS) S.hcnt[k] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        float c = 0.f, mu = 0.f, mm = 0.f, a = INFINITY, b = -INFINITY;
        for (int w = 0; w < MS_WARPS; w++) {
            const float nb = S.redf[w], mb = S.redf[MS_WARPS + w], qb = S.redf[2 * MS_WARPS + w];
            const float nt = c + nb;
            if (nt > 0.f) {
                const float dl = mb - mu;
                mu = mu + dl * (nb / nt);
                mm = mm + qb + dl * dl * (c * nb / nt);
            }
            c = nt;
            a = fminf(a, __int_as_float(S.redi[w]));
            b = fmaxf(b, __int_as_float(S.redi[MS_WARPS + w]));
        }
        S.bc_i[0] = (int)c;
        S.bc_f[0] = mu;
        S.bc_f[1] = c > 0.f ? sqrtf(mm / c) : 0.f;
        S.bc_f[2] = a;
        S.bc_f[3] = b;
    }
    __syncthreads();
    const int n0 = S.bc_i[0];
    const float mu0 = S.bc_f[0], sd0 = S.bc_f[1];
    vmin = S.bc_f[2];
    vmax = S.bc_f[3];

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

    // ---- histogram window: bw = 2^e, width NB*bw in (4, 8] sigma0, centre c* a
    // multiple of bw near the mean; refined once around the median bin when it
    // is crowded (outliers inflate sigma0).  Values outside the window land in
    // the two end bins, whose slices are handled element by element. ---------
    int e;
    float cstar, bw, inv_bw;
    {
        float span = fmaxf(8.0f * sd0, (vmax - vmin) * 1e-6f);
        span = fmaxf(span, fabsf(mu0) * 1e-6f + 1e-30f);
        e = (int)floorf(log2f(span / MS_NB));
        e = max(min(e, 100), -110);
        bw = ldexpf(1.0f, e);
        inv_bw = ldexpf(1.0f, -e);
        cstar = rintf(mu0 * inv_bw) * bw;
    }
    // (S.hcnt was cleared before the barrier above)
    for (int round = 0; round < 2; round++) {
#pragma unroll
        for (int k = 0; k < PPT; k++)
            if (v[k] == v[k]) atomicAdd(&S.hcnt[bin_of(v[k], cstar, inv_bw)], 1u);
        __syncthreads();
        if (warp == 0) {  // exclusive scan of the counts; bins of the 15.87 / 50 / 84.13 percentiles
            constexpr int PER = (MS_NBT + 31) / 32;
            const int b0 = lane * PER;
            int acc = 0;
            for (int b = b0; b < min(b0 + PER, MS_NBT); b++) acc += (int)S.hcnt[b];
            int inc = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            int run = inc - acc;
            // each lane resolves the percentiles that fall in its range of bins
            const int kq[3] = {(int)(0.1587f * n0), n0 / 2, (int)(0.8413f * n0)};
            int bq[3] = {0, 0, 0};
            unsigned hit = 0;
            for (int b = b0; b < min(b0 + PER, MS_NBT); b++) {
                const int h = (int)S.hcnt[b];
                S.hstart[b] = (uint32_t)run;
                S.hfill[b] = (uint32_t)run;  // scatter cursor
#pragma unroll
                for (int t = 0; t < 3; t++)
                    if (kq[t] >= run && kq[t] < run + h) { bq[t] = b; hit |= 1u << t; }
                run += h;
            }
            if (lane == 31) S.hstart[MS_NBT] = (uint32_t)inc;
            int bqa[3];
#pragma unroll
            for (int t = 0; t < 3; t++) {
                const unsigned who = __ballot_sync(0xffffffffu, (hit >> t) & 1u);
                bqa[t] = __shfl_sync(0xffffffffu, bq[t], who ? __ffs(who) - 1 : 0);
            }
            if (lane == 0) {
                int refine = 0;
                float nc = cstar, nbw = bw, ninv = inv_bw;
                int ne = e;
                const int b16 = bqa[0], b50 = bqa[1], b84 = bqa[2];
                if (round == 0 && b50 >= 1 && b50 <= MS_NB && S.hcnt[b50] > 64) {
                    // window of about +-4 sigma_r: the median bins then hold ~n/100 values
                    const float sr = fmaxf(0.5f * (float)(b84 - b16 + 1) * bw, bw * 0.5f);
                    int e2 = (int)floorf(log2f(8.0f * sr / MS_NB));
                    e2 = max(e2, -110);
                    if (e2 < e) {
                        refine = 1;
                        ne = e2;
                        nbw = ldexpf(1.0f, e2);
                        ninv = ldexpf(1.0f, -e2);
                        const float centre = cstar + ((float)(b50 - MS_NB / 2 - 1) + 0.5f) * bw;
                        nc = rintf(centre * ninv) * nbw;
                    }
                }
                S.bc_i[7] = refine;
                S.bc_i[5] = ne;
                S.bc_f[0] = nc;
                S.bc_f[1] = nbw;
                S.bc_f[2] = ninv;
            }
        }
        __syncthreads();
        const int refine = S.bc_i[7];
        if (!refine) break;
        e = S.bc_i[5];
        cstar = S.bc_f[0];
        bw = S.bc_f[1];
        inv_bw = S.bc_f[2];
        for (int k = threadIdx.x; k < MS_NBT; k += MS_THREADS) S.hcnt[k] = 0;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < (MS_NBT + 31) / 32; k += MS_THREADS) S.sorted_bits[k] = 0;

    // ---- scatter into bin order + exact sums of the whole set ----------------
    // 8 cursor increments are in flight before their stores, not one at a time
    const float fxs = ldexpf(1.0f, MS_SCALE_BITS - e);           // fixed-point scale
    const double unit = ldexp(1.0, e - MS_SCALE_BITS);
    {
        Sums tot{0, 0, df{0.f, 0.f}, df{0.f, 0.f}};
        constexpr int CH = PPT < 8 ? PPT : 8;
#pragma unroll
        for (int k0 = 0; k0 < PPT; k0 += CH) {
            int bb[CH];
            uint32_t pos[CH];
#pragma unroll
            for (int j = 0; j < CH; j++) bb[j] = v[k0 + j] == v[k0 + j] ? bin_of(v[k0 + j], cstar, inv_bw) : -1;
#pragma unroll
            for (int j = 0; j < CH; j++)
                if (bb[j] >= 0) pos[j] = atomicAdd(&S.hfill[bb[j]], 1u);
#pragma unroll
            for (int j = 0; j < CH; j++)
                if (bb[j] >= 0) {
                    sval[pos[j]] = v[k0 + j];
                    sums_add(tot, v[k0 + j], bb[j], cstar, fxs);
                }
        }
        const int cz[3] = {0, 0, 0};
        warp_partial(S, tot, cz, lane, warp);
    }
    __syncthreads();  // scatter and partials complete

    // ---- clip passes ----------------------------------------------------------
    // Warp 0 owns the kept set: it reduces the last pass's removals, selects the
    // median, evaluates Eq. 1-2's statistics and the next bounds (scalar FP64 on
    // lane 0; the FP64 pipe is narrow) and publishes them.  Every warp then
    // scans only the bins at the two ends of the kept range for the values the
    // new bounds remove.  Two barriers per pass.
    KeptSet K;
    K.lo = -INFINITY; K.hi = INFINITY; K.bl = 0; K.bh = MS_NB + 1;
    K.nbl = (int)S.hcnt[0]; K.nbh = (int)S.hcnt[MS_NB + 1];
    K.n = n0;
    // the running sums and statistics live in shared memory (lane 0 of warp 0
    // reads and writes them): registers are scarce at two 512-thread CTAs per SM
    float plo = 0.f, phi = 0.f;            // bounds published for the pending pass (warp 0)
    if (warp == 0) {
        int cz[3];
        double o1 = 0.0, o2 = 0.0;
        long long i1, i2;
        warp0_totals(S, lane, cz, &i1, &i2, &o1, &o2);
        if (lane == 0) { S.ks_i[0] = i1; S.ks_i[1] = i2; S.ks_o[0] = o1; S.ks_o[1] = o2; }
    }
    for (int it = 0;; it++) {
        if (warp == 0) {
            bool cont = true;
            if (it > 0) {  // removals of pass it-1
                int c[3];
                long long i1, i2;
                double o1 = 0.0, o2 = 0.0;
                warp0_totals(S, lane, c, &i1, &i2, &o1, &o2);
                // no value dropped: the set is stable (c >= n cannot happen: the
                // median lies inside [med - k sd, med + k sd])
                if (c[0] == 0 || c[0] >= K.n) {
                    cont = false;
                } else {
                    if (lane == 0) { S.ks_i[0] -= i1; S.ks_i[1] -= i2; S.ks_o[0] -= o1; S.ks_o[1] -= o2; }
                    K.bl = bin_of(plo, cstar, inv_bw); K.bh = bin_of(phi, cstar, inv_bw);
                    K.lo = plo; K.hi = phi;
                    K.nbl = c[1]; K.nbh = c[2];
                    K.n -= c[0];
                }
            }
            if (cont) {
                float mid[2];
                kept_middle(S, sval, K, mid, lane);
                if (lane == 0) {
                    double mu, sd;
                    kept_stats(KeptSums{S.ks_i[0], S.ks_i[1], S.ks_o[0], S.ks_o[1]}, K.n, cstar, unit, &mu, &sd);
                    S.st[0] = 0.5 * ((double)mid[0] + (double)mid[1]);
                    S.st[1] = mu;
                    S.st[2] = sd;
                }
                if (it == J.maxiters) {
                    cont = false;  // statistics of the set left after maxiters passes
                } else {
                    if (lane == 0) {
                        const double med = S.st[0], sd = S.st[2];
                        const double blo = __dsub_rn(med, __dmul_rn(J.nsigma, sd));
                        const double bhi = __dadd_rn(med, __dmul_rn(J.nsigma, sd));
                        plo = fmaxf(K.lo, __double2float_ru(blo));
                        phi = fminf(K.hi, __double2float_rd(bhi));
                    }
                    plo = __shfl_sync(0xffffffffu, plo, 0);
                    phi = __shfl_sync(0xffffffffu, phi, 0);
                    if (lane == 0) {
                        S.bc_f[0] = plo; S.bc_f[1] = phi; S.bc_f[2] = K.lo; S.bc_f[3] = K.hi;
                        S.bc_i[0] = K.bl; S.bc_i[1] = K.bh;
                    }
                }
            }
            if (lane == 0) S.bc_i[4] = cont;
        }
        __syncthreads();
        if (!S.bc_i[4]) break;
        const float nlo = S.bc_f[0], nhi = S.bc_f[1], klo = S.bc_f[2], khi = S.bc_f[3];
        const int kbl = S.bc_i[0], kbh = S.bc_i[1];
        const int nbl_bin = bin_of(nlo, cstar, inv_bw), nbh_bin = bin_of(nhi, cstar, inv_bw);
        // values removed by this pass lie in bins [bl, nbl_bin] and [nbh_bin, bh]
        Sums rem{0, 0, df{0.f, 0.f}, df{0.f, 0.f}};
        int c[3] = {0, 0, 0};  // removed, kept in new bin bl, kept in new bin bh
        {
            const int a0 = S.hstart[kbl], a1 = S.hstart[nbl_bin + 1];
            for (int k = a0 + (int)threadIdx.x; k < a1; k += MS_THREADS) {
                const float x = sval[k];
                if (!(x >= klo && x <= khi)) continue;
                if (x < nlo || x > nhi) { c[0]++; sums_add(rem, x, bin_of(x, cstar, inv_bw), cstar, fxs); }
                else if (k >= (int)S.hstart[nbl_bin]) c[1]++;
            }
            const int b0 = S.hstart[max(nbh_bin, nbl_bin + 1)], b1 = S.hstart[kbh + 1];
            for (int k = b0 + (int)threadIdx.x; k < b1; k += MS_THREADS) {
                const float x = sval[k];
                if (!(x >= klo && x <= khi)) continue;
                if (x < nlo || x > nhi) { c[0]++; sums_add(rem, x, bin_of(x, cstar, inv_bw), cstar, fxs); }
                else if (k < (int)S.hstart[nbh_bin + 1] && nbh_bin != nbl_bin) c[2]++;
            }
        }
        warp_partial(S, rem, c, lane, warp);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double med = S.st[0], mu = S.st[1], sd = S.st[2];
        double bk;
        switch (J.estimator) {
            case IPP_EST_MEDIAN: bk = med; break;
            case IPP_EST_MEAN: bk = mu; break;
            case IPP_EST_FACTORS: bk = J.mf * med - J.mnf * mu; break;
            default: bk = 2.5 * med - 1.5 * mu; break;
        }
        J.raw_bkg[mesh] = (float)bk;
        J.raw_rms[mesh] = (float)sd;
    }
}

// ---------------------------------------------------------------------------
// Invalid-mesh fill and median filter on the mesh grid.  An invalid node takes
// the median of the valid nodes in the smallest (2k+1)^2 neighbourhood holding
// any; each node then becomes the median of the in-bounds (filled) nodes of its
// fw x fh window.  One thread per node; the fill of an invalid neighbour is
// recomputed where needed (invalid meshes are rare).
constexpr int MF_THREADS = 256;

// median (Eq. 1) of src over the valid nodes of a window, by rank counting
__device__ float window_median_valid(const float* src, const float* raw_rms, int nx, int p0, int p1, int q0,
                                     int q1, int cnt) {
    const int k0 = (cnt - 1) / 2, k1 = cnt / 2;
    float a = 0.f, b = 0.f;
    for (int p = p0; p <= p1; p++)
        for (int q = q0; q <= q1; q++) {
            const int id = p * nx + q;
            if (raw_rms[id] < 0.f) continue;
            const float x = src[id];
            int less = 0, leq = 0;
            for (int pp = p0; pp <= p1; pp++)
                for (int qq = q0; qq <= q1; qq++) {
                    const int j = pp * nx + qq;
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

// filled value of node (p, q) of src; false when the grid has no valid node
__device__ bool filled_value(const float* src, const float* raw_rms, int nx, int ny, int p, int q, float* out) {
    const int id = p * nx + q;
    if (raw_rms[id] >= 0.f) { *out = src[id]; return true; }
    for (int k = 1; k <= max(nx, ny); k++) {
        const int p0 = max(p - k, 0), p1 = min(p + k, ny - 1), q0 = max(q - k, 0), q1 = min(q + k, nx - 1);
        int cnt = 0;
        for (int pp = p0; pp <= p1; pp++)
            for (int qq = q0; qq <= q1; qq++) cnt += raw_rms[pp * nx + qq] >= 0.f;
        if (cnt > 0) {
            *out = window_median_valid(src, raw_rms, nx, p0, p1, q0, q1, cnt);
            return true;
        }
    }
    return false;
}

__global__ void __launch_bounds__(MF_THREADS) k_mesh_filter(const float* raw_bkg, const float* raw_rms, int nx,
                                                            int ny, int fw, int fh, float* out_bkg,
                                                            float* out_rms, int32_t* status_dev) {
    const int id = blockIdx.x * MF_THREADS + threadIdx.x;
    if (id >= nx * ny) return;
    const int p = id / nx, q = id - p * nx;
    const int hw = fw / 2, hh = fh / 2;
    const int p0 = max(p - hh, 0), p1 = min(p + hh, ny - 1), q0 = max(q - hw, 0), q1 = min(q + hw, nx - 1);
    float wb[49], wr[49];
    int n = 0;
    bool ok = true;
    for (int pp = p0; pp <= p1; pp++)
        for (int qq = q0; qq <= q1; qq++) {
            float b, r;
            ok &= filled_value(raw_bkg, raw_rms, nx, ny, pp, qq, &b);
            ok &= filled_value(raw_rms, raw_rms, nx, ny, pp, qq, &r);
            // insertion into the two sorted windows
            int i = n - 1;
            while (i >= 0 && wb[i] > b) { wb[i + 1] = wb[i]; i--; }
            wb[i + 1] = b;
            i = n - 1;
            while (i >= 0 && wr[i] > r) { wr[i + 1] = wr[i]; i--; }
            wr[i + 1] = r;
            n++;
        }
    if (!ok) {  // no valid mesh anywhere
        out_bkg[id] = 0.f;
        out_rms[id] = 0.f;
        if (id == 0 && status_dev) *status_dev = IPP_ERR_NO_VALID_MESH;
        return;
    }
    out_bkg[id] = (float)(0.5 * ((double)wb[(n - 1) / 2] + (double)wb[n / 2]));
    out_rms[id] = (float)(0.5 * ((double)wr[(n - 1) / 2] + (double)wr[n / 2]));
    if (id == 0 && status_dev) *status_dev = IPP_OK;
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

static int mesh_ppt(int area) {
    if (area <= MS_THREADS * 8) return 8;
    if (area <= MS_THREADS * 16) return 16;
    if (area <= MS_THREADS * 32) return 32;
    return 0;
}

size_t ipp_mesh_smem_bytes(int ppt) { return sizeof(MeshShared) + (size_t)ppt * MS_THREADS * sizeof(float); }

int ipp_launch_mesh_stats(const MeshJob& J, cudaStream_t s) {
    int ppt = mesh_ppt(J.mesh_w * J.mesh_h);
    if (!ppt) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "mesh area %d > %d", J.mesh_w * J.mesh_h, MS_THREADS * 32);
    size_t sm = ipp_mesh_smem_bytes(ppt);
    int nm = J.nx * J.ny;
    switch (ppt) {
        case 8:
            cudaFuncSetAttribute(k_mesh_stats<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_mesh_stats<8><<<nm, MS_THREADS, sm, s>>>(J);
            break;
        case 16:
            cudaFuncSetAttribute(k_mesh_stats<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_mesh_stats<16><<<nm, MS_THREADS, sm, s>>>(J);
            break;
        default:
            cudaFuncSetAttribute(k_mesh_stats<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_mesh_stats<32><<<nm, MS_THREADS, sm, s>>>(J);
            break;
    }
    return ipp_check_launch("k_mesh_stats");
}

int ipp_launch_mesh_filter(const float* raw_bkg, const float* raw_rms, float* fill_bkg, float* fill_rms,
                           int nx, int ny, int fw, int fh, float* out_bkg, float* out_rms,
                           int32_t* status_dev, cudaStream_t s) {
    (void)fill_bkg;
    (void)fill_rms;  // the fill is computed on the fly
    const int nn = nx * ny;
    k_mesh_filter<<<(nn + MF_THREADS - 1) / MF_THREADS, MF_THREADS, 0, s>>>(raw_bkg, raw_rms, nx, ny, fw, fh,
                                                                            out_bkg, out_rms, status_dev);
    return ipp_check_launch("k_mesh_filter");
}

int ipp_launch_bg_subtract(const SubJob& J, cudaStream_t s) {
    if (J.mesh_w < 4 || J.mesh_h < 4)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "mesh size below 4 px");
    dim3 grid((unsigned)cdiv(J.W, BG_TW), (unsigned)cdiv(J.H, BG_TH));
    k_bg_subtract<<<grid, BG_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_bg_subtract");
}
