// bg.cu -- mesh background (Sec. 2.2.2, Eqs. 1-4): per-mesh iterative sigma
// clip, invalid-mesh fill and mesh median filter, interpolation + subtraction.
//
// k_mesh_stats: one CTA (512 threads) per mesh.  The mesh is read once from HBM
// into registers; a histogram over a window around the mean turns it into a
// bin-sorted copy in shared memory, with per-bin sums.  Every clip pass then
// costs O(pixels in the two boundary bins + the median bin) instead of O(mesh):
// counts and sums of full bins come from prefix sums, the exact order
// statistics from the small slice that holds them.  Sums are kept in
// double-float (pairs of FP32) and combined in FP64, so the clip bounds agree
// with an FP64 evaluation to ~1e-12 relative.
#include <math.h>

#include "jobs.cuh"

namespace ipp {

constexpr int MS_THREADS = 512;
constexpr int MS_WARPS = MS_THREADS / kWarp;
constexpr int MS_NB = 1024;          // window bins 1..MS_NB; 0 = below, MS_NB+1 = above
constexpr int MS_NBT = MS_NB + 2;
constexpr int MS_RANKCOUNT_MAX = 1024;  // slices up to this size: select by rank counting


struct MeshShared {
    uint32_t hcnt[MS_NBT];
    uint32_t hstart[MS_NBT + 1];
    uint32_t hfill[MS_NBT];
    float d1[MS_NBT];  // per-bin sum of (v - bin centre); reused as radix scratch
    float d2[MS_NBT];  // per-bin sum of (v - bin centre)^2
    float2 P1[MS_NBT + 1];  // double-float prefix over window bins of sum(v - c*)
    float2 P2[MS_NBT + 1];  // ... of sum (v - c*)^2
    // reductions / broadcasts
    float2 red1[MS_WARPS], red2[MS_WARPS];
    int redi[MS_WARPS * 2];
    float redf[MS_WARPS * 2];
    double bc_d[8];
    int bc_i[8];
    float bc_f[4];
    uint32_t bc_u[4];
};

// Bin of a value: monotone in v (FP subtraction and the power-of-two scaling
// are monotone), clamped to [0, MS_NB+1].
__device__ __forceinline__ int bin_of(float v, float cstar, float inv_bw) {
    float t = floorf((v - cstar) * inv_bw);
    t = fmaxf(fminf(t, (float)(MS_NB / 2)), (float)(-MS_NB / 2 - 1));
    return (int)t + MS_NB / 2 + 1;
}

__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return df{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

// Block-wide sum of (count, df, df); result valid in all threads.
struct Red3 {
    int n;
    double s1, s2;
};
__device__ Red3 block_red3(MeshShared& S, int n, df a, df b) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    n = warp_sum_i(n);
    a = warp_sum_df(a);
    b = warp_sum_df(b);
    __syncthreads();
    if (lane == 0) {
        S.redi[warp] = n;
        S.red1[warp] = make_float2(a.hi, a.lo);
        S.red2[warp] = make_float2(b.hi, b.lo);
    }
    __syncthreads();
    if (warp == 0) {
        int nn = lane < MS_WARPS ? S.redi[lane] : 0;
        df aa = lane < MS_WARPS ? df{S.red1[lane].x, S.red1[lane].y} : df{0.f, 0.f};
        df bb = lane < MS_WARPS ? df{S.red2[lane].x, S.red2[lane].y} : df{0.f, 0.f};
        nn = warp_sum_i(nn);
        aa = warp_sum_df(aa);
        bb = warp_sum_df(bb);
        if (lane == 0) {
            S.bc_i[0] = nn;
            S.bc_d[0] = df_to_d(aa);
            S.bc_d[1] = df_to_d(bb);
        }
    }
    __syncthreads();
    Red3 r{S.bc_i[0], S.bc_d[0], S.bc_d[1]};
    __syncthreads();
    return r;
}

// Count, sum(v - c*) and sum((v - c*)^2) of the set {v : lo <= v <= hi} (kept
// set of a clip pass), plus the kept counts of its two boundary bins.
struct SetStats {
    int n;
    double a1, a2;  // relative to c*
    int bl, bh;     // boundary bins
    int nbl, nbh;   // kept elements in slices bl and bh (nbh = 0 when bl == bh)
};

__device__ SetStats set_stats(MeshShared& S, const float* sval, float lo, float hi, float cstar,
                              float inv_bw) {
    SetStats st;
    st.bl = (lo == -INFINITY) ? 0 : bin_of(lo, cstar, inv_bw);
    st.bh = (hi == INFINITY) ? MS_NB + 1 : bin_of(hi, cstar, inv_bw);
    // explicit part: the boundary slices
    int cl = 0, ch = 0;
    df e1{0.f, 0.f}, e2{0.f, 0.f};
    {
        int s0 = S.hstart[st.bl], s1 = S.hstart[st.bl + 1];
        for (int k = s0 + (int)threadIdx.x; k < s1; k += MS_THREADS) {
            float v = sval[k];
            if (v >= lo && v <= hi) {
                cl++;
                df d = two_sum(v, -cstar);
                e1 = df_add(e1, d);
                df q = sq_exact(d.hi);
                q = df_add_f(q, __fmul_rn(2.0f * d.hi, d.lo));
                e2 = df_add(e2, q);
            }
        }
    }
    if (st.bh != st.bl) {
        int s0 = S.hstart[st.bh], s1 = S.hstart[st.bh + 1];
        for (int k = s0 + (int)threadIdx.x; k < s1; k += MS_THREADS) {
            float v = sval[k];
            if (v >= lo && v <= hi) {
                ch++;
                df d = two_sum(v, -cstar);
                e1 = df_add(e1, d);
                df q = sq_exact(d.hi);
                q = df_add_f(q, __fmul_rn(2.0f * d.hi, d.lo));
                e2 = df_add(e2, q);
            }
        }
    }
    // counts of the two boundary slices, reduced separately
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int a = warp_sum_i(cl), b = warp_sum_i(ch);
        if (lane == 0) { S.redi[warp] = a; S.redi[MS_WARPS + warp] = b; }
        __syncthreads();
        if (threadIdx.x == 0) {
            int x = 0, y = 0;
            for (int w = 0; w < MS_WARPS; w++) { x += S.redi[w]; y += S.redi[MS_WARPS + w]; }
            S.bc_i[4] = x;
            S.bc_i[5] = y;
        }
        __syncthreads();
        st.nbl = S.bc_i[4];
        st.nbh = S.bc_i[5];
        __syncthreads();
    }
    Red3 r = block_red3(S, cl + ch, e1, e2);
    st.n = r.n;
    st.a1 = r.s1;
    st.a2 = r.s2;
    if (st.bh > st.bl + 1) {  // full window bins strictly between
        st.n += (int)(S.hstart[st.bh] - S.hstart[st.bl + 1]);
        float2 p1h = S.P1[st.bh], p1l = S.P1[st.bl + 1];
        float2 p2h = S.P2[st.bh], p2l = S.P2[st.bl + 1];
        st.a1 += ((double)p1h.x + (double)p1h.y) - ((double)p1l.x + (double)p1l.y);
        st.a2 += ((double)p2h.x + (double)p2h.y) - ((double)p2l.x + (double)p2l.y);
    }
    return st;
}

// r-th smallest (0-based) of the elements of slice [s0, s1) that lie in
// [lo, hi].  Rank counting with ties broken by position for small slices; an
// 11-bit radix select over the order-preserving keys otherwise.
__device__ float select_in_slice(MeshShared& S, const float* sval, int s0, int s1, float lo,
                                 float hi, int r) {
    const int m = s1 - s0;
    if (m <= MS_RANKCOUNT_MAX) {
        for (int k = s0 + (int)threadIdx.x; k < s1; k += MS_THREADS) {
            float v = sval[k];
            if (!(v >= lo && v <= hi)) continue;
            int rank = 0;
            for (int u = s0; u < s1; u++) {
                float x = sval[u];
                bool in = (x >= lo && x <= hi);
                rank += in && (x < v || (x == v && u < k));
            }
            if (rank == r) S.bc_f[0] = v;
        }
        __syncthreads();
        float res = S.bc_f[0];
        __syncthreads();
        return res;
    }
    // radix select, 3 passes of 11/11/10 bits over keys
    uint32_t* hist = reinterpret_cast<uint32_t*>(S.d1);  // 2 * MS_NBT >= 2048 words
    uint32_t prefix = 0, pmask = 0;
    int rr = r;
    const int shifts[3] = {21, 10, 0};
    const int widths[3] = {11, 11, 10};
    for (int pass = 0; pass < 3; pass++) {
        const int sh = shifts[pass], nb = 1 << widths[pass];
        for (int k = threadIdx.x; k < nb; k += MS_THREADS) hist[k] = 0;
        __syncthreads();
        for (int k = s0 + (int)threadIdx.x; k < s1; k += MS_THREADS) {
            float v = sval[k];
            if (!(v >= lo && v <= hi)) continue;
            uint32_t key = fkey(v);
            if ((key & pmask) != prefix) continue;
            atomicAdd(&hist[(key >> sh) & (nb - 1)], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0, d = 0;
            for (d = 0; d < nb; d++) {
                int c = (int)hist[d];
                if (rr < acc + c) break;
                acc += c;
            }
            if (d >= nb) d = nb - 1;  // unreachable for a valid rank
            S.bc_u[0] = (uint32_t)d;
            S.bc_i[6] = rr - acc;
        }
        __syncthreads();
        prefix |= S.bc_u[0] << sh;
        pmask |= (uint32_t)(nb - 1) << sh;
        rr = S.bc_i[6];
        __syncthreads();
    }
    return fkey_inv(prefix);
}

// Median (Eq. 1) of the kept set described by st.
__device__ double set_median(MeshShared& S, const float* sval, const SetStats& st, float lo,
                             float hi) {
    const int full = (st.bh > st.bl + 1) ? (int)(S.hstart[st.bh] - S.hstart[st.bl + 1]) : 0;
    float vals[2];
    int ks[2] = {(st.n - 1) / 2, st.n / 2};
    for (int q = 0; q < 2; q++) {
        if (q == 1 && ks[1] == ks[0]) { vals[1] = vals[0]; break; }
        int k = ks[q];
        int s0, s1, r;
        if (k < st.nbl) {
            s0 = S.hstart[st.bl]; s1 = S.hstart[st.bl + 1]; r = k;
        } else if (k - st.nbl < full) {
            int kk = k - st.nbl;
            // bin b in (bl, bh) with hstart[b] - base <= kk < hstart[b+1] - base
            uint32_t base = S.hstart[st.bl + 1];
            int a = st.bl + 1, b = st.bh - 1;
            while (a < b) {
                int mid = (a + b + 1) >> 1;
                if ((int)(S.hstart[mid] - base) <= kk) a = mid; else b = mid - 1;
            }
            s0 = S.hstart[a]; s1 = S.hstart[a + 1]; r = kk - (int)(S.hstart[a] - base);
        } else {
            s0 = S.hstart[st.bh]; s1 = S.hstart[st.bh + 1]; r = k - st.nbl - full;
        }
        vals[q] = select_in_slice(S, sval, s0, s1, lo, hi, r);
    }
    return 0.5 * ((double)vals[0] + (double)vals[1]);
}

template <int PPT>
__global__ void __launch_bounds__(MS_THREADS, 2) k_mesh_stats(MeshJob J) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MeshShared& S = *reinterpret_cast<MeshShared*>(smem_raw);
    float* sval = reinterpret_cast<float*>(smem_raw + sizeof(MeshShared));

    const int mesh = blockIdx.x;
    const int mx = mesh % J.nx, my = mesh / J.nx;
    const int64_t x0 = (int64_t)mx * J.mesh_w, y0 = (int64_t)my * J.mesh_h;
    const int we = (int)min((int64_t)J.mesh_w, J.W - x0);
    const int he = (int)min((int64_t)J.mesh_h, J.H - y0);
    const int slots = J.mesh_w * J.mesh_h;

    // ---- load (one HBM read of the mesh), exact double-float sums ----------
    float v[PPT];
    int n_loc = 0;
    df s1{0.f, 0.f}, s2{0.f, 0.f};
    float vmin = INFINITY, vmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        int e = threadIdx.x + k * MS_THREADS;
        float x = __int_as_float(0x7fc00000);  // NaN = not usable
        if (e < slots) {
            int r = e / J.mesh_w, c = e - r * J.mesh_w;
            if (r < he && c < we) {
                int64_t yy = y0 + r, xx = x0 + c;
                if (J.dtype == IPP_F32) {
                    x = __ldg(reinterpret_cast<const float*>(J.img) + yy * J.pitch + xx);
                } else {
                    float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(J.img) + yy * J.pitch + xx);
                    float b = J.bias_map ? __ldg(J.bias_map + yy * J.W + xx) : J.bias;
                    x = (raw - b) * __ldg(J.inv_flat + yy * J.W + xx);
                }
                if (J.mask && J.mask[yy * J.W + xx]) x = __int_as_float(0x7fc00000);
                if (!isfinite(x)) x = __int_as_float(0x7fc00000);
            }
        }
        v[k] = x;
        if (x == x) {
            n_loc++;
            s1 = df_add_f(s1, x);
            s2 = df_add(s2, sq_exact(x));
            vmin = fminf(vmin, x);
            vmax = fmaxf(vmax, x);
        }
    }
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
            vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        }
        if (lane == 0) { S.redf[warp] = vmin; S.redf[MS_WARPS + warp] = vmax; }
    }
    Red3 tot = block_red3(S, n_loc, s1, s2);  // contains __syncthreads
    if (threadIdx.x == 0) {
        float a = INFINITY, b = -INFINITY;
        for (int w = 0; w < MS_WARPS; w++) { a = fminf(a, S.redf[w]); b = fmaxf(b, S.redf[MS_WARPS + w]); }
        S.bc_f[1] = a;
        S.bc_f[2] = b;
    }
    __syncthreads();
    vmin = S.bc_f[1];
    vmax = S.bc_f[2];
    const int n0 = tot.n;

    if (n0 < J.min_valid || n0 == 0) {
        if (threadIdx.x == 0) { J.raw_bkg[mesh] = 0.f; J.raw_rms[mesh] = -1.f; }
        return;
    }
    if (vmin == vmax) {  // constant mesh: every statistic is that value, sigma 0
        if (threadIdx.x == 0) {
            double c = (double)vmin, bk;
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

    // ---- histogram window ---------------------------------------------------
    // Width NB*bw in [10 sigma0, 20 sigma0), bw a power of two, centre c* a
    // multiple of bw near the mean; refined once around the median bin when
    // outliers made it coarse.
    float cstar, bw, inv_bw;
    {
        double mu0 = tot.s1 / n0;
        double var0 = tot.s2 / n0 - mu0 * mu0;
        double sd0 = sqrt(fmax(var0, 0.0));
        double span = fmax(10.0 * sd0, (double)(vmax - vmin) * 1e-6);
        span = fmax(span, fabs(mu0) * 1e-6 + 1e-30);
        int e = (int)ceil(log2(span / MS_NB));
        e = max(min(e, 100), -120);
        bw = ldexpf(1.0f, e);
        inv_bw = ldexpf(1.0f, -e);
        cstar = rintf((float)mu0 * inv_bw) * bw;
    }
    for (int round = 0; round < 2; round++) {
        for (int k = threadIdx.x; k < MS_NBT; k += MS_THREADS) S.hcnt[k] = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PPT; k++)
            if (v[k] == v[k]) atomicAdd(&S.hcnt[bin_of(v[k], cstar, inv_bw)], 1u);
        __syncthreads();
        if (round == 1) break;
        // robust width from the 16th / 84th percentile bins; refine when the
        // median bin is crowded and the window could be at least 8x finer
        if (threadIdx.x == 0) {
            int acc = 0, b16 = -1, b50 = -1, b84 = -1;
            int k16 = (int)(0.1587 * n0), k50 = n0 / 2, k84 = (int)(0.8413 * n0);
            for (int b = 0; b < MS_NBT; b++) {
                acc += (int)S.hcnt[b];
                if (b16 < 0 && acc > k16) b16 = b;
                if (b50 < 0 && acc > k50) b50 = b;
                if (b84 < 0 && acc > k84) b84 = b;
            }
            int refine = 0;
            float nc = cstar, nbw = bw, ninv = inv_bw;
            if (b50 >= 1 && b50 <= MS_NB && S.hcnt[b50] > 96 && b16 >= 1 && b84 <= MS_NB) {
                double sr = 0.5 * (double)(b84 - b16 + 1) * bw;
                double span = 10.0 * sr;
                int e = (int)ceil(log2(span / MS_NB));
                float cand = ldexpf(1.0f, e);
                if (cand * 8.0f <= bw) {
                    refine = 1;
                    nbw = cand;
                    ninv = ldexpf(1.0f, -e);
                    float centre = cstar + ((float)(b50 - MS_NB / 2 - 1) + 0.5f) * bw;
                    nc = rintf(centre * ninv) * nbw;
                }
            }
            S.bc_i[7] = refine;
            S.bc_f[0] = nc;
            S.bc_f[1] = nbw;
            S.bc_f[2] = ninv;
        }
        __syncthreads();
        int refine = S.bc_i[7];
        cstar = S.bc_f[0];
        bw = S.bc_f[1];
        inv_bw = S.bc_f[2];
        __syncthreads();
        if (!refine) break;
    }

    // ---- exclusive scan of the bin counts (one warp) -------------------------
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        constexpr int PER = (MS_NBT + 31) / 32;
        int b0 = lane * PER, acc = 0;
        for (int b = b0; b < min(b0 + PER, MS_NBT); b++) acc += (int)S.hcnt[b];
        int inc = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        int run = inc - acc;
        for (int b = b0; b < min(b0 + PER, MS_NBT); b++) {
            S.hstart[b] = (uint32_t)run;
            run += (int)S.hcnt[b];
        }
        if (lane == 31) S.hstart[MS_NBT] = (uint32_t)inc;
    }
    for (int k = threadIdx.x; k < MS_NBT; k += MS_THREADS) {
        S.hfill[k] = 0;
        S.d1[k] = 0.f;
        S.d2[k] = 0.f;
    }
    __syncthreads();

    // ---- scatter into bin order; per-bin sums of offsets from the bin centre
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        float x = v[k];
        if (x == x) {
            int b = bin_of(x, cstar, inv_bw);
            uint32_t pos = S.hstart[b] + atomicAdd(&S.hfill[b], 1u);
            sval[pos] = x;
            if (b >= 1 && b <= MS_NB) {
                float cb = cstar + ((float)(b - MS_NB / 2 - 1) + 0.5f) * bw;
                float d = x - cb;
                atomicAdd(&S.d1[b], d);
                atomicAdd(&S.d2[b], d * d);
            }
        }
    }
    __syncthreads();

    // ---- prefix over window bins of sums relative to c* (one warp, df) ------
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        constexpr int PER = (MS_NB + 31) / 32;
        int b0 = 1 + lane * PER;
        df t1{0.f, 0.f}, t2{0.f, 0.f};
        for (int b = b0; b < min(b0 + PER, MS_NB + 1); b++) {
            float nb = (float)S.hcnt[b];
            float ob = ((float)(b - MS_NB / 2 - 1) + 0.5f) * bw;  // exact: bw power of 2
            float d1b = S.d1[b], d2b = S.d2[b];
            df x1 = df_add_f(two_prod(nb, ob), d1b);
            df x2 = two_prod(nb, ob * ob);
            x2 = df_add(x2, two_prod(2.0f * ob, d1b));
            x2 = df_add_f(x2, d2b);
            t1 = df_add(t1, x1);
            t2 = df_add(t2, x2);
        }
        df i1 = t1, i2 = t2;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            df u1{__shfl_up_sync(0xffffffffu, i1.hi, o), __shfl_up_sync(0xffffffffu, i1.lo, o)};
            df u2{__shfl_up_sync(0xffffffffu, i2.hi, o), __shfl_up_sync(0xffffffffu, i2.lo, o)};
            if (lane >= o) { i1 = df_add(i1, u1); i2 = df_add(i2, u2); }
        }
        df r1 = df_add(i1, df_neg(t1)), r2 = df_add(i2, df_neg(t2));  // exclusive
        for (int b = b0; b < min(b0 + PER, MS_NB + 1); b++) {
            S.P1[b] = make_float2(r1.hi, r1.lo);
            S.P2[b] = make_float2(r2.hi, r2.lo);
            float nb = (float)S.hcnt[b];
            float ob = ((float)(b - MS_NB / 2 - 1) + 0.5f) * bw;
            float d1b = S.d1[b], d2b = S.d2[b];
            df x1 = df_add_f(two_prod(nb, ob), d1b);
            df x2 = two_prod(nb, ob * ob);
            x2 = df_add(x2, two_prod(2.0f * ob, d1b));
            x2 = df_add_f(x2, d2b);
            r1 = df_add(r1, x1);
            r2 = df_add(r2, x2);
        }
        if (lane == 31) {
            S.P1[MS_NB + 1] = make_float2(r1.hi, r1.lo);
            S.P2[MS_NB + 1] = make_float2(r2.hi, r2.lo);
        }
    }
    __syncthreads();

    // ---- clip passes -----------------------------------------------------------
    float lo = -INFINITY, hi = INFINITY;
    SetStats st = set_stats(S, sval, lo, hi, cstar, inv_bw);
    double med = 0.0, mu = 0.0, sd = 0.0;
    bool done = false;
    for (int it = 0; it < J.maxiters; it++) {
        mu = (double)cstar + st.a1 / st.n;
        double m1 = st.a1 / st.n;
        sd = sqrt(fmax(st.a2 / st.n - m1 * m1, 0.0));
        med = set_median(S, sval, st, lo, hi);
        double blo = med - J.nsigma * sd, bhi = med + J.nsigma * sd;
        float nlo = fmaxf(lo, __double2float_ru(blo));
        float nhi = fminf(hi, __double2float_rd(bhi));
        SetStats st2 = set_stats(S, sval, nlo, nhi, cstar, inv_bw);
        if (st2.n == st.n || st2.n == 0) { done = true; break; }
        lo = nlo;
        hi = nhi;
        st = st2;
    }
    if (!done) {
        mu = (double)cstar + st.a1 / st.n;
        double m1 = st.a1 / st.n;
        sd = sqrt(fmax(st.a2 / st.n - m1 * m1, 0.0));
        med = set_median(S, sval, st, lo, hi);
    }
    if (threadIdx.x == 0) {
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
// Invalid-mesh fill and median filter on the mesh grid (one CTA; the grid is
// small).  An invalid node takes the median of the valid nodes in the smallest
// (2k+1)^2 neighbourhood holding any; then each node becomes the median of the
// in-bounds nodes of its fw x fh window.
constexpr int MF_THREADS = 1024;

// median (Eq. 1) of the values of `src` at the valid nodes of a window, found
// by rank counting (windows are small)
__device__ float window_median(const float* src, const float* valid_rms, int nx, int ny, int p0,
                               int p1, int q0, int q1, int cnt) {
    int k0 = (cnt - 1) / 2, k1 = cnt / 2;
    float a = 0.f, b = 0.f;
    for (int p = p0; p <= p1; p++)
        for (int q = q0; q <= q1; q++) {
            int id = p * nx + q;
            if (valid_rms && valid_rms[id] < 0.f) continue;
            float x = src[id];
            int less = 0, leq = 0;
            for (int pp = p0; pp <= p1; pp++)
                for (int qq = q0; qq <= q1; qq++) {
                    int j = pp * nx + qq;
                    if (valid_rms && valid_rms[j] < 0.f) continue;
                    float y = src[j];
                    less += y < x;
                    leq += y <= x;
                }
            if (less <= k0 && k0 < leq) a = x;
            if (less <= k1 && k1 < leq) b = x;
        }
    return (float)(0.5 * ((double)a + (double)b));
}

__global__ void __launch_bounds__(MF_THREADS) k_mesh_fill_filter(
    const float* raw_bkg, const float* raw_rms, float* fill_bkg, float* fill_rms, int nx, int ny,
    int fw, int fh, float* out_bkg, float* out_rms, int32_t* status_dev) {
    __shared__ int nvalid;
    if (threadIdx.x == 0) nvalid = 0;
    __syncthreads();
    const int nn = nx * ny;
    int c = 0;
    for (int id = threadIdx.x; id < nn; id += MF_THREADS) c += raw_rms[id] >= 0.f;
    atomicAdd(&nvalid, c);
    __syncthreads();
    if (nvalid == 0) {
        for (int id = threadIdx.x; id < nn; id += MF_THREADS) { out_bkg[id] = 0.f; out_rms[id] = 0.f; }
        if (threadIdx.x == 0 && status_dev) *status_dev = IPP_ERR_NO_VALID_MESH;
        return;
    }
    for (int id = threadIdx.x; id < nn; id += MF_THREADS) {
        if (raw_rms[id] >= 0.f) {
            fill_bkg[id] = raw_bkg[id];
            fill_rms[id] = raw_rms[id];
            continue;
        }
        int p = id / nx, q = id - p * nx;
        for (int k = 1; k <= max(nx, ny); k++) {
            int p0 = max(p - k, 0), p1 = min(p + k, ny - 1), q0 = max(q - k, 0), q1 = min(q + k, nx - 1);
            int cnt = 0;
            for (int pp = p0; pp <= p1; pp++)
                for (int qq = q0; qq <= q1; qq++) cnt += raw_rms[pp * nx + qq] >= 0.f;
            if (cnt > 0) {
                fill_bkg[id] = window_median(raw_bkg, raw_rms, nx, ny, p0, p1, q0, q1, cnt);
                fill_rms[id] = window_median(raw_rms, raw_rms, nx, ny, p0, p1, q0, q1, cnt);
                break;
            }
        }
    }
    __syncthreads();  // fill_* written by this block are visible to it after the barrier
    const int hw = fw / 2, hh = fh / 2;
    for (int id = threadIdx.x; id < nn; id += MF_THREADS) {
        int p = id / nx, q = id - p * nx;
        int p0 = max(p - hh, 0), p1 = min(p + hh, ny - 1), q0 = max(q - hw, 0), q1 = min(q + hw, nx - 1);
        int cnt = (p1 - p0 + 1) * (q1 - q0 + 1);
        out_bkg[id] = window_median(fill_bkg, nullptr, nx, ny, p0, p1, q0, q1, cnt);
        out_rms[id] = window_median(fill_rms, nullptr, nx, ny, p0, p1, q0, q1, cnt);
    }
    if (threadIdx.x == 0 && status_dev) *status_dev = IPP_OK;
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
    const int qa = (int)floorf(((float)tx0 + 0.5f) / J.mesh_w - 0.5f) - 1;
    const int qbase = max(qa, 0);
    // per-row vertical interpolation of the needed node columns
    const float ref = J.mesh[0];
    for (int t = threadIdx.x; t < BG_TH * BG_NQ; t += BG_THREADS) {
        int r = t / BG_NQ, qq = t - r * BG_NQ;
        int q = min(qbase + qq, J.nx - 1);
        float vy = ((float)(ty0 + r) + 0.5f) / J.mesh_h - 0.5f;
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
        float u = ((float)(xc + c) + 0.5f) / J.mesh_w - 0.5f;
        float qf = floorf(u);
        keys_weights(u - qf, wx[c]);
        int q0 = (int)qf;
#pragma unroll
        for (int b = 0; b < 4; b++) qi[c][b] = min(clampi(q0 - 1 + b, 0, J.nx - 1) - qbase, BG_NQ - 1);
    }
    const bool vec = (J.dtype == IPP_F32) && (J.pitch % 4 == 0) && (J.sub_pitch % 4 == 0) &&
                     (((uintptr_t)J.img & 15) == 0) && (((uintptr_t)J.sub & 15) == 0) &&
                     (!J.bkg_map || ((uintptr_t)J.bkg_map & 15) == 0) && (xc + 4 <= J.W);
    for (int r = warp; r < BG_TH; r += BG_THREADS / 32) {
        int64_t y = ty0 + r;
        if (y >= J.H) break;
        float f[4], B[4];
        if (vec) {
            float4 t4 = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(J.img) + y * J.pitch + xc));
            f[0] = t4.x; f[1] = t4.y; f[2] = t4.z; f[3] = t4.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++) f[c] = (xc + c < J.W) ? load_pix(J, y, xc + c) : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float acc = 0.f;
#pragma unroll
            for (int b = 0; b < 4; b++) acc = fmaf(wx[c][b], cv[r][qi[c][b]], acc);
            B[c] = ref + acc;
        }
        if (vec) {
            float4 o = make_float4(f[0] - B[0], f[1] - B[1], f[2] - B[2], f[3] - B[3]);
            *reinterpret_cast<float4*>(J.sub + y * J.sub_pitch + xc) = o;
            if (J.bkg_map) *reinterpret_cast<float4*>(J.bkg_map + y * J.sub_pitch + xc) = make_float4(B[0], B[1], B[2], B[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (xc + c < J.W) {
                    J.sub[y * J.sub_pitch + xc + c] = f[c] - B[c];
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
    k_mesh_fill_filter<<<1, MF_THREADS, 0, s>>>(raw_bkg, raw_rms, fill_bkg, fill_rms, nx, ny, fw, fh,
                                                 out_bkg, out_rms, status_dev);
    return ipp_check_launch("k_mesh_fill_filter");
}

int ipp_launch_bg_subtract(const SubJob& J, cudaStream_t s) {
    if (J.mesh_w < 4 || J.mesh_h < 4)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "mesh size below 4 px");
    dim3 grid((unsigned)cdiv(J.W, BG_TW), (unsigned)cdiv(J.H, BG_TH));
    k_bg_subtract<<<grid, BG_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_bg_subtract");
}
