// deblend.cu -- deblending of the detected candidates (Sec. 2.2.5: multi-level
// thresholds between a candidate's threshold and its peak, a tree of the
// sub-components found at each level, traversed bottom-up and pruned on
// intensity).  Reading of the steps:
//   levels  L_i = T (P/T)^(i/N), i = 1..N-1, T / P = lowest / highest pixel of
//           the candidate, in FP64 (for N a power of two by square roots and
//           products, bit-identical to the oracle); T <= 0 or P <= T keeps the
//           candidate whole;
//   tree    the nodes of level i are the 8-connected components of the
//           candidate's pixels above L_i; level 0 is the whole candidate;
//   objects from the top level down, a node with two or more children holding
//           at least mincont of the candidate's flux passes on their objects,
//           a node with one such child passes on its objects when it has two
//           or more, and any other node is one object (its pixels its core);
//   pixels  a pixel outside every core goes to the object whose elliptical
//           Gaussian (core flux, barycentre and second moments) is largest
//           there, compared as log-likelihoods, ties to the object whose core
//           starts first;
//   numbers candidate by candidate, within one by the raster order of each
//           object's first pixel.
//
// One block per candidate.  The candidate's pixels are gathered in raster
// order into slots [base, base + n) of frame-sized workspace arrays, so every
// per-pixel and per-node array of the candidate lives in its own slot range
// (L1/L2 resident for all but the largest candidates).  Each level runs a
// lock-free union-find over the pixels above it (links always point to a lower
// slot, so a component's root is its first pixel in raster order), numbers the
// roots in slot order and applies the pruning rule node by node; only the core
// owner of each pixel is carried from level to level.  Candidates with a single
// local maximum cannot split (every level set holds one component) and skip the
// tree, as do levels whose pixel set equals the one above.
#include <math.h>

#include <algorithm>

#include "jobs.cuh"

namespace ipp {

constexpr int DB_T = 128;
constexpr int DB_W = DB_T / 32;

constexpr int DB_MAXLV = 256;  // nthresh limit of the C ABI

struct DbShared {  // block helpers below work for blocks of 1 .. DB_W warps
    double red_d[DB_W];
    int red_i[DB_W];
    int scan_w[DB_W];
    // level thresholds as floats: for a float v, (double)v > L exactly when
    // v > L rounded toward -infinity to float (no float lies in between)
    float lev[DB_MAXLV];
};

__device__ __forceinline__ double db_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Keyed sums of a warp: every lane with key >= 0 adds v into slot `key`; the
// lanes sharing a key are summed with shuffles first, so each distinct key of
// the warp costs one update (an atomic when several warps share the slots,
// a plain store of the complete sum when `alone`).  All 32 lanes must call.
template <int NV>
__device__ __forceinline__ void db_keyed_add(double* const (&acc)[NV], int key, const double (&v)[NV], bool alone) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(FULL, key >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(FULL, key, leader);
        const bool mine = key == k;
#pragma unroll
        for (int a = 0; a < NV; a++) {
            const double sv = db_warp_sum(mine ? v[a] : 0.0);
            if (lane == leader) {
                if (alone) acc[a][k] = sv;
                else atomicAdd(acc[a] + k, sv);
            }
        }
        pending &= ~__ballot_sync(FULL, mine);
    }
}

// Keyed sums of one warp in double-float (an unevaluated pair of floats, sums
// by Knuth's TwoSum): the node fluxes of a small candidate on the FP32 pipe.
// Every lane with key >= 0 adds v into slot `key`; the leader of each distinct
// key stores hi + lo as a double.  All 32 lanes must call.
__device__ __forceinline__ void db_keyed_store_df(double* acc, int key, float v) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(FULL, key >= 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int k = __shfl_sync(FULL, key, leader);
        const bool mine = key == k;
        float hi = mine ? v : 0.f, lo = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(FULL, hi, o), l2 = __shfl_xor_sync(FULL, lo, o);
            const float sum = __fadd_rn(hi, h2);
            const float bb = __fsub_rn(sum, hi);
            const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(h2, bb));
            const float low = __fadd_rn(__fadd_rn(lo, l2), err);
            hi = __fadd_rn(sum, low);
            lo = __fsub_rn(low, __fsub_rn(hi, sum));
        }
        if (lane == leader) acc[k] = (double)hi + (double)lo;
        pending &= ~__ballot_sync(FULL, mine);
    }
}

// Block reductions (every thread gets the result).
__device__ __forceinline__ double db_sum(double v, DbShared& S) {
    v = db_warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_d[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < DB_W; w++) t += w < (int)(blockDim.x >> 5) ? S.red_d[w] : 0.0;
    return t;
}
__device__ __forceinline__ double db_min(double v, DbShared& S) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_d[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = S.red_d[0];
#pragma unroll
    for (int w = 1; w < DB_W; w++) t = w < (int)(blockDim.x >> 5) ? fmin(t, S.red_d[w]) : t;
    return t;
}
__device__ __forceinline__ double db_max(double v, DbShared& S) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_d[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = S.red_d[0];
#pragma unroll
    for (int w = 1; w < DB_W; w++) t = w < (int)(blockDim.x >> 5) ? fmax(t, S.red_d[w]) : t;
    return t;
}
__device__ __forceinline__ int db_sum_i(int v, DbShared& S) {
    v = __reduce_add_sync(0xffffffffu, v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_i[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int w = 0; w < DB_W; w++) t += w < (int)(blockDim.x >> 5) ? S.red_i[w] : 0;
    return t;
}

// Exclusive prefix of `flag` over the block in thread order; `total` = count.
__device__ __forceinline__ int db_scan(bool flag, int& total, DbShared& S) {
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int pre = __popc(b & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) S.scan_w[w] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < DB_W; k++) {
        const int v = k < (int)(blockDim.x >> 5) ? S.scan_w[k] : 0;
        off += k < w ? v : 0;
        tot += v;
    }
    total = tot;
    return off + pre;
}

// Lock-free union-find on slot indices; a link always points to the lower slot.
__device__ __forceinline__ int db_find(volatile int* par, int t) {
    while (true) {
        const int p = par[t];
        if (p == t) return t;
        const int gp = par[p];
        if (gp != p) par[t] = gp;  // path halving (gp is an ancestor of t)
        t = p;
    }
}
__device__ __forceinline__ void db_union(int* par, int a, int b) {
    volatile int* vp = par;
    while (true) {
        a = db_find(vp, a);
        b = db_find(vp, b);
        if (a == b) return;
        if (a < b) { const int x = a; a = b; b = x; }
        const int old = atomicCAS(par + a, a, b);
        if (old == a) return;
        a = old;
    }
}

enum { DB_PASS_ALL = 0, DB_PASS_ONE = 1, DB_OBJECT = 2 };

// Level lv of N between T and P, rounded toward -infinity to float (for a float
// v, (double)v > L exactly when v > that float).  For N a power of two the
// ratio's N-th root is taken by log2(N) correctly rounded square roots and
// L_lv = L_{lv-1} r from L_0 = T, in that order -- IEEE basic operations only,
// so the oracle's identical sequence gives bit-identical levels; other N use pow.
__device__ __forceinline__ void db_levels(double T, double Pk, int N, float* lev, int rank, int nt) {
    if ((N & (N - 1)) == 0) {
        if (rank == 0) {
            double r = Pk / T;
            for (int m = N; m > 1; m >>= 1) r = sqrt(r);
            double L = T;
            lev[0] = -INFINITY;
            for (int lv = 1; lv < N; lv++) {
                L = L * r;
                lev[lv] = __double2float_rd(L);
            }
        }
    } else {
        for (int lv = rank; lv < N; lv += nt)
            lev[lv] = lv > 0 ? __double2float_rd(T * pow(Pk / T, (double)lv / (double)N)) : -INFINITY;
    }
}

// ---------------------------------------------------------------------------
// Candidates of at most 32 pixels (most of a frame's): one warp each, one
// pixel a lane, no block barrier.  A level's components are closures of the
// lanes' 8-neighbour bit masks within the ballot of the pixels above the level;
// a component's root is its lowest slot, as in the union-find of larger ones.
constexpr int DB_SMALL = 32;

struct DbWarp {
    int P[32], qi[32], qj[32];
    float F[32];
    unsigned adj[32];
    float lev[DB_MAXLV];
    int rootN[32], nobN[32], rootC[32], nobC[32], nsig[32], tot[32], sgc[32], dec[32];
    double fluxN[32], fluxC[32];
    double o[6][32];
    int ofirst[32], orank[32];
};

__device__ __noinline__ void db_small(const DeblendJob& J, int64_t c, DbWarp& Wp) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int W = (int)J.W;
    const int lab = (int)(c + 1);
    const int b0 = J.ws.base[c];
    const int x0 = __ldg(J.xmin + c), y0 = __ldg(J.ymin + c);
    const int bw = __ldg(J.xmax + c) - x0 + 1, bh = __ldg(J.ymax + c) - y0 + 1;
    const int64_t nb = (int64_t)bw * bh;
    const int64_t room = (int64_t)W * J.H - b0;
    const int cap = b0 < 0 ? 0 : (int)min((int64_t)min(max(__ldg(J.area + c), 0), DB_SMALL), max(room, (int64_t)0));
    // gather in raster order
    int n = 0;
    for (int64_t t0 = 0; t0 < nb && n < cap; t0 += 32) {
        const int64_t t = t0 + lane;
        bool in = false;
        int i = 0, j = 0;
        if (t < nb) {
            i = y0 + (int)(t / bw);
            j = x0 + (int)(t - (t / bw) * bw);
            in = __ldg(J.labels + (int64_t)i * W + j) == lab;
        }
        const unsigned bal = __ballot_sync(FULL, in);
        const int pos = __popc(bal & ((1u << lane) - 1u));
        if (in && n + pos < cap) {
            Wp.P[n + pos] = i * W + j; Wp.qi[n + pos] = i; Wp.qj[n + pos] = j;
            Wp.F[n + pos] = __ldg(J.sub + (int64_t)i * J.pitch + j);
        }
        n += __popc(bal);
    }
    n = min(n, cap);
    __syncwarp();
    const bool have = lane < n;
    const int q = have ? Wp.P[lane] : 0, qi = have ? Wp.qi[lane] : 0, qj = have ? Wp.qj[lane] : 0;
    const float f = have ? Wp.F[lane] : 0.f;
    unsigned adj = 0u;
    for (int u = 0; u < n; u++)
        if (u != lane && abs(Wp.qi[u] - qi) <= 1 && abs(Wp.qj[u] - qj) <= 1) adj |= 1u << u;
    Wp.adj[lane] = have ? adj : 0u;
    // lowest / highest pixel, flux, local maxima
    float lo = have ? f : INFINITY, hi = have ? f : -INFINITY;
    double fc = have ? (double)f : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
        fc += __shfl_xor_sync(FULL, fc, o);
    }
    __syncwarp();
    bool top = have;
    for (unsigned r = adj; r; r &= r - 1u) top = top && !(Wp.F[__ffs(r) - 1] > f);
    const int nmax = __popc(__ballot_sync(FULL, top));
    const double T = (double)lo, Pk = (double)hi, cut = J.mincont * fc;
    int no = n > 0 ? 1 : 0, asg = 0;
    if (T > 0.0 && Pk > T && nmax > 1 && n >= 2) {
        db_levels(T, Pk, J.nthresh, Wp.lev, lane, 32);
        __syncwarp();
        int core = -1, nidN = -1, mN = 0;
        unsigned prevA = 0u;
        bool firstlv = true;
        for (int lv = J.nthresh - 1; lv >= 0; lv--) {
            const bool above = have && f > Wp.lev[lv];
            const unsigned A = __ballot_sync(FULL, above);
            if (!firstlv && A == prevA) continue;  // same pixel set as the level above
            firstlv = false;
            prevA = A;
            unsigned m = above ? 1u << lane : 0u;
            while (m) {  // closure of the lane's component within A
                unsigned m2 = m;
                for (unsigned r = m; r; r &= r - 1u) m2 |= Wp.adj[__ffs(r) - 1];
                m2 &= A;
                if (m2 == m) break;
                m = m2;
            }
            const int root = above ? __ffs(m) - 1 : -1;
            const unsigned R = __ballot_sync(FULL, above && root == lane);
            const int nid = above ? __popc(R & ((1u << root) - 1u)) : -1;
            const int mC = __popc(R);
            if (lane < mC) { Wp.nsig[lane] = 0; Wp.tot[lane] = 0; Wp.sgc[lane] = -1; }
            if (above && root == lane) Wp.rootC[nid] = lane;
            __syncwarp();
            db_keyed_store_df(Wp.fluxC, above ? nid : -1, f);
            {
                const int src = lane < mN ? Wp.rootN[lane] : 0;
                const int g = __shfl_sync(FULL, nid, src);
                if (lane < mN && Wp.fluxN[lane] >= cut) {
                    atomicAdd(&Wp.nsig[g], 1);
                    atomicAdd(&Wp.tot[g], Wp.nobN[lane]);
                    Wp.sgc[g] = lane;
                }
            }
            __syncwarp();
            if (lane < mC) {
                const int k = Wp.nsig[lane];
                const int d = k >= 2 ? DB_PASS_ALL : (k == 1 && Wp.nobN[Wp.sgc[lane]] >= 2 ? DB_PASS_ONE : DB_OBJECT);
                Wp.dec[lane] = d;
                Wp.nobC[lane] = d == DB_PASS_ALL ? Wp.tot[lane] : (d == DB_PASS_ONE ? Wp.nobN[Wp.sgc[lane]] : 1);
            }
            __syncwarp();
            if (above) {
                if (Wp.dec[nid] == DB_OBJECT) core = Wp.rootC[nid];
                else if (nidN >= 0 && !(Wp.fluxN[nidN] >= cut)) core = -1;
            }
            __syncwarp();
            if (lane < mC) { Wp.rootN[lane] = Wp.rootC[lane]; Wp.fluxN[lane] = Wp.fluxC[lane]; Wp.nobN[lane] = Wp.nobC[lane]; }
            nidN = nid;
            mN = mC;
            __syncwarp();
        }
        no = Wp.nobN[0];
        if (no >= 2) {
            const unsigned CORES = __reduce_or_sync(FULL, core >= 0 ? 1u << core : 0u);
            no = __popc(CORES);
            const int ec = core >= 0 ? __popc(CORES & ((1u << core) - 1u)) : -1;
            if (lane < no) Wp.ofirst[lane] = INT32_MAX;
            __syncwarp();
            const double x = (double)qj, y = (double)qi;
            {
                double* const acc[3] = {Wp.o[0], Wp.o[1], Wp.o[2]};
                const double v[3] = {(double)f, (double)f * x, (double)f * y};
                db_keyed_add<3>(acc, ec, v, true);
            }
            __syncwarp();
            if (lane < no) { Wp.o[1][lane] /= Wp.o[0][lane]; Wp.o[2][lane] /= Wp.o[0][lane]; }
            __syncwarp();
            {
                const double dx = ec >= 0 ? x - Wp.o[1][ec] : 0.0, dy = ec >= 0 ? y - Wp.o[2][ec] : 0.0;
                double* const acc[3] = {Wp.o[3], Wp.o[4], Wp.o[5]};
                const double v[3] = {(double)f * dx * dx, (double)f * dy * dy, (double)f * dx * dy};
                db_keyed_add<3>(acc, ec, v, true);
            }
            __syncwarp();
            if (lane < no) {
                const double F0 = Wp.o[0][lane];
                double x2 = Wp.o[3][lane] / F0, y2 = Wp.o[4][lane] / F0, xy = Wp.o[5][lane] / F0;
                if (x2 * y2 - xy * xy < 1.0 / 144.0) { x2 += 1.0 / 12.0; y2 += 1.0 / 12.0; }
                const double det = x2 * y2 - xy * xy;
                Wp.o[3][lane] = y2 / det;
                Wp.o[4][lane] = x2 / det;
                Wp.o[5][lane] = -2.0 * xy / det;
                Wp.o[0][lane] = log(F0) - 0.5 * log(det);  // log of F / sqrt(det)
            }
            __syncwarp();
            int best = ec;
            if (have && ec < 0) {
                double bv = -INFINITY;
                best = 0;
                for (int e = 0; e < no; e++) {  // largest log-likelihood
                    const double dx = x - Wp.o[1][e], dy = y - Wp.o[2][e];
                    const double r2 = Wp.o[3][e] * dx * dx + Wp.o[5][e] * dx * dy + Wp.o[4][e] * dy * dy;
                    const double v = Wp.o[0][e] - 0.5 * r2;
                    if (v > bv) { bv = v; best = e; }
                }
            }
            if (have) atomicMin(&Wp.ofirst[best], lane);
            __syncwarp();
            if (lane < no) {
                int r = 0;
                for (int e2 = 0; e2 < no; e2++) r += Wp.ofirst[e2] < Wp.ofirst[lane];
                Wp.orank[lane] = r;
            }
            __syncwarp();
            asg = have ? Wp.orank[best] : 0;
        } else {
            no = 1;
        }
    }
    if (have) { J.ws.pidx[b0 + lane] = q; J.ws.asg[b0 + lane] = asg; }
    if (lane == 0) { J.ws.nobj[c] = no; J.ws.npx[c] = n; }
    __syncwarp();
}


// The block path keeps a candidate of at most DB_SMEM_PX pixels in shared
// memory (the same buffer the warps used for the small candidates), larger
// ones in their workspace slots.
constexpr int DB_SMEM_PX = 384;  // even: the double views of int pairs stay 8-byte aligned

struct DbArrays {
    int* nb4;  // shared-memory path: slots of the 4 backward neighbours (-1: none)
    int *P, *par, *core, *asg, *nidA, *nidB, *rootA, *rootB, *nobA, *nobB, *nsig, *tot, *sgc, *dec;
    float* F;
    double *fluxA, *fluxB, *o2, *o3, *o4, *o5;
};

__device__ __forceinline__ DbArrays db_arrays(const DeblendJob& J, int b0, bool sm, char* buf) {
    DbArrays a;
    if (sm) {
        double* d = (double*)buf;
        a.fluxA = d; a.fluxB = d + DB_SMEM_PX;
        int* q = (int*)(d + 2 * DB_SMEM_PX);
        int** ints[] = {&a.P, &a.par, &a.core, &a.asg, &a.nidA, &a.nidB, &a.rootA, &a.rootB, &a.nobA, &a.nobB,
                        &a.nsig, &a.tot, &a.sgc, &a.dec};
        for (int k = 0; k < 14; k++) *ints[k] = q + k * DB_SMEM_PX;
        a.F = (float*)(q + 14 * DB_SMEM_PX);
        a.nb4 = q + 15 * DB_SMEM_PX;
        // object moments reuse arrays the tree no longer needs once it is built:
        // the neighbour slots and the node ids / roots of the two levels
        a.o2 = (double*)(q + 15 * DB_SMEM_PX);
        a.o3 = (double*)(q + 17 * DB_SMEM_PX);
        a.o4 = (double*)(q + 4 * DB_SMEM_PX);
        a.o5 = (double*)(q + 6 * DB_SMEM_PX);
    } else {
        a.nb4 = nullptr;
        a.P = J.ws.pidx + b0; a.par = J.ws.par + b0; a.core = J.ws.core + b0; a.asg = J.ws.asg + b0;
        a.nidA = J.ws.nidA + b0; a.nidB = J.ws.nidB + b0; a.rootA = J.ws.rootA + b0; a.rootB = J.ws.rootB + b0;
        a.nobA = J.ws.nobA + b0; a.nobB = J.ws.nobB + b0; a.nsig = J.ws.nsig + b0; a.tot = J.ws.tot + b0;
        a.sgc = J.ws.sgc + b0; a.dec = J.ws.dec + b0; a.F = J.ws.f + b0;
        a.fluxA = J.ws.fluxA + b0; a.fluxB = J.ws.fluxB + b0; a.o2 = J.ws.o2 + b0; a.o3 = J.ws.o3 + b0;
        a.o4 = J.ws.o4 + b0; a.o5 = J.ws.o5 + b0;
    }
    return a;
}
constexpr size_t DB_SMEM_BYTES = (size_t)DB_SMEM_PX * (2 * 8 + 19 * 4);
constexpr size_t DB_DYN_BYTES = DB_SMEM_BYTES > sizeof(DbWarp) * DB_W ? DB_SMEM_BYTES : sizeof(DbWarp) * DB_W;


__global__ void __launch_bounds__(DB_T) k_deblend(DeblendJob J) {
    const int NT = blockDim.x;
    __shared__ DbShared S;
    extern __shared__ __align__(16) char buf[];  // DB_DYN_BYTES
    const int64_t nsrc = min((int64_t)__ldg(J.n_src_dev), (int64_t)J.max_src);
    const int W = (int)J.W, H = (int)J.H;
    const double NEG = -INFINITY;
    // candidates above DB_SMALL pixels: a block each
    for (int64_t c = blockIdx.x; c < nsrc; c += gridDim.x) {
        const int area_c = __ldg(J.area + c);
        if (area_c <= DB_SMALL) continue;
        const int lab = (int)(c + 1);
        const int b0 = J.ws.base[c];
        const bool sm = area_c <= DB_SMEM_PX;
        const DbArrays A = db_arrays(J, b0, sm, buf);
        int* P = A.P;
        float* F = A.F;
        int* par = A.par;
        int* core = A.core;
        int* asg = A.asg;
        // ---- gather the candidate's pixels in raster order ------------------
        const int x0 = __ldg(J.xmin + c), y0 = __ldg(J.ymin + c);
        const int bw = __ldg(J.xmax + c) - x0 + 1, bh = __ldg(J.ymax + c) - y0 + 1;
        const int64_t nb = (int64_t)bw * bh;
        // this candidate's slots: [b0, b0 + area), inside the W*H slot arrays
        const int64_t room = (int64_t)W * H - b0;
        const int cap = b0 < 0 ? 0 : (int)min((int64_t)max(__ldg(J.area + c), 0), max(room, (int64_t)0));
        int n = 0;
        for (int64_t t0 = 0; t0 < nb; t0 += NT) {
            const int64_t t = t0 + threadIdx.x;
            bool in = false;
            int i = 0, j = 0;
            if (t < nb) {
                i = y0 + (int)(t / bw);
                j = x0 + (int)(t - (t / bw) * bw);
                in = __ldg(J.labels + (int64_t)i * W + j) == lab;
            }
            int tot;
            const int pos = db_scan(in, tot, S);
            if (in && n + pos < cap) {  // at most `area` pixels: the slots of this candidate
                const int s = n + pos;
                P[s] = i * W + j;
                F[s] = __ldg(J.sub + (int64_t)i * J.pitch + j);
                J.ws.map[(int64_t)i * W + j] = s;
            }
            n += tot;
        }
        n = min(n, cap);
        __syncthreads();
        // ---- levels, flux, local maxima -------------------------------------
        double lo = INFINITY, hi = NEG, fc = 0.0;
        int nmax = 0;
        for (int t = threadIdx.x; t < n; t += NT) {
            const double v = (double)F[t];
            lo = fmin(lo, v);
            hi = fmax(hi, v);
            fc += v;
            const int q = P[t], qi = q / W, qj = q - qi * W;
            bool top = true;
            for (int di = -1; di <= 1; di++)
                for (int dj = -1; dj <= 1; dj++) {
                    const int ni = qi + di, nj = qj + dj;
                    if ((di | dj) == 0 || (unsigned)ni >= (unsigned)H || (unsigned)nj >= (unsigned)W) continue;
                    if (__ldg(J.labels + (int64_t)ni * W + nj) != lab) continue;
                    const int u = J.ws.map[(int64_t)ni * W + nj];
                    if ((unsigned)u >= (unsigned)n || P[u] != ni * W + nj) continue;  // not gathered
                    if (F[u] > F[t]) top = false;
                }
            nmax += top;
        }
        const double T = db_min(lo, S), Pk = db_max(hi, S), Fc = db_sum(fc, S);
        nmax = db_sum_i(nmax, S);
        const double cut = J.mincont * Fc;
        int no = 1;
        bool whole = !(T > 0.0 && Pk > T) || nmax <= 1 || n < 2;
        if (!whole) {
            if (A.nb4) {  // backward neighbours of each pixel, looked up once
                for (int t = threadIdx.x; t < n; t += NT) {
                    const int q = P[t], qi = q / W, qj = q - qi * W;
                    const int nbr[4][2] = {{0, -1}, {-1, -1}, {-1, 0}, {-1, 1}};
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const int ni = qi + nbr[k][0], nj = qj + nbr[k][1];
                        int u = -1;
                        if ((unsigned)ni < (unsigned)H && (unsigned)nj < (unsigned)W &&
                            __ldg(J.labels + (int64_t)ni * W + nj) == lab) {
                            u = J.ws.map[(int64_t)ni * W + nj];
                            if ((unsigned)u >= (unsigned)n || P[u] != ni * W + nj) u = -1;  // not gathered
                        }
                        A.nb4[4 * t + k] = u;
                    }
                }
            }
            db_levels(T, Pk, J.nthresh, S.lev, threadIdx.x, NT);
            for (int t = threadIdx.x; t < n; t += NT) core[t] = -1;
            int* nidC = A.nidA;
            int* nidN = A.nidB;
            int* rootC = A.rootA;
            int* rootN = A.rootB;
            int* nobC = A.nobA;
            int* nobN = A.nobB;
            double* fluxC = A.fluxA;
            double* fluxN = A.fluxB;
            int* nsig = A.nsig;
            int* tot = A.tot;
            int* sgc = A.sgc;
            int* dec = A.dec;
            int mN = 0, prev = -1;
            for (int t = threadIdx.x; t < n; t += NT) nidN[t] = -1;
            for (int lv = J.nthresh - 1; lv >= 0; lv--) {
                __syncthreads();  // S.lev written
                const float L = S.lev[lv];
                int cnt = 0;
                for (int t = threadIdx.x; t < n; t += NT) cnt += F[t] > L;
                cnt = db_sum_i(cnt, S);
                if (cnt == prev) continue;  // same pixel set as the level above: same tree
                prev = cnt;
                // union-find over the pixels above L (backward neighbours suffice)
                for (int t = threadIdx.x; t < n; t += NT) par[t] = F[t] > L ? t : -1;
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += NT) {
                    if (!(F[t] > L)) continue;
                    if (A.nb4) {
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            const int u = A.nb4[4 * t + k];
                            if (u >= 0 && F[u] > L) db_union(par, t, u);
                        }
                        continue;
                    }
                    const int q = P[t], qi = q / W, qj = q - qi * W;
                    const int nbr[4][2] = {{0, -1}, {-1, -1}, {-1, 0}, {-1, 1}};
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        const int ni = qi + nbr[k][0], nj = qj + nbr[k][1];
                        if ((unsigned)ni >= (unsigned)H || (unsigned)nj >= (unsigned)W) continue;
                        if (__ldg(J.labels + (int64_t)ni * W + nj) != lab) continue;
                        const int u = J.ws.map[(int64_t)ni * W + nj];
                        if ((unsigned)u >= (unsigned)n || P[u] != ni * W + nj) continue;  // not gathered
                        if (F[u] > L) db_union(par, t, u);
                    }
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += NT)
                    if (par[t] >= 0) par[t] = db_find(par, t);
                __syncthreads();
                // node ids: roots in slot order
                int m = 0;
                for (int t0 = 0; t0 < n; t0 += NT) {
                    const int t = t0 + threadIdx.x;
                    const bool root = t < n && par[t] == t;
                    int cntr;
                    const int pos = db_scan(root, cntr, S);
                    if (root) { nidC[t] = m + pos; rootC[m + pos] = t; }
                    m += cntr;
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += NT) {
                    const int p = par[t];
                    if (p < 0) nidC[t] = -1;
                    else if (p != t) nidC[t] = nidC[p];
                }
                for (int g = threadIdx.x; g < m; g += NT) { fluxC[g] = 0.0; nsig[g] = 0; tot[g] = 0; sgc[g] = -1; }
                __syncthreads();
                for (int t0 = 0; t0 < n; t0 += NT) {  // whole warps: keyed sums
                    const int t = t0 + threadIdx.x;
                    double* const acc[1] = {fluxC};
                    const double v[1] = {t < n ? (double)F[t] : 0.0};
                    db_keyed_add<1>(acc, t < n ? nidC[t] : -1, v, false);
                }
                // children: the nodes of the level processed before this one
                for (int h = threadIdx.x; h < mN; h += NT) {
                    if (!(fluxN[h] >= cut)) continue;
                    const int g = nidC[rootN[h]];
                    atomicAdd(nsig + g, 1);
                    atomicAdd(tot + g, nobN[h]);
                    sgc[g] = h;
                }
                __syncthreads();
                for (int g = threadIdx.x; g < m; g += NT) {
                    const int k = nsig[g];
                    const int d = k >= 2 ? DB_PASS_ALL : (k == 1 && nobN[sgc[g]] >= 2 ? DB_PASS_ONE : DB_OBJECT);
                    dec[g] = d;
                    nobC[g] = d == DB_PASS_ALL ? tot[g] : (d == DB_PASS_ONE ? nobN[sgc[g]] : 1);
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += NT) {
                    const int g = nidC[t];
                    if (g < 0) continue;
                    if (dec[g] == DB_OBJECT) {
                        core[t] = rootC[g];
                    } else {
                        const int h = nidN[t];
                        if (h >= 0 && !(fluxN[h] >= cut)) core[t] = -1;
                    }
                }
                __syncthreads();
                // roll the level
                { int* x = nidC; nidC = nidN; nidN = x; }
                { int* x = rootC; rootC = rootN; rootN = x; }
                { int* x = nobC; nobC = nobN; nobN = x; }
                { double* x = fluxC; fluxC = fluxN; fluxN = x; }
                mN = m;
            }
            // level 0 is one node (the whole candidate), now in the N arrays
            no = nobN[0];
            whole = no <= 1;
            if (!whole) {
                // objects: distinct core owners, numbered in slot order of their root
                int* oid = A.nsig;    // per slot: object of the root at this slot
                int* ofirst = A.tot;  // per object: first slot of its pixels
                int* otmp = A.sgc;    // per slot: provisional object
                int* orank = A.dec;   // per object: rank by first pixel
                double* o0 = A.fluxA;
                double* o1 = A.fluxB;
                double* o2 = A.o2;
                double* o3 = A.o3;
                double* o4 = A.o4;
                double* o5 = A.o5;
                for (int t = threadIdx.x; t < n; t += NT) oid[t] = 0;
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += NT)
                    if (core[t] >= 0) oid[core[t]] = 1;
                __syncthreads();
                int ne = 0;
                for (int t0 = 0; t0 < n; t0 += NT) {
                    const int t = t0 + threadIdx.x;
                    const bool isr = t < n && oid[t] == 1;
                    int cntr;
                    const int pos = db_scan(isr, cntr, S);
                    __syncthreads();
                    if (isr) oid[t] = 2 + ne + pos;  // 2 + object index (0, 1 are flags)
                    ne += cntr;
                }
                no = ne;
                for (int e = threadIdx.x; e < no; e += NT) {
                    o0[e] = 0.0; o1[e] = 0.0; o2[e] = 0.0; o3[e] = 0.0; o4[e] = 0.0; o5[e] = 0.0;
                    ofirst[e] = INT32_MAX;
                }
                __syncthreads();
                // core flux and barycentre
                for (int t0 = 0; t0 < n; t0 += NT) {
                    const int t = t0 + threadIdx.x;
                    const int e = t < n && core[t] >= 0 ? oid[core[t]] - 2 : -1;
                    const double v = e >= 0 ? (double)F[t] : 0.0;
                    const int q = e >= 0 ? P[t] : 0;
                    double* const acc[3] = {o0, o1, o2};
                    const double vv[3] = {v, v * (double)(q % W), v * (double)(q / W)};
                    db_keyed_add<3>(acc, e, vv, false);
                }
                __syncthreads();
                for (int e = threadIdx.x; e < no; e += NT) { o1[e] /= o0[e]; o2[e] /= o0[e]; }
                __syncthreads();
                for (int t0 = 0; t0 < n; t0 += NT) {
                    const int t = t0 + threadIdx.x;
                    const int e = t < n && core[t] >= 0 ? oid[core[t]] - 2 : -1;
                    const double v = e >= 0 ? (double)F[t] : 0.0;
                    const int q = e >= 0 ? P[t] : 0;
                    const double dx = e >= 0 ? (double)(q % W) - o1[e] : 0.0, dy = e >= 0 ? (double)(q / W) - o2[e] : 0.0;
                    double* const acc[3] = {o3, o4, o5};
                    const double vv[3] = {v * dx * dx, v * dy * dy, v * dx * dy};
                    db_keyed_add<3>(acc, e, vv, false);
                }
                __syncthreads();
                // the elliptical Gaussian of each core: o0 <- F / sqrt(det),
                // o3, o4, o5 <- r^2 coefficients of dx^2, dy^2, dx dy
                for (int e = threadIdx.x; e < no; e += NT) {
                    double x2 = o3[e] / o0[e], y2 = o4[e] / o0[e], xy = o5[e] / o0[e];
                    if (x2 * y2 - xy * xy < 1.0 / 144.0) { x2 += 1.0 / 12.0; y2 += 1.0 / 12.0; }
                    const double det = x2 * y2 - xy * xy;
                    o3[e] = y2 / det;
                    o4[e] = x2 / det;
                    o5[e] = -2.0 * xy / det;
                    o0[e] = log(o0[e]) - 0.5 * log(det);  // log of F / sqrt(det)
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += NT) {
                    int best;
                    if (core[t] >= 0) {
                        best = oid[core[t]] - 2;
                    } else {
                        const int q = P[t];
                        const double x = (double)(q % W), y = (double)(q / W);
                        double bv = -INFINITY;
                        best = 0;
                        for (int e = 0; e < no; e++) {  // largest log-likelihood
                            const double dx = x - o1[e], dy = y - o2[e];
                            const double r2 = o3[e] * dx * dx + o5[e] * dx * dy + o4[e] * dy * dy;
                            const double v = o0[e] - 0.5 * r2;
                            if (v > bv) { bv = v; best = e; }
                        }
                    }
                    otmp[t] = best;
                    atomicMin(ofirst + best, t);
                }
                __syncthreads();
                for (int e = threadIdx.x; e < no; e += NT) {
                    int r = 0;
                    for (int e2 = 0; e2 < no; e2++) r += ofirst[e2] < ofirst[e];
                    orank[e] = r;
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += NT) asg[t] = orank[otmp[t]];
            }
        }
        if (whole) {
            no = n > 0 ? 1 : 0;  // an empty candidate yields no object
            for (int t = threadIdx.x; t < n; t += NT) asg[t] = 0;
        }
        if (sm) {  // the write pass reads pixel indices and objects from the slots
            __syncthreads();
            for (int t = threadIdx.x; t < n; t += NT) { J.ws.pidx[b0 + t] = P[t]; J.ws.asg[b0 + t] = asg[t]; }
        }
        if (threadIdx.x == 0) { J.ws.nobj[c] = no; J.ws.npx[c] = n; }
        __syncthreads();
    }
    // then the candidates of at most DB_SMALL pixels, a warp each (blocks that
    // met no large candidate start on them at once)
    DbWarp* WS = reinterpret_cast<DbWarp*>(buf);
    const int64_t nw = (int64_t)gridDim.x * (NT >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (NT >> 5) + (threadIdx.x >> 5); c < nsrc; c += nw)
        if (__ldg(J.area + c) <= DB_SMALL) db_small(J, c, WS[threadIdx.x >> 5]);
}

// Exclusive scan of per-candidate counts in one block; total to *total.
__global__ void __launch_bounds__(1024) k_deblend_scan(const int32_t* n_src_dev, int32_t max_src, const int32_t* v,
                                                        int32_t* out, int32_t* total) {
    __shared__ int wsum[32];
    const int n = min(__ldg(n_src_dev), max_src);
    const int per = (n + 1023) / 1024;
    const int s0 = threadIdx.x * per, s1 = min(n, s0 + per);
    int acc = 0;
    for (int s = s0; s < s1; s++) acc += v[s];
    // block exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int z = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z;
    }
    __syncthreads();
    int run = x - acc + (w > 0 ? wsum[w - 1] : 0);
    for (int s = s0; s < s1; s++) { out[s] = run; run += v[s]; }
    if (threadIdx.x == 1023) *total = run;
}

__global__ void __launch_bounds__(DB_T) k_deblend_write(DeblendJob J) {
    const int64_t nsrc = min((int64_t)__ldg(J.n_src_dev), (int64_t)J.max_src);
    for (int64_t c = blockIdx.x; c < nsrc; c += gridDim.x) {
        const int b0 = J.ws.base[c], n = J.ws.npx[c], o = J.ws.offs[c];
        for (int t = threadIdx.x; t < n; t += DB_T) J.out[J.ws.pidx[b0 + t]] = o + J.ws.asg[b0 + t] + 1;
    }
}

}  // namespace ipp

using namespace ipp;

static int db_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 132;
}

int ipp_launch_deblend(const DeblendJob& J, cudaStream_t s) {
    if (cudaMemsetAsync(J.out, 0, sizeof(int32_t) * (size_t)(J.W * J.H), s) != cudaSuccess)
        return ipp_check_launch("deblend memset");
    if (J.max_src <= 0) {
        cudaMemsetAsync(J.n_out_dev, 0, sizeof(int32_t), s);
        return ipp_check_launch("deblend memset");
    }
    k_deblend_scan<<<1, 1024, 0, s>>>(J.n_src_dev, J.max_src, J.area, J.ws.base, J.ws.counters);
    if (int e = ipp_check_launch("k_deblend_scan")) return e;
    cudaFuncSetAttribute(k_deblend, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DB_DYN_BYTES);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_deblend, DB_T, DB_DYN_BYTES) != cudaSuccess || per < 1)
        per = 1;
    k_deblend<<<db_sms() * per, DB_T, DB_DYN_BYTES, s>>>(J);
    if (int e = ipp_check_launch("k_deblend")) return e;
    k_deblend_scan<<<1, 1024, 0, s>>>(J.n_src_dev, J.max_src, J.ws.nobj, J.ws.offs, J.n_out_dev);
    if (int e = ipp_check_launch("k_deblend_scan")) return e;
    k_deblend_write<<<db_sms() * 8, DB_T, 0, s>>>(J);
    return ipp_check_launch("k_deblend_write");
}

// Carve the deblending workspace (256-byte aligned pieces); returns its size.
size_t ipp_deblend_ws_carve(int64_t W, int64_t H, int32_t max_src, void* ws, DeblendWs* out) {
    const size_t npx = (size_t)W * (size_t)H, nc = (size_t)(max_src > 0 ? max_src : 0) + 1;
    size_t off = 0;
    char* b = (char*)ws;
    auto take = [&](size_t bytes) -> void* {
        void* p = b ? (void*)(b + off) : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    DeblendWs w;
    w.base = (int32_t*)take(nc * 4);
    w.nobj = (int32_t*)take(nc * 4);
    w.npx = (int32_t*)take(nc * 4);
    w.offs = (int32_t*)take(nc * 4);
    w.counters = (int32_t*)take(64);
    w.map = (int32_t*)take(npx * 4);
    int32_t** ints[] = {&w.pidx, &w.par, &w.nidA, &w.nidB, &w.core, &w.asg, &w.rootA,
                        &w.rootB, &w.nobA, &w.nobB, &w.nsig, &w.tot, &w.sgc, &w.dec};
    for (int32_t** p : ints) *p = (int32_t*)take(npx * 4);
    w.f = (float*)take(npx * 4);
    double** dbl[] = {&w.fluxA, &w.fluxB, &w.o2, &w.o3, &w.o4, &w.o5};
    for (double** p : dbl) *p = (double*)take(npx * 8);
    if (out) *out = w;
    return off;
}
