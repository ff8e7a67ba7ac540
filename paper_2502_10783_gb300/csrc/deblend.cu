// deblend.cu -- deblending of the detected candidates (Sec. 2.2.4: multi-level
// thresholds between a candidate's threshold and its peak, a tree of the
// sub-components found at each level, traversed bottom-up and pruned on
// intensity).  Reading of the steps:
//   levels  L_i = T (P/T)^(i/N), i = 1..N-1, T / P = lowest / highest pixel of
//           the candidate, in FP64; T <= 0 or P <= T keeps the candidate whole;
//   tree    the nodes of level i are the 8-connected components of the
//           candidate's pixels above L_i; level 0 is the whole candidate;
//   objects from the top level down, a node with two or more children holding
//           at least mincont of the candidate's flux passes on their objects,
//           a node with one such child passes on its objects when it has two
//           or more, and any other node is one object (its pixels its core);
//   pixels  a pixel outside every core goes to the object whose elliptical
//           Gaussian (core flux, barycentre and second moments) is largest
//           there, ties to the object whose core starts first;
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

struct DbShared {
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

// Block reductions (every thread gets the result).
__device__ __forceinline__ double db_sum(double v, DbShared& S) {
    v = db_warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_d[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < DB_W; w++) t += S.red_d[w];
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
    for (int w = 1; w < DB_W; w++) t = fmin(t, S.red_d[w]);
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
    for (int w = 1; w < DB_W; w++) t = fmax(t, S.red_d[w]);
    return t;
}
__device__ __forceinline__ int db_sum_i(int v, DbShared& S) {
    v = __reduce_add_sync(0xffffffffu, v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) S.red_i[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int w = 0; w < DB_W; w++) t += S.red_i[w];
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
        off += k < w ? S.scan_w[k] : 0;
        tot += S.scan_w[k];
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

__global__ void __launch_bounds__(DB_T) k_deblend(DeblendJob J) {
    __shared__ DbShared S;
    const int64_t nsrc = min((int64_t)__ldg(J.n_src_dev), (int64_t)J.max_src);
    const int W = (int)J.W, H = (int)J.H;
    const double NEG = -INFINITY;
    for (int64_t c = blockIdx.x; c < nsrc; c += gridDim.x) {
        const int lab = (int)(c + 1);
        const int b0 = J.ws.base[c];
        int* P = J.ws.pidx + b0;
        float* F = J.ws.f + b0;
        int* par = J.ws.par + b0;
        int* core = J.ws.core + b0;
        int* asg = J.ws.asg + b0;
        // ---- gather the candidate's pixels in raster order ------------------
        const int x0 = __ldg(J.xmin + c), y0 = __ldg(J.ymin + c);
        const int bw = __ldg(J.xmax + c) - x0 + 1, bh = __ldg(J.ymax + c) - y0 + 1;
        const int64_t nb = (int64_t)bw * bh;
        // this candidate's slots: [b0, b0 + area), inside the W*H slot arrays
        const int64_t room = (int64_t)W * H - b0;
        const int cap = b0 < 0 ? 0 : (int)min((int64_t)max(__ldg(J.area + c), 0), max(room, (int64_t)0));
        int n = 0;
        for (int64_t t0 = 0; t0 < nb; t0 += DB_T) {
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
        for (int t = threadIdx.x; t < n; t += DB_T) {
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
            for (int lv = threadIdx.x; lv < J.nthresh; lv += DB_T)
                S.lev[lv] = lv > 0 ? __double2float_rd(T * pow(Pk / T, (double)lv / (double)J.nthresh)) : -INFINITY;
            for (int t = threadIdx.x; t < n; t += DB_T) core[t] = -1;
            int* nidC = J.ws.nidA + b0;
            int* nidN = J.ws.nidB + b0;
            int* rootC = J.ws.rootA + b0;
            int* rootN = J.ws.rootB + b0;
            int* nobC = J.ws.nobA + b0;
            int* nobN = J.ws.nobB + b0;
            double* fluxC = J.ws.fluxA + b0;
            double* fluxN = J.ws.fluxB + b0;
            int* nsig = J.ws.nsig + b0;
            int* tot = J.ws.tot + b0;
            int* sgc = J.ws.sgc + b0;
            int* dec = J.ws.dec + b0;
            int mN = 0, prev = -1;
            for (int t = threadIdx.x; t < n; t += DB_T) nidN[t] = -1;
            for (int lv = J.nthresh - 1; lv >= 0; lv--) {
                __syncthreads();  // S.lev written
                const float L = S.lev[lv];
                int cnt = 0;
                for (int t = threadIdx.x; t < n; t += DB_T) cnt += F[t] > L;
                cnt = db_sum_i(cnt, S);
                if (cnt == prev) continue;  // same pixel set as the level above: same tree
                prev = cnt;
                // union-find over the pixels above L (backward neighbours suffice)
                for (int t = threadIdx.x; t < n; t += DB_T) par[t] = F[t] > L ? t : -1;
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T) {
                    if (!(F[t] > L)) continue;
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
                for (int t = threadIdx.x; t < n; t += DB_T)
                    if (par[t] >= 0) par[t] = db_find(par, t);
                __syncthreads();
                // node ids: roots in slot order
                int m = 0;
                for (int t0 = 0; t0 < n; t0 += DB_T) {
                    const int t = t0 + threadIdx.x;
                    const bool root = t < n && par[t] == t;
                    int cntr;
                    const int pos = db_scan(root, cntr, S);
                    if (root) { nidC[t] = m + pos; rootC[m + pos] = t; }
                    m += cntr;
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T) {
                    const int p = par[t];
                    if (p < 0) nidC[t] = -1;
                    else if (p != t) nidC[t] = nidC[p];
                }
                for (int g = threadIdx.x; g < m; g += DB_T) { fluxC[g] = 0.0; nsig[g] = 0; tot[g] = 0; sgc[g] = -1; }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T)
                    if (nidC[t] >= 0) atomicAdd(fluxC + nidC[t], (double)F[t]);
                // children: the nodes of the level processed before this one
                for (int h = threadIdx.x; h < mN; h += DB_T) {
                    if (!(fluxN[h] >= cut)) continue;
                    const int g = nidC[rootN[h]];
                    atomicAdd(nsig + g, 1);
                    atomicAdd(tot + g, nobN[h]);
                    sgc[g] = h;
                }
                __syncthreads();
                for (int g = threadIdx.x; g < m; g += DB_T) {
                    const int k = nsig[g];
                    const int d = k >= 2 ? DB_PASS_ALL : (k == 1 && nobN[sgc[g]] >= 2 ? DB_PASS_ONE : DB_OBJECT);
                    dec[g] = d;
                    nobC[g] = d == DB_PASS_ALL ? tot[g] : (d == DB_PASS_ONE ? nobN[sgc[g]] : 1);
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T) {
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
                int* oid = J.ws.nsig + b0;   // per slot: object of the root at this slot
                int* ofirst = J.ws.tot + b0; // per object: first slot of its pixels
                int* otmp = J.ws.sgc + b0;   // per slot: provisional object
                int* orank = J.ws.dec + b0;  // per object: rank by first pixel
                double* o0 = J.ws.fluxA + b0;
                double* o1 = J.ws.fluxB + b0;
                double* o2 = J.ws.o2 + b0;
                double* o3 = J.ws.o3 + b0;
                double* o4 = J.ws.o4 + b0;
                double* o5 = J.ws.o5 + b0;
                for (int t = threadIdx.x; t < n; t += DB_T) oid[t] = 0;
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T)
                    if (core[t] >= 0) oid[core[t]] = 1;
                __syncthreads();
                int ne = 0;
                for (int t0 = 0; t0 < n; t0 += DB_T) {
                    const int t = t0 + threadIdx.x;
                    const bool isr = t < n && oid[t] == 1;
                    int cntr;
                    const int pos = db_scan(isr, cntr, S);
                    __syncthreads();
                    if (isr) oid[t] = 2 + ne + pos;  // 2 + object index (0, 1 are flags)
                    ne += cntr;
                }
                no = ne;
                for (int e = threadIdx.x; e < no; e += DB_T) {
                    o0[e] = 0.0; o1[e] = 0.0; o2[e] = 0.0; o3[e] = 0.0; o4[e] = 0.0; o5[e] = 0.0;
                    ofirst[e] = INT32_MAX;
                }
                __syncthreads();
                // core flux and barycentre
                for (int t = threadIdx.x; t < n; t += DB_T) {
                    if (core[t] < 0) continue;
                    const int e = oid[core[t]] - 2;
                    const double v = (double)F[t];
                    const int q = P[t];
                    atomicAdd(o0 + e, v);
                    atomicAdd(o1 + e, v * (double)(q % W));
                    atomicAdd(o2 + e, v * (double)(q / W));
                }
                __syncthreads();
                for (int e = threadIdx.x; e < no; e += DB_T) { o1[e] /= o0[e]; o2[e] /= o0[e]; }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T) {
                    if (core[t] < 0) continue;
                    const int e = oid[core[t]] - 2;
                    const double v = (double)F[t];
                    const int q = P[t];
                    const double dx = (double)(q % W) - o1[e], dy = (double)(q / W) - o2[e];
                    atomicAdd(o3 + e, v * dx * dx);
                    atomicAdd(o4 + e, v * dy * dy);
                    atomicAdd(o5 + e, v * dx * dy);
                }
                __syncthreads();
                // the elliptical Gaussian of each core: o0 <- F / sqrt(det),
                // o3, o4, o5 <- r^2 coefficients of dx^2, dy^2, dx dy
                for (int e = threadIdx.x; e < no; e += DB_T) {
                    double x2 = o3[e] / o0[e], y2 = o4[e] / o0[e], xy = o5[e] / o0[e];
                    if (x2 * y2 - xy * xy < 1.0 / 144.0) { x2 += 1.0 / 12.0; y2 += 1.0 / 12.0; }
                    const double det = x2 * y2 - xy * xy;
                    o3[e] = y2 / det;
                    o4[e] = x2 / det;
                    o5[e] = -2.0 * xy / det;
                    o0[e] = o0[e] / sqrt(det);
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T) {
                    int best;
                    if (core[t] >= 0) {
                        best = oid[core[t]] - 2;
                    } else {
                        const int q = P[t];
                        const double x = (double)(q % W), y = (double)(q / W);
                        double bv = -1.0;
                        best = 0;
                        for (int e = 0; e < no; e++) {
                            const double dx = x - o1[e], dy = y - o2[e];
                            const double r2 = o3[e] * dx * dx + o5[e] * dx * dy + o4[e] * dy * dy;
                            const double v = o0[e] * exp(-0.5 * r2);
                            if (v > bv) { bv = v; best = e; }
                        }
                    }
                    otmp[t] = best;
                    atomicMin(ofirst + best, t);
                }
                __syncthreads();
                for (int e = threadIdx.x; e < no; e += DB_T) {
                    int r = 0;
                    for (int e2 = 0; e2 < no; e2++) r += ofirst[e2] < ofirst[e];
                    orank[e] = r;
                }
                __syncthreads();
                for (int t = threadIdx.x; t < n; t += DB_T) asg[t] = orank[otmp[t]];
            }
        }
        if (whole) {
            no = n > 0 ? 1 : 0;  // an empty candidate yields no object
            for (int t = threadIdx.x; t < n; t += DB_T) asg[t] = 0;
        }
        if (threadIdx.x == 0) { J.ws.nobj[c] = no; J.ws.npx[c] = n; }
        __syncthreads();
    }
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
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_deblend, DB_T, 0) != cudaSuccess || per < 1) per = 1;
    k_deblend<<<db_sms() * per, DB_T, 0, s>>>(J);
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
