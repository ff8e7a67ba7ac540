// detect.cu -- pixel detection and connection into candidates, with the
// per-candidate pre-analysis of Sec. 2.2.5 (peak, total flux, ...).
//
// k_sub_thresh streams the frame in 32 x 128 tiles: Keys-interpolated
// background and rms, sub = f - B (written once, float4), and the detection
// mask sub > k rms(x, y) as bit rows (one 32-bit word per 32 pixels).  It is
// HBM-bound and holds nothing but the node columns of its tile on chip.
// k_tile_label then works from the bit rows alone (a given mask, in the parity
// path): one CTA per 32 x 128 tile cuts the rows into runs of detected pixels
// and unites runs of adjacent rows that touch (8-connectivity) with a
// union-find whose roots are the earliest run in raster order.  Components
// touching the tile border, or large enough, are kept and get a node with
// their partial statistics (values read back from the subtracted frame for the
// kept runs only); each run records its node for the final write.  The global
// phase unites nodes across tile seams, folds the stats into the roots, keeps
// roots of at least min_area pixels and numbers them by the raster index of
// their first pixel (survivors bucketed by tile row; a block per tile row
// ranks its bucket and adds the counts of earlier tile rows).  k_tile_final
// expands the runs into the label map, writing every pixel once.  Nothing
// depends on the tile shape but the work split.
#include <algorithm>
#include <vector>

#include "jobs.cuh"
#include "spline.cuh"

namespace ipp {

constexpr int T_TH = 32, T_TW = 128;
constexpr int T_WPR = T_TW / 32;                 // mask words per tile row
constexpr int T_CAP = (T_TH / 2) * (T_TW / 2);   // max 8-connected components in a tile
constexpr int T_RCAP = T_TH * (T_TW / 2);        // max runs in a tile
constexpr int T_THREADS = 128;
// tile kernel capacities: the common pass keeps up to 1024 runs (and the stats
// of 128 kept components) in shared memory, so ten tiles fit on an SM; tiles
// with more runs are redone by a second pass with the full capacity
constexpr int T_RCAP_FAST = 1024, KCAP_FAST = 128;
constexpr int KCAP_FULL = 256;
constexpr int T_NQ = 40;

enum TileMode { MODE_SUB_THRESH = 0, MODE_MASK = 1, MODE_FUSED = 2 };

// Global scratch of the labeling (node = tile * T_CAP + kept id; run = tile * T_RCAP + run id).
struct CclWs {
    int32_t* nkept;      // [ntiles]
    int32_t* nruns;      // [ntiles]
    uint32_t* runs;      // [ntiles*T_RCAP]: row << 16 | start << 8 | end
    int32_t* run_node;   // [ntiles*T_RCAP]: node of the run's component, -1 if dropped
    int32_t* parent;     // [ntiles*T_CAP]
    int32_t* area;
    unsigned long long* first;
    uint32_t* peak;      // order-preserving key
    int32_t* xmin; int32_t* xmax; int32_t* ymin; int32_t* ymax;
    // component sums sum f, sum f x, sum f y, each as two integers (see FxSum):
    // integer adds are exact, so the totals do not depend on the order in which
    // runs, tiles and nodes are merged
    long long* sum; long long* sx; long long* sy;     // [nodes][2]
    int32_t* label;
    int32_t* btop; int32_t* bbot;    // [ntiles*T_TW]
    int32_t* blef; int32_t* brig;    // [ntiles*T_TH]
    int32_t* counters;   // [0] kept nodes listed, [1] overflow tiles (zeroed by the host before the tile pass)
    int32_t* trcnt;      // [nty] surviving components per tile row (zeroed with counters)
    int32_t* klist;      // [ntiles*T_CAP] kept node ids, in no particular order
    int32_t* lpos;       // [nodes] tile-local index (row * T_TW + col) of the node's own first pixel
    int32_t* pk;         // [nodes] rank of a surviving component among its home tile's survivors, else -1
    int32_t* rowcnt;     // [ntiles][T_TH] survivors whose first pixel lies in that row of the tile
    int32_t* ovf;        // [ntiles] tiles left to the full-capacity pass (count in counters[1])
};

// Background subtraction + threshold into bit rows (streaming pass).
struct SubThreshJob {
    int64_t W, H;
    bool fused;                       // subtract the background from img and write sub
    const void* img; int dtype; int64_t pitch;
    const float* bias_map; float bias; const float* inv_flat;
    const float* mesh_bkg;
    float* sub; int64_t sub_pitch;    // output when fused, input otherwise
    const float* mesh_rms;
    int nx, ny, mesh_w, mesh_h;
    float k, thresh_abs;
    bool filter;                      // threshold the 3 x 3 pyramid-smoothed sub (not fused)
    uint32_t* mask;                   // [H][mw] bit rows, bit b of word w = column 32 w + b
    int64_t mw;
};

struct TileJob {
    int64_t W, H;
    int ntx, nty;
    const float* sub; int64_t sub_pitch;   // values of the statistics
    const uint32_t* mask; int64_t mw;      // bit rows (row stride mw words)
    int min_area;
    CclWs ws;
};

template <int RCAP, int KCAP>
struct TileShared {
    static constexpr int kRcap = RCAP, kKcap = KCAP;
    uint32_t mask[T_TH][T_WPR];
    int32_t roff[T_TH + 1];
    int16_t rs[RCAP], re[RCAP];      // run start / end column (inclusive)
    int32_t rpar[RCAP];              // union-find over runs
    int32_t rarea[RCAP];             // area at the root run; border flag in bit 30
    int16_t rkid[RCAP];              // kept id at the root run, -1 if dropped
    int32_t nruns, nkept;
    // statistics of the first KCAP kept components
    long long k_sum[KCAP][2], k_sx[KCAP][2], k_sy[KCAP][2];
    uint32_t k_peak[KCAP];
    int32_t k_xmin[KCAP], k_xmax[KCAP], k_ymin[KCAP], k_ymax[KCAP];
    int32_t wsum[2 * (T_TH * T_WPR / 32) > T_THREADS / 32 ? 2 * (T_TH * T_WPR / 32) : T_THREADS / 32];
};
using TileFast = TileShared<T_RCAP_FAST, KCAP_FAST>;
using TileFull = TileShared<T_RCAP, KCAP_FULL>;

constexpr int BORDER_BIT = 1 << 30;


static_assert(T_TH * T_WPR <= T_THREADS, "one thread per mask word");

__device__ __forceinline__ int rfind(const int32_t* P, int x) {
    int p = P[x];
    while (p != x) { x = p; p = P[x]; }
    return x;
}
// lock-free union by atomicMin: the larger root is linked under the smaller
__device__ __forceinline__ void runite(int32_t* P, int a, int b) {
    while (true) {
        a = rfind(P, a);
        b = rfind(P, b);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicMin(&P[b], a);
        if (old == b) return;
        b = old;
    }
}
template <class SH>
__device__ __forceinline__ bool mbit(const SH& S, int r, int c) {
    return (S.mask[r][c >> 5] >> (c & 31)) & 1u;
}

__device__ __forceinline__ float tile_load_pix(const SubThreshJob& J, int64_t y, int64_t x) {
    if (J.dtype == IPP_F32) return __ldg(reinterpret_cast<const float*>(J.img) + y * J.pitch + x);
    float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(J.img) + y * J.pitch + x);
    float b = J.bias_map ? __ldg(J.bias_map + y * J.W + x) : J.bias;
    return (raw - b) * __ldg(J.inv_flat + y * J.W + x);
}

template <class SH>
__device__ __forceinline__ int row_of_run(const SH& S, int i) {  // largest r with roff[r] <= i
    int a = 0, b = T_TH - 1;
    while (a < b) { const int m = (a + b + 1) >> 1; if (S.roff[m] <= i) a = m; else b = m - 1; }
    return a;
}

// Cut the mask rows into runs (row-major, increasing start), one thread per
// mask word: run starts are set bits whose left neighbour is clear, run ends set
// bits whose right neighbour is clear (neighbours across word edges included);
// the k-th start and the k-th end of the tile bound the k-th run.
template <class SH>
__device__ void tile_runs(SH& S) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t st = 0, en = 0;
    if (t < T_TH * T_WPR) {
        const int r = t / T_WPR, w = t % T_WPR;
        const uint32_t m = S.mask[r][w];
        const uint32_t pb = w > 0 ? S.mask[r][w - 1] >> 31 : 0u;
        const uint32_t nb = w < T_WPR - 1 ? S.mask[r][w + 1] & 1u : 0u;
        st = m & ~((m << 1) | pb);
        en = m & ~((m >> 1) | (nb << 31));
    }
    const int cs = __popc(st), ce = __popc(en);
    int is = cs, ie = ce;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, is, o), b = __shfl_up_sync(0xffffffffu, ie, o);
        if (lane >= o) { is += a; ie += b; }
    }
    constexpr int NWW = (T_TH * T_WPR) / 32;  // warps holding mask words
    if (lane == 31 && warp < NWW) { S.wsum[warp] = is; S.wsum[NWW + warp] = ie; }
    __syncthreads();
    int total = 0;
    for (int k = 0; k < NWW; k++) total += S.wsum[k];
    if (total > SH::kRcap) {  // more runs than this pass holds: the tile is redone by the full pass
        if (t == 0) S.nruns = -1;
        __syncthreads();
        return;
    }
    if (t < T_TH * T_WPR) {
        int bs = 0, be = 0;
        for (int k = 0; k < warp; k++) { bs += S.wsum[k]; be += S.wsum[NWW + k]; }
        int ps = bs + is - cs, pe = be + ie - ce;
        if (t % T_WPR == 0) S.roff[t / T_WPR] = ps;
        const int base = (t % T_WPR) * 32;
        while (st) { const int b = __ffs(st) - 1; st &= st - 1; S.rs[ps++] = (int16_t)(base + b); }
        while (en) { const int b = __ffs(en) - 1; en &= en - 1; S.re[pe++] = (int16_t)(base + b); }
        if (t == T_TH * T_WPR - 1) { S.roff[T_TH] = ps; S.nruns = ps; }
    }
    __syncthreads();
}

// Union-find over the runs of the tile: run i of row r joins the runs of row
// r - 1 that overlap [start - 1, end + 1] (8-connectivity).  Roots end up as the
// smallest run id of the component (its first run in raster order).
template <class SH>
__device__ void tile_union(SH& S) {
    const int nr = S.nruns;
    for (int i = threadIdx.x; i < nr; i += T_THREADS) S.rpar[i] = i;
    __syncthreads();
    for (int i = threadIdx.x; i < nr; i += T_THREADS) {
        const int r = row_of_run(S, i);
        if (r == 0) continue;
        const int a = S.rs[i] - 1, b = S.re[i] + 1;
        int lo = S.roff[r - 1], hi = S.roff[r];      // first run of row r-1 ending at or after a
        const int end = hi;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (S.re[m] < a) lo = m + 1; else hi = m; }
        for (int k = lo; k < end && S.rs[k] <= b; k++) runite(S.rpar, i, k);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nr; i += T_THREADS) S.rpar[i] = rfind(S.rpar, i);
    __syncthreads();
}

constexpr int ST_TH = 32, ST_TW = 128, ST_THREADS = 256;

__device__ __forceinline__ void sub_thresh_body(const SubThreshJob& J, int bx, int by) {
    __shared__ float cvb[ST_TH][T_NQ], cvr[ST_TH][T_NQ];
    const int64_t tx0 = (int64_t)bx * ST_TW, ty0 = (int64_t)by * ST_TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per row: vertical interpolation of the node columns this tile reads
    const int qa = (int)floorf(((float)(int)tx0 + 0.5f) / J.mesh_w - 0.5f) - 1;
    const int qz = (int)floorf(((float)((int)tx0 + ST_TW - 1) + 0.5f) / J.mesh_w - 0.5f) + 2;
    const int qbase = max(qa, 0);
    const int nq = min(min(qz, J.nx - 1) - qbase + 1, T_NQ);
    const float refr = J.mesh_rms[0];
    const float refb = J.fused ? J.mesh_bkg[0] : 0.f;
    for (int t = threadIdx.x; t < ST_TH * nq; t += ST_THREADS) {
        const int r = t / nq, qq = t - r * nq;
        const int q = min(qbase + qq, J.nx - 1);
        const float vy = ((float)((int)ty0 + r) + 0.5f) / J.mesh_h - 0.5f;
        const float pf = floorf(vy);
        float w[4];
        keys_weights(vy - pf, w);
        const int p0 = (int)pf;
        float ab = 0.f, ar = 0.f;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int p = clampi(p0 - 1 + a, 0, J.ny - 1);
            ar = fmaf(w[a], J.mesh_rms[p * J.nx + q] - refr, ar);
            if (J.fused) ab = fmaf(w[a], J.mesh_bkg[p * J.nx + q] - refb, ab);
        }
        cvr[r][qq] = ar;
        cvb[r][qq] = ab;
    }
    __syncthreads();
    const int64_t xc = tx0 + lane * 4;
    float wx[4][4];
    int q0c[4];  // first node column of each of the 4 pixels (node index = clamp(q0 - 1 + b))
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const float u = ((float)((int)xc + c) + 0.5f) / J.mesh_w - 0.5f;
        const float qf = floorf(u);
        keys_weights(u - qf, wx[c]);
        q0c[c] = (int)qf;
    }
    auto qi = [&](int c, int b) { return min(clampi(q0c[c] - 1 + b, 0, J.nx - 1) - qbase, T_NQ - 1); };
    const bool vin = (J.pitch % 4 == 0) && (((uintptr_t)J.img & 15) == 0) && J.dtype == IPP_F32;
    const bool vsub = (J.sub_pitch % 4 == 0) && (((uintptr_t)J.sub & 15) == 0);
    const bool full4 = xc + 4 <= J.W;
    // the warp's rows: all loads first (several in flight per thread), then the arithmetic
    constexpr int RPW = ST_TH / (ST_THREADS / 32);
    float f[RPW][4];
#pragma unroll
    for (int q = 0; q < RPW; q++) {
        const int64_t y = ty0 + warp + q * (ST_THREADS / 32);
#pragma unroll
        for (int c = 0; c < 4; c++) f[q][c] = 0.f;
        if (y >= J.H || xc >= J.W) continue;
        if (J.fused) {
            if (vin && full4) {
                const float4 t4 = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(J.img) + y * J.pitch + xc));
                f[q][0] = t4.x; f[q][1] = t4.y; f[q][2] = t4.z; f[q][3] = t4.w;
            } else {
#pragma unroll
                for (int c = 0; c < 4; c++) f[q][c] = (xc + c < J.W) ? tile_load_pix(J, y, xc + c) : 0.f;
            }
        } else if (J.filter) {
            // detection filter: [1 2 1; 2 4 2; 1 2 1] over the taps inside the frame,
            // divided by the sum of their weights
            float row[3][6];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int64_t yy = y - 1 + a;
#pragma unroll
                for (int b = 0; b < 6; b++) {
                    const int64_t xx = xc - 1 + b;
                    row[a][b] = (yy >= 0 && yy < J.H && xx >= 0 && xx < J.W) ? __ldg(J.sub + yy * J.sub_pitch + xx) : 0.f;
                }
            }
            const float wy0 = y > 0 ? 1.f : 0.f, wy2 = y + 1 < J.H ? 1.f : 0.f;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int64_t x = xc + c;
                const float wx0 = x > 0 ? 1.f : 0.f, wx2 = x + 1 < J.W ? 1.f : 0.f;
                float num = 0.f;
#pragma unroll
                for (int a = 0; a < 3; a++)
                    num += (a == 1 ? 2.f : 1.f) * (row[a][c] + 2.f * row[a][c + 1] + row[a][c + 2]);
                const float den = (wy0 + 2.f + wy2) * (wx0 + 2.f + wx2);
                f[q][c] = num / den;
            }
        } else {
            if (vsub && full4) {
                const float4 t4 = __ldg(reinterpret_cast<const float4*>(J.sub + y * J.sub_pitch + xc));
                f[q][0] = t4.x; f[q][1] = t4.y; f[q][2] = t4.z; f[q][3] = t4.w;
            } else {
#pragma unroll
                for (int c = 0; c < 4; c++) f[q][c] = (xc + c < J.W) ? __ldg(J.sub + y * J.sub_pitch + xc + c) : 0.f;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPW; q++) {
        const int r = warp + q * (ST_THREADS / 32);
        const int64_t y = ty0 + r;
        uint32_t nib = 0;
        if (y < J.H && xc < J.W) {
            if (J.fused) {
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    float acc = 0.f;
#pragma unroll
                    for (int b = 0; b < 4; b++) acc = fmaf(wx[c][b], cvb[r][qi(c, b)], acc);
                    f[q][c] = f[q][c] - (refb + acc);
                }
                if (vsub && full4) {
                    *reinterpret_cast<float4*>(J.sub + y * J.sub_pitch + xc) =
                        make_float4(f[q][0], f[q][1], f[q][2], f[q][3]);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        if (xc + c < J.W) J.sub[y * J.sub_pitch + xc + c] = f[q][c];
                }
            }
#pragma unroll
            for (int c = 0; c < 4; c++) {
                float acc = 0.f;
#pragma unroll
                for (int b = 0; b < 4; b++) acc = fmaf(wx[c][b], cvr[r][qi(c, b)], acc);
                const float thr = fmaxf(J.k * (refr + acc), J.thresh_abs);
                if (xc + c < J.W && f[q][c] > thr) nib |= 1u << c;
            }
        }
        // 8 lanes x 4 bits -> one 32-bit word of the row
        uint32_t wv = nib << (4 * (lane & 7));
        wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 4);
        const int64_t wcol = (xc >> 5);
        if ((lane & 7) == 0 && y < J.H && wcol < J.mw) J.mask[y * J.mw + wcol] = wv;
    }
}

__global__ void __launch_bounds__(ST_THREADS, 4) k_sub_thresh(SubThreshJob J) {
    sub_thresh_body(J, blockIdx.x, blockIdx.y);
}

// Same pass with the horizontal Keys interpolation in polynomial form: per tile
// row and node interval q0 the four (row-interpolated) node values give
// B(t) = c0 + c1 t + c2 t^2 + c3 t^3, t = u - q0 (relative to the reference
// node value, so a constant sky still subtracts to exactly 0); a pixel costs one
// shared float4 and three FMAs per map.  For meshes of at least 16 px, where a
// 128 px tile spans at most 9 intervals.
constexpr int ST_NINT = 9;

__device__ __forceinline__ float4 keys_poly(float d0, float d1, float d2, float d3) {
    return make_float4(d1, 0.5f * (d2 - d0), d0 - 2.5f * d1 + 2.0f * d2 - 0.5f * d3,
                       0.5f * (d3 - d0) + 1.5f * (d1 - d2));
}

__device__ __forceinline__ void sub_thresh_poly_body(const SubThreshJob& J, int bx, int by) {
    __shared__ float cvb[ST_TH][T_NQ], cvr[ST_TH][T_NQ];
    __shared__ float4 pb[ST_TH][ST_NINT], pr[ST_TH][ST_NINT];
    const int64_t tx0 = (int64_t)bx * ST_TW, ty0 = (int64_t)by * ST_TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int qa = (int)floorf(((float)(int)tx0 + 0.5f) / J.mesh_w - 0.5f) - 1;
    const int qz = (int)floorf(((float)((int)tx0 + ST_TW - 1) + 0.5f) / J.mesh_w - 0.5f) + 2;
    const int qbase = max(qa, 0);
    const int nq = min(min(qz, J.nx - 1) - qbase + 1, T_NQ);
    const int q0min = qa + 1, nint = min(qz - 2 - q0min + 1, ST_NINT);
    const float refr = J.mesh_rms[0];
    const float refb = J.fused ? J.mesh_bkg[0] : 0.f;
    for (int t = threadIdx.x; t < ST_TH * nq; t += ST_THREADS) {
        const int r = t / nq, qq = t - r * nq;
        const int q = min(qbase + qq, J.nx - 1);
        const float vy = ((float)((int)ty0 + r) + 0.5f) / J.mesh_h - 0.5f;
        const float pf = floorf(vy);
        float w[4];
        keys_weights(vy - pf, w);
        const int p0 = (int)pf;
        float ab = 0.f, ar = 0.f;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int p = clampi(p0 - 1 + a, 0, J.ny - 1);
            ar = fmaf(w[a], J.mesh_rms[p * J.nx + q] - refr, ar);
            if (J.fused) ab = fmaf(w[a], J.mesh_bkg[p * J.nx + q] - refb, ab);
        }
        cvr[r][qq] = ar;
        cvb[r][qq] = ab;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ST_TH * nint; t += ST_THREADS) {
        const int r = t / nint, k = t - r * nint;
        const int q0 = q0min + k;
        int ix[4];
#pragma unroll
        for (int b = 0; b < 4; b++) ix[b] = min(clampi(q0 - 1 + b, 0, J.nx - 1) - qbase, T_NQ - 1);
        pr[r][k] = keys_poly(cvr[r][ix[0]], cvr[r][ix[1]], cvr[r][ix[2]], cvr[r][ix[3]]);
        if (J.fused) pb[r][k] = keys_poly(cvb[r][ix[0]], cvb[r][ix[1]], cvb[r][ix[2]], cvb[r][ix[3]]);
    }
    __syncthreads();
    const int64_t xc = tx0 + lane * 4;
    float tc[4];
    int kc[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const float u = ((float)((int)xc + c) + 0.5f) / J.mesh_w - 0.5f;
        const float qf = floorf(u);
        tc[c] = u - qf;
        kc[c] = min(max((int)qf - q0min, 0), ST_NINT - 1);
    }
    const bool vin = (J.pitch % 4 == 0) && (((uintptr_t)J.img & 15) == 0) && J.dtype == IPP_F32;
    const bool vsub = (J.sub_pitch % 4 == 0) && (((uintptr_t)J.sub & 15) == 0);
    const bool full4 = xc + 4 <= J.W;
    constexpr int RPW = ST_TH / (ST_THREADS / 32);
    float f[RPW][4];
#pragma unroll
    for (int q = 0; q < RPW; q++) {
        const int64_t y = ty0 + warp + q * (ST_THREADS / 32);
#pragma unroll
        for (int c = 0; c < 4; c++) f[q][c] = 0.f;
        if (y >= J.H || xc >= J.W) continue;
        if (J.fused) {
            if (vin && full4) {
                const float4 t4 = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(J.img) + y * J.pitch + xc));
                f[q][0] = t4.x; f[q][1] = t4.y; f[q][2] = t4.z; f[q][3] = t4.w;
            } else {
#pragma unroll
                for (int c = 0; c < 4; c++) f[q][c] = (xc + c < J.W) ? tile_load_pix(J, y, xc + c) : 0.f;
            }
        } else if (J.filter) {
            // detection filter: [1 2 1; 2 4 2; 1 2 1] over the taps inside the frame,
            // divided by the sum of their weights
            float row[3][6];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const int64_t yy = y - 1 + a;
#pragma unroll
                for (int b = 0; b < 6; b++) {
                    const int64_t xx = xc - 1 + b;
                    row[a][b] = (yy >= 0 && yy < J.H && xx >= 0 && xx < J.W) ? __ldg(J.sub + yy * J.sub_pitch + xx) : 0.f;
                }
            }
            const float wy0 = y > 0 ? 1.f : 0.f, wy2 = y + 1 < J.H ? 1.f : 0.f;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int64_t x = xc + c;
                const float wx0 = x > 0 ? 1.f : 0.f, wx2 = x + 1 < J.W ? 1.f : 0.f;
                float num = 0.f;
#pragma unroll
                for (int a = 0; a < 3; a++)
                    num += (a == 1 ? 2.f : 1.f) * (row[a][c] + 2.f * row[a][c + 1] + row[a][c + 2]);
                const float den = (wy0 + 2.f + wy2) * (wx0 + 2.f + wx2);
                f[q][c] = num / den;
            }
        } else {
            if (vsub && full4) {
                const float4 t4 = __ldg(reinterpret_cast<const float4*>(J.sub + y * J.sub_pitch + xc));
                f[q][0] = t4.x; f[q][1] = t4.y; f[q][2] = t4.z; f[q][3] = t4.w;
            } else {
#pragma unroll
                for (int c = 0; c < 4; c++) f[q][c] = (xc + c < J.W) ? __ldg(J.sub + y * J.sub_pitch + xc + c) : 0.f;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPW; q++) {
        const int r = warp + q * (ST_THREADS / 32);
        const int64_t y = ty0 + r;
        uint32_t nib = 0;
        if (y < J.H && xc < J.W) {
            if (J.fused) {
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    const float4 P = pb[r][kc[c]];
                    const float t = tc[c];
                    f[q][c] = f[q][c] - (refb + fmaf(fmaf(fmaf(P.w, t, P.z), t, P.y), t, P.x));
                }
                if (vsub && full4) {
                    *reinterpret_cast<float4*>(J.sub + y * J.sub_pitch + xc) =
                        make_float4(f[q][0], f[q][1], f[q][2], f[q][3]);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; c++)
                        if (xc + c < J.W) J.sub[y * J.sub_pitch + xc + c] = f[q][c];
                }
            }
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const float4 P = pr[r][kc[c]];
                const float t = tc[c];
                const float thr = fmaxf(J.k * (refr + fmaf(fmaf(fmaf(P.w, t, P.z), t, P.y), t, P.x)), J.thresh_abs);
                if (xc + c < J.W && f[q][c] > thr) nib |= 1u << c;
            }
        }
        uint32_t wv = nib << (4 * (lane & 7));
        wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
        wv |= __shfl_xor_sync(0xffffffffu, wv, 4);
        const int64_t wcol = (xc >> 5);
        if ((lane & 7) == 0 && y < J.H && wcol < J.mw) J.mask[y * J.mw + wcol] = wv;
    }
}

__global__ void __launch_bounds__(ST_THREADS, 4) k_sub_thresh_poly(SubThreshJob J) {
    sub_thresh_poly_body(J, blockIdx.x, blockIdx.y);
}

// One tile, all threads of the block.  Returns false, having written nothing
// to global memory, when the tile has more runs than SH holds.
template <class SH>
__device__ bool tile_label_body(const TileJob& J, SH& S, int tile) {
    constexpr int KCAP = SH::kKcap;
    const int ty = tile / J.ntx, tx = tile - ty * J.ntx;
    const int64_t tx0 = (int64_t)tx * T_TW, ty0 = (int64_t)ty * T_TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();  // shared state of a previous tile of this block is dead

    // ---- phase A: the tile's bit rows (bits beyond W dropped) ---------------
    if (threadIdx.x < T_TH * T_WPR) {
        const int r = threadIdx.x / T_WPR, wi = threadIdx.x % T_WPR;
        const int64_t y = ty0 + r, wcol = (tx0 >> 5) + wi;
        uint32_t m = 0;
        if (y < J.H && wcol < J.mw) {
            m = __ldg(J.mask + y * J.mw + wcol);
            const int64_t valid = J.W - 32 * wcol;
            if (valid < 32) m &= valid > 0 ? ((1u << valid) - 1u) : 0u;
        }
        S.mask[r][wi] = m;
    }
    __syncthreads();

    // ---- phase B/C: runs and their union-find --------------------------------
    tile_runs(S);
    if (S.nruns < 0) return false;
    tile_union(S);
    const int nr = S.nruns;

    // ---- phase D: area and border flag at the root runs -----------------------
    for (int i = threadIdx.x; i < nr; i += T_THREADS) S.rarea[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nr; i += T_THREADS) {
        const int r = row_of_run(S, i);
        const int st = S.rs[i], en = S.re[i];
        const int root = S.rpar[i];
        if (r == 0 || r == T_TH - 1 || st == 0 || en == T_TW - 1) atomicOr(&S.rarea[root], BORDER_BIT);
        atomicAdd(&S.rarea[root], en - st + 1);
    }
    __syncthreads();

    // ---- phase E: kept components get consecutive ids (raster order of roots) --
    {
        int chunk0 = 0;
        for (int base = 0; base < nr; base += T_THREADS) {
            const int i = base + threadIdx.x;
            bool kept = false;
            if (i < nr && S.rpar[i] == i) {
                const int v = S.rarea[i];
                kept = (v & BORDER_BIT) || (v & ~BORDER_BIT) >= J.min_area;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, kept);
            if (lane == 0) S.wsum[warp] = __popc(bal);
            __syncthreads();
            int before = chunk0;
            for (int w = 0; w < warp; w++) before += S.wsum[w];
            int total = chunk0;
            for (int w = 0; w < T_THREADS / 32; w++) total += S.wsum[w];
            if (i < nr) S.rkid[i] = kept ? before + __popc(bal & ((1u << lane) - 1u)) : -1;
            __syncthreads();
            chunk0 = total;
        }
        if (threadIdx.x == 0) S.nkept = chunk0;
    }
    __syncthreads();
    const int nk = S.nkept;
    for (int c = threadIdx.x; c < min(nk, KCAP); c += T_THREADS) {
        S.k_sum[c][0] = S.k_sum[c][1] = 0; S.k_sx[c][0] = S.k_sx[c][1] = 0; S.k_sy[c][0] = S.k_sy[c][1] = 0;
        S.k_peak[c] = 0u;
        S.k_xmin[c] = T_TW; S.k_xmax[c] = -1; S.k_ymin[c] = T_TH; S.k_ymax[c] = -1;
    }
    // kept components beyond the shared tables accumulate in the global node
    // arrays directly (only masks with more than KCAP kept components per tile)
    for (int i = threadIdx.x; i < nr; i += T_THREADS) {
        const int kid = (S.rpar[i] == i) ? S.rkid[i] : -1;
        if (kid >= KCAP) {
            const int node = tile * T_CAP + kid;
            for (int h = 0; h < 2; h++) J.ws.sum[2 * node + h] = J.ws.sx[2 * node + h] = J.ws.sy[2 * node + h] = 0;
            J.ws.peak[node] = 0u;
            J.ws.xmin[node] = INT32_MAX; J.ws.xmax[node] = -1; J.ws.ymin[node] = INT32_MAX; J.ws.ymax[node] = -1;
        }
    }
    __syncthreads();

    // ---- phase F: per-run partial stats (values re-read from L2) ---------------
    for (int i = threadIdx.x; i < nr; i += T_THREADS) {
        const int kid = S.rkid[S.rpar[i]];
        if (kid < 0) continue;
        const int r = row_of_run(S, i);
        const int st = S.rs[i], en = S.re[i];
        float s0 = 0.f, s1 = 0.f, pk = -INFINITY;
        const float* row = J.sub + (ty0 + r) * J.sub_pitch + tx0;
        for (int c0 = st; c0 <= en; c0 += 8) {  // 8 loads in flight, summed in column order
            float f[8];
#pragma unroll
            for (int u = 0; u < 8; u++) f[u] = c0 + u <= en ? __ldg(row + c0 + u) : 0.f;
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (c0 + u <= en) {
                    s0 += f[u];
                    s1 = fmaf(f[u], (float)(c0 + u), s1);
                    pk = fmaxf(pk, f[u]);
                }
        }
        // the run's FP32 partial sums as exact integer pairs
        long long f0[2], f1[2];
        fx_split(s0, f0);
        fx_split(s1, f1);
        if (kid < KCAP) {
            for (int h = 0; h < 2; h++) {
                atomicAdd(reinterpret_cast<unsigned long long*>(&S.k_sum[kid][h]), (unsigned long long)f0[h]);
                atomicAdd(reinterpret_cast<unsigned long long*>(&S.k_sx[kid][h]), (unsigned long long)f1[h]);
                atomicAdd(reinterpret_cast<unsigned long long*>(&S.k_sy[kid][h]), (unsigned long long)(f0[h] * r));
            }
            atomicMax(&S.k_peak[kid], fkey(pk));
            atomicMin(&S.k_xmin[kid], st);
            atomicMax(&S.k_xmax[kid], en);
            atomicMin(&S.k_ymin[kid], r);
            atomicMax(&S.k_ymax[kid], r);
        } else {
            const int node = tile * T_CAP + kid;
            for (int h = 0; h < 2; h++) {
                atomicAdd(reinterpret_cast<unsigned long long*>(&J.ws.sum[2 * node + h]), (unsigned long long)f0[h]);
                atomicAdd(reinterpret_cast<unsigned long long*>(&J.ws.sx[2 * node + h]),
                          (unsigned long long)(f1[h] + tx0 * f0[h]));
                atomicAdd(reinterpret_cast<unsigned long long*>(&J.ws.sy[2 * node + h]),
                          (unsigned long long)(f0[h] * (ty0 + r)));
            }
            atomicMax(&J.ws.peak[node], fkey(pk));
            atomicMin(&J.ws.xmin[node], (int)tx0 + st);
            atomicMax(&J.ws.xmax[node], (int)tx0 + en);
            atomicMin(&J.ws.ymin[node], (int)ty0 + r);
            atomicMax(&J.ws.ymax[node], (int)ty0 + r);
        }
    }
    __syncthreads();

    // ---- phase G: nodes, run table, border nodes -------------------------------
    for (int i = threadIdx.x; i < nr; i += T_THREADS) {
        const int root = S.rpar[i];
        const int kid = S.rkid[root];
        const int node = kid >= 0 ? tile * T_CAP + kid : -1;
        const int r = row_of_run(S, i);
        J.ws.runs[(int64_t)tile * T_RCAP + i] = ((uint32_t)r << 16) | ((uint32_t)S.rs[i] << 8) | (uint32_t)S.re[i];
        J.ws.run_node[(int64_t)tile * T_RCAP + i] = node;
        if (root == i && kid >= 0) {
            J.ws.parent[node] = node;
            J.ws.area[node] = S.rarea[i] & ~BORDER_BIT;
            J.ws.first[node] = (unsigned long long)((ty0 + r) * J.W + tx0 + S.rs[i]);
            J.ws.lpos[node] = r * T_TW + S.rs[i];
            if (kid < KCAP) {

                J.ws.peak[node] = S.k_peak[kid];
                J.ws.xmin[node] = (int)tx0 + S.k_xmin[kid];
                J.ws.xmax[node] = (int)tx0 + S.k_xmax[kid];
                J.ws.ymin[node] = (int)ty0 + S.k_ymin[kid];
                J.ws.ymax[node] = (int)ty0 + S.k_ymax[kid];
                for (int h = 0; h < 2; h++) {
                    const long long sm = S.k_sum[kid][h];
                    J.ws.sum[2 * node + h] = sm;
                    J.ws.sx[2 * node + h] = S.k_sx[kid][h] + tx0 * sm;
                    J.ws.sy[2 * node + h] = S.k_sy[kid][h] + ty0 * sm;
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        J.ws.nkept[tile] = nk;
        J.ws.nruns[tile] = nr;
        S.nkept = nk > 0 ? atomicAdd(&J.ws.counters[0], nk) : 0;  // base of this tile in klist
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += T_THREADS) J.ws.klist[S.nkept + k] = tile * T_CAP + k;
    // border pixels: node of the run covering them (runs of a row are sorted)
    for (int t = threadIdx.x; t < 2 * T_TW + 2 * T_TH; t += T_THREADS) {
        int r, c;
        int32_t* dst;
        if (t < T_TW) { r = 0; c = t; dst = J.ws.btop + (int64_t)tile * T_TW + c; }
        else if (t < 2 * T_TW) { r = T_TH - 1; c = t - T_TW; dst = J.ws.bbot + (int64_t)tile * T_TW + c; }
        else if (t < 2 * T_TW + T_TH) { r = t - 2 * T_TW; c = 0; dst = J.ws.blef + (int64_t)tile * T_TH + r; }
        else { r = t - 2 * T_TW - T_TH; c = T_TW - 1; dst = J.ws.brig + (int64_t)tile * T_TH + r; }
        int v = -1;
        if (mbit(S, r, c)) {
            int a = S.roff[r], b = S.roff[r + 1] - 1;   // last run starting at or before c
            while (a < b) { const int m = (a + b + 1) >> 1; if (S.rs[m] <= c) a = m; else b = m - 1; }
            const int kid = S.rkid[S.rpar[a]];
            v = kid >= 0 ? tile * T_CAP + kid : -1;
        }
        *dst = v;
    }
    return true;
}

// Common pass: one tile per block with the small capacities; tiles that do not
// fit are listed for the full pass.
__device__ __forceinline__ void tile_label_fast(const TileJob& J, int tile) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileFast& S = *reinterpret_cast<TileFast*>(smem_raw);
    if (!tile_label_body(J, S, tile) && threadIdx.x == 0) {
        const int slot = atomicAdd(&J.ws.counters[1], 1);
        J.ws.ovf[slot] = tile;
    }
}

__global__ void __launch_bounds__(T_THREADS) k_tile_label(TileJob J) { tile_label_fast(J, blockIdx.y * J.ntx + blockIdx.x); }

// Full pass over the listed tiles (any mask fits: T_RCAP is the most runs a
// tile can have).
__device__ __forceinline__ void tile_label_full(const TileJob& J, int vb, int nvb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileFull& S = *reinterpret_cast<TileFull*>(smem_raw);
    const int n = __ldcg(J.ws.counters + 1);
    for (int i = vb; i < n; i += nvb) tile_label_body(J, S, __ldcg(J.ws.ovf + i));
}

__global__ void __launch_bounds__(T_THREADS) k_tile_label_full(TileJob J) { tile_label_full(J, blockIdx.x, gridDim.x); }

// ------------------------------------------------------------ global phase
__device__ __forceinline__ int gfind(int32_t* P, int x) {
    int p = __ldcg(P + x);
    while (p != x) { x = p; p = __ldcg(P + x); }
    return x;
}
__device__ __forceinline__ void gunite(int32_t* P, int a, int b) {
    while (true) {
        a = gfind(P, a);
        b = gfind(P, b);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicMin(&P[b], a);
        if (old == b) return;
        b = old;
    }
}

// ---- global phase, as per-unit bodies run by the persistent kernel below ----
// seams of one tile: threads 0..127 the bottom seam (diagonal corners
// included), threads 128..159 the right seam
__device__ void ccl_union_tile(const CclWs& ws, int tile, int ntx, int nty) {
    const int ty = tile / ntx, tx = tile - ty * ntx;
    const int t = threadIdx.x;
    if (t < T_TW) {
        if (ty + 1 < nty) {
            const int below = tile + ntx;
            const int a = __ldcg(ws.bbot + (int64_t)tile * T_TW + t);
            if (a >= 0) {
                for (int d = -1; d <= 1; d++) {
                    const int j = t + d;
                    int b;
                    if (j < 0) b = (tx > 0) ? __ldcg(ws.btop + (int64_t)(below - 1) * T_TW + T_TW - 1) : -1;
                    else if (j >= T_TW) b = (tx + 1 < ntx) ? __ldcg(ws.btop + (int64_t)(below + 1) * T_TW) : -1;
                    else b = __ldcg(ws.btop + (int64_t)below * T_TW + j);
                    if (b >= 0) gunite(ws.parent, a, b);
                }
            }
        }
    } else if (t < T_TW + T_TH) {
        const int i0 = t - T_TW;
        if (tx + 1 < ntx) {
            const int right = tile + 1;
            const int a = __ldcg(ws.brig + (int64_t)tile * T_TH + i0);
            if (a >= 0) {
                for (int d = -1; d <= 1; d++) {
                    const int i = i0 + d;
                    if (i < 0 || i >= T_TH) continue;
                    const int b = __ldcg(ws.blef + (int64_t)right * T_TH + i);
                    if (b >= 0) gunite(ws.parent, a, b);
                }
            }
        }
    }
}

// fold kept node `node` into its root
__device__ __forceinline__ void ccl_resolve_node(const CclWs& ws, int node) {
    const int r = gfind(ws.parent, node);
    if (r == node) return;
    ws.parent[node] = r;
    atomicAdd(&ws.area[r], ws.area[node]);
    atomicMin(&ws.first[r], ws.first[node]);
    atomicMax(&ws.peak[r], ws.peak[node]);
    atomicMin(&ws.xmin[r], ws.xmin[node]);
    atomicMax(&ws.xmax[r], ws.xmax[node]);
    atomicMin(&ws.ymin[r], ws.ymin[node]);
    atomicMax(&ws.ymax[r], ws.ymax[node]);
    for (int h = 0; h < 2; h++) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&ws.sum[2 * r + h]), (unsigned long long)ws.sum[2 * node + h]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ws.sx[2 * r + h]), (unsigned long long)ws.sx[2 * node + h]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&ws.sy[2 * r + h]), (unsigned long long)ws.sy[2 * node + h]);
    }
}

// Numbering without a sort.  Labels follow the raster order of first pixels.
// The first pixel of a component lies in one node's own runs (its home node,
// in its home tile); within a tile, kept ids already follow the raster order of
// the nodes' first pixels.  So a component's label is
//   (survivors of earlier tile rows) + (survivors of this tile row whose first
//   pixel lies in an earlier row, or in the same row in an earlier tile)
//   + (its rank among its home tile's survivors of that row) + 1.
// ccl_count_tile: ranks the tile's home survivors in kept-id order and counts
// them per row; dropped roots get label 0.  Block-wide.
constexpr int G_THREADS = 256, G_WARPS = G_THREADS / 32;
struct GShared {
    int cnt[T_TH];
    int red[G_WARPS];
    int carry;
};
constexpr int CT_WORDS = 8;   // CclWs::counters words before the per-tile-row counts

__device__ void ccl_count_tile(const CclWs& ws, GShared& G, int tile, int64_t W, int ntx, int min_area) {
    const int ty = tile / ntx, tx = tile - ty * ntx;
    const int64_t tx0 = (int64_t)tx * T_TW, ty0 = (int64_t)ty * T_TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < T_TH) G.cnt[threadIdx.x] = 0;
    __syncthreads();
    const int nk = __ldcg(ws.nkept + tile);
    int chunk0 = 0;
    for (int base = 0; base < nk; base += G_THREADS) {
        const int k = base + threadIdx.x;
        bool surv = false;
        int r = 0;
        if (k < nk) {
            const int node = tile * T_CAP + k;
            const int root = __ldcg(ws.parent + node);
            const int lp = __ldcg(ws.lpos + node);
            r = lp / T_TW;
            const unsigned long long gf = (unsigned long long)((ty0 + r) * W + tx0 + (lp - r * T_TW));
            const bool big = __ldcg(ws.area + root) >= min_area;
            surv = big && __ldcg(ws.first + root) == gf;
            if (root == node && !big) ws.label[node] = 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, surv);
        if (lane == 0) G.red[warp] = __popc(bal);
        __syncthreads();
        int before = chunk0, total = chunk0;
        for (int w = 0; w < G_WARPS; w++) {
            if (w < warp) before += G.red[w];
            total += G.red[w];
        }
        if (k < nk) ws.pk[tile * T_CAP + k] = surv ? before + __popc(bal & ((1u << lane) - 1u)) : -1;
        if (surv) atomicAdd(&G.cnt[r], 1);
        __syncthreads();
        chunk0 = total;
    }
    if (threadIdx.x < T_TH) ws.rowcnt[tile * T_TH + threadIdx.x] = G.cnt[threadIdx.x];
    if (threadIdx.x == 0 && chunk0 > 0) atomicAdd(&ws.trcnt[ty], chunk0);
    __syncthreads();
}

// ccl_scan_row: one tile row, block-wide.  Exclusive scan of the (row, tile)
// survivor counts in raster order; each (tile, row) entry of rowcnt is replaced
// by the label offset of its survivors: (survivors of earlier tile rows) +
// (scan value) - (the tile's survivors in earlier rows).  `sm` holds 2 T_TH ntx ints.
__device__ void ccl_scan_row(const CclWs& ws, GShared& G, int* sm, int ty, int ntx, int nty, int32_t* n_src_dev) {
    int* off = sm;                   // [T_TH][ntx] counts, then their exclusive prefix
    int* rstart = sm + T_TH * ntx;   // [T_TH][ntx] survivors of the tile in earlier rows
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int base = 0;  // survivors of earlier tile rows
    for (int t = threadIdx.x; t < ty; t += G_THREADS) base += __ldcg(ws.trcnt + t);
    base = __reduce_add_sync(0xffffffffu, base);
    if (lane == 0) G.red[warp] = base;
    for (int i = threadIdx.x; i < T_TH * ntx; i += G_THREADS) {
        const int r = i / ntx, tx = i - r * ntx;
        off[i] = __ldcg(ws.rowcnt + (int64_t)(ty * ntx + tx) * T_TH + r);
    }
    if (threadIdx.x == 0) G.carry = 0;
    __syncthreads();
    base = 0;
    for (int w = 0; w < G_WARPS; w++) base += G.red[w];
    for (int tx = threadIdx.x; tx < ntx; tx += G_THREADS) {
        int acc = 0;
        for (int r = 0; r < T_TH; r++) { rstart[r * ntx + tx] = acc; acc += off[r * ntx + tx]; }
    }
    __syncthreads();
    for (int c0 = 0; c0 < T_TH * ntx; c0 += G_THREADS) {
        const int i = c0 + threadIdx.x;
        const int v = i < T_TH * ntx ? off[i] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) G.red[warp] = inc;
        __syncthreads();
        int before = G.carry;
        for (int w = 0; w < warp; w++) before += G.red[w];
        if (i < T_TH * ntx) off[i] = before + inc - v;
        __syncthreads();
        if (threadIdx.x == G_THREADS - 1) G.carry = before + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0 && ty == nty - 1) *n_src_dev = base + G.carry;
    for (int i = threadIdx.x; i < T_TH * ntx; i += G_THREADS) {
        const int r = i / ntx, tx = i - r * ntx;
        ws.rowcnt[(int64_t)(ty * ntx + tx) * T_TH + r] = base + off[i] - rstart[i];
    }
    __syncthreads();
}

// a home survivor writes its component's label (offset + rank + 1) and its
// catalog entry
__device__ __forceinline__ void ccl_emit_node(const CclWs& ws, int node, int32_t max_src, const ipp_src_stats& out) {
    const int p = __ldcg(ws.pk + node);
    if (p < 0) return;
    const int tile = node / T_CAP;
    const int r = __ldcg(ws.lpos + node) / T_TW;
    const int lab = __ldcg(ws.rowcnt + (int64_t)tile * T_TH + r) + p + 1;
    const int root = __ldcg(ws.parent + node);
    ws.label[root] = lab;
    if (lab <= max_src) {
        const int k = lab - 1;
        out.area[k] = __ldcg(ws.area + root);
        out.first[k] = (int64_t)__ldcg(ws.first + root);
        out.xmin[k] = __ldcg(ws.xmin + root);
        out.xmax[k] = __ldcg(ws.xmax + root);
        out.ymin[k] = __ldcg(ws.ymin + root);
        out.ymax[k] = __ldcg(ws.ymax + root);
        out.peak[k] = fkey_inv(__ldcg(ws.peak + root));
        // flux and barycentre from the exact sums, in double-float
        const df dsm = fx_value(ws.sum + 2 * root);
        out.flux[k] = __fadd_rn(dsm.hi, dsm.lo);
        const df bx = df_div(fx_value(ws.sx + 2 * root), dsm);
        const df by = df_div(fx_value(ws.sy + 2 * root), dsm);
        out.xbar[k] = __fadd_rn(bx.hi, bx.lo);
        out.ybar[k] = __fadd_rn(by.hi, by.lo);
    }
}

// expand one tile's runs into the label map (0 for background and dropped
// components), writing every pixel once, coalesced; `lab` holds T_TH x T_TW ints
__device__ void ccl_final_tile(const CclWs& ws, int32_t* lab, int tile, int64_t W, int64_t H, int ntx,
                               int32_t* labels) {
    const int ty = tile / ntx, tx = tile - ty * ntx;
    const int64_t tx0 = (int64_t)tx * T_TW, ty0 = (int64_t)ty * T_TH;
    int4* l4 = reinterpret_cast<int4*>(lab);
    for (int t = threadIdx.x; t < T_TH * T_TW / 4; t += G_THREADS) l4[t] = make_int4(0, 0, 0, 0);
    __syncthreads();
    const int nr = __ldcg(ws.nruns + tile);
    for (int i = threadIdx.x; i < nr; i += G_THREADS) {
        const int node = __ldcg(ws.run_node + (int64_t)tile * T_RCAP + i);
        if (node < 0) continue;
        const int v = __ldcg(ws.label + __ldcg(ws.parent + node));
        if (v == 0) continue;
        const uint32_t rr = __ldcg(ws.runs + (int64_t)tile * T_RCAP + i);
        const int r = rr >> 16, st = (rr >> 8) & 0xff, en = rr & 0xff;
        for (int c = st; c <= en; c++) lab[r * T_TW + c] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t xc = tx0 + lane * 4;
    const bool vec = (W % 4 == 0) && (((uintptr_t)labels & 15) == 0) && (xc + 4 <= W);
    for (int r = warp; r < T_TH; r += G_WARPS) {
        const int64_t y = ty0 + r;
        if (y >= H || xc >= W) continue;
        const int4 o = *reinterpret_cast<const int4*>(&lab[r * T_TW + lane * 4]);
        if (vec) {
            *reinterpret_cast<int4*>(labels + y * W + xc) = o;
        } else {
            const int vals[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (xc + c < W) labels[y * W + xc + c] = vals[c];
        }
    }
    __syncthreads();
}


// ---- the global phase: one launch per step ------------------------------------
// (Folding these into one cooperative persistent kernel with grid-wide barriers
// was measured slower: each barrier added 3-5 us, and a cooperative launch,
// which needs all its blocks resident at once, stops the labeling of one frame
// from overlapping the kernels of frames on other streams.)
__global__ void __launch_bounds__(G_THREADS) k_ccl_union(CclWs ws, int ntx, int nty) {
    ccl_union_tile(ws, blockIdx.x, ntx, nty);
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_resolve(CclWs ws) {
    const int n = __ldcg(ws.counters);
    for (int t = blockIdx.x * G_THREADS + threadIdx.x; t < n; t += gridDim.x * G_THREADS)
        ccl_resolve_node(ws, __ldcg(ws.klist + t));
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_count(CclWs ws, int64_t W, int ntx, int min_area) {
    __shared__ GShared G;
    ccl_count_tile(ws, G, blockIdx.x, W, ntx, min_area);
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_scan(CclWs ws, int ntx, int nty, int32_t* n_src_dev) {
    extern __shared__ __align__(16) int g_sm[];   // 2 T_TH ntx ints
    __shared__ GShared G;
    ccl_scan_row(ws, G, g_sm, blockIdx.x, ntx, nty, n_src_dev);
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_emit(CclWs ws, int32_t max_src, ipp_src_stats out) {
    const int n = __ldcg(ws.counters);
    for (int t = blockIdx.x * G_THREADS + threadIdx.x; t < n; t += gridDim.x * G_THREADS)
        ccl_emit_node(ws, __ldcg(ws.klist + t), max_src, out);
}

__global__ void __launch_bounds__(G_THREADS) k_tile_final(CclWs ws, int64_t W, int64_t H, int ntx, int32_t* labels) {
    __shared__ __align__(16) int32_t lab[T_TH * T_TW];
    ccl_final_tile(ws, lab, blockIdx.x, W, H, ntx, labels);
}

// The same pass with the natural-spline reading of the interpolation (the
// interp option of the mesh parameters): B and rms from the node tables
// {f, Mx, My, Mxy} of the filtered mesh grids (k_spline_nodes), a thread per 4
// pixels of a row, 8 rows per 256-thread block; the mask nibbles of 8 lanes
// make one 32-bit word.
__global__ void __launch_bounds__(256) k_sub_thresh_spline(SubThreshJob T, const float4* nb, const float4* nr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t y = (int64_t)blockIdx.y * 8 + warp;
    if (y >= T.H) return;                                   // uniform over the warp
    const int64_t x0 = ((int64_t)blockIdx.x * 32 + lane) * 4;
    const float v = ((float)y + 0.5f) / T.mesh_h - 0.5f;
    unsigned nib = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int64_t x = x0 + c;
        if (x >= T.W) break;
        const float u = ((float)x + 0.5f) / T.mesh_w - 0.5f;
        float s;
        if (T.fused) {
            float f;
            if (T.dtype == IPP_F32) {
                f = __ldg(reinterpret_cast<const float*>(T.img) + y * T.pitch + x);
            } else {
                const float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(T.img) + y * T.pitch + x);
                const float b = T.bias_map ? __ldg(T.bias_map + y * T.W + x) : T.bias;
                f = (raw - b) * __ldg(T.inv_flat + y * T.W + x);
            }
            s = f - spline_at(nb, T.nx, T.ny, u, v);
            T.sub[y * T.sub_pitch + x] = s;
        } else {
            s = T.sub[y * T.sub_pitch + x];
        }
        const float thr = fmaxf(T.k * spline_at(nr, T.nx, T.ny, u, v), T.thresh_abs);
        if (s > thr) nib |= 1u << c;
    }
    unsigned word = nib << (4 * (lane & 7));
    word |= __shfl_xor_sync(0xffffffffu, word, 1);
    word |= __shfl_xor_sync(0xffffffffu, word, 2);
    word |= __shfl_xor_sync(0xffffffffu, word, 4);
    const int64_t wi = (x0 >> 5);
    if ((lane & 7) == 0 && wi < T.mw) T.mask[y * T.mw + wi] = word;
}

// ---- batched form: the same bodies over a table of frames ------------------
struct CclJob {
    CclWs ws;
    int ntx, nty;
    int64_t W, H;
    int min_area;
    int32_t* n_src_dev;
    int32_t max_src;
    ipp_src_stats stats;
    int32_t* labels;
};
struct ZeroJob {
    int32_t* p;
    int words;
};

#define IPP_MULTI_FRAME(bs, nf) \
    const int f_ = frame_of(bs, nf, blockIdx.x); \
    const int vb = blockIdx.x - bs[f_], nvb = bs[f_ + 1] - bs[f_];

__global__ void __launch_bounds__(256) k_zero_multi(const ZeroJob* Z, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    (void)vb; (void)nvb;
    for (int i = threadIdx.x; i < Z[f_].words; i += 256) Z[f_].p[i] = 0;
}

__global__ void __launch_bounds__(ST_THREADS, 4) k_sub_thresh_poly_multi(const SubThreshJob* T, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    (void)nvb;
    const int gx = (int)cdiv(T[f_].W, ST_TW);
    sub_thresh_poly_body(T[f_], vb % gx, vb / gx);
}

__global__ void __launch_bounds__(ST_THREADS, 4) k_sub_thresh_multi(const SubThreshJob* T, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    (void)nvb;
    const int gx = (int)cdiv(T[f_].W, ST_TW);
    sub_thresh_body(T[f_], vb % gx, vb / gx);
}

__global__ void __launch_bounds__(T_THREADS) k_tile_label_multi(const TileJob* J, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    (void)nvb;
    tile_label_fast(J[f_], vb);
}

__global__ void __launch_bounds__(T_THREADS) k_tile_label_full_multi(const TileJob* J, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    tile_label_full(J[f_], vb, nvb);
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_union_multi(const CclJob* C, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    (void)nvb;
    ccl_union_tile(C[f_].ws, vb, C[f_].ntx, C[f_].nty);
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_resolve_multi(const CclJob* C, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    const CclWs& ws = C[f_].ws;
    const int n = __ldcg(ws.counters);
    for (int t = vb * G_THREADS + threadIdx.x; t < n; t += nvb * G_THREADS) ccl_resolve_node(ws, __ldcg(ws.klist + t));
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_count_multi(const CclJob* C, const int* bs, int nf) {
    __shared__ GShared G;
    IPP_MULTI_FRAME(bs, nf)
    (void)nvb;
    ccl_count_tile(C[f_].ws, G, vb, C[f_].W, C[f_].ntx, C[f_].min_area);
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_scan_multi(const CclJob* C, const int* bs, int nf) {
    extern __shared__ __align__(16) int g_sm[];   // 2 T_TH ntx ints of the widest frame
    __shared__ GShared G;
    IPP_MULTI_FRAME(bs, nf)
    (void)nvb;
    ccl_scan_row(C[f_].ws, G, g_sm, vb, C[f_].ntx, C[f_].nty, C[f_].n_src_dev);
}

__global__ void __launch_bounds__(G_THREADS) k_ccl_emit_multi(const CclJob* C, const int* bs, int nf) {
    IPP_MULTI_FRAME(bs, nf)
    const CclJob& c = C[f_];
    const int n = __ldcg(c.ws.counters);
    for (int t = vb * G_THREADS + threadIdx.x; t < n; t += nvb * G_THREADS)
        ccl_emit_node(c.ws, __ldcg(c.ws.klist + t), c.max_src, c.stats);
}

__global__ void __launch_bounds__(G_THREADS) k_tile_final_multi(const CclJob* C, const int* bs, int nf) {
    __shared__ __align__(16) int32_t lab[T_TH * T_TW];
    IPP_MULTI_FRAME(bs, nf)
    (void)nvb;
    ccl_final_tile(C[f_].ws, lab, vb, C[f_].W, C[f_].H, C[f_].ntx, C[f_].labels);
}

}  // namespace ipp

// ------------------------------------------------------------------ host side
using namespace ipp;

struct CclLayout {
    int ntx, nty;
    int64_t ntiles, nodes, runs;
    size_t off[28];
    size_t total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static CclLayout ccl_layout(int64_t W, int64_t H) {
    CclLayout L;
    L.ntx = (int)cdiv(W, T_TW);
    L.nty = (int)cdiv(H, T_TH);
    L.ntiles = (int64_t)L.ntx * L.nty;
    L.nodes = L.ntiles * T_CAP;
    L.runs = L.ntiles * T_RCAP;
    const size_t sizes[] = {
        (size_t)L.ntiles * 4, (size_t)L.ntiles * 4,            // nkept nruns
        (size_t)L.runs * 4, (size_t)L.runs * 4,                // runs run_node
        (size_t)L.nodes * 4, (size_t)L.nodes * 4,              // parent, area
        (size_t)L.nodes * 8, (size_t)L.nodes * 4,              // first, peak
        (size_t)L.nodes * 4, (size_t)L.nodes * 4, (size_t)L.nodes * 4, (size_t)L.nodes * 4,  // bbox
        (size_t)L.nodes * 16, (size_t)L.nodes * 16, (size_t)L.nodes * 16,  // sum sx sy (integer pairs)
        (size_t)L.nodes * 4,                                   // label
        (size_t)L.ntiles * T_TW * 4, (size_t)L.ntiles * T_TW * 4,  // btop bbot
        (size_t)L.ntiles * T_TH * 4, (size_t)L.ntiles * T_TH * 4,  // blef brig
        (size_t)(L.nty + CT_WORDS) * 4,                        // counters + trcnt
        (size_t)L.nodes * 4,                                   // klist
        (size_t)L.nodes * 4, (size_t)L.nodes * 4,              // lpos, pk
        (size_t)cdiv(W, 32) * (size_t)H * 4,                   // detection bit rows
        (size_t)L.ntiles * T_TH * 4,                           // rowcnt
        (size_t)L.ntiles * 4,                                  // ovf
    };
    size_t o = 0;
    for (int k = 0; k < 27; k++) { L.off[k] = o; o += align256(sizes[k]); }
    L.total = o;
    return L;
}

static CclWs ccl_ws(const CclLayout& L, void* ws) {
    unsigned char* b = (unsigned char*)ws;
    CclWs w;
    w.nkept = (int32_t*)(b + L.off[0]);
    w.nruns = (int32_t*)(b + L.off[1]);
    w.runs = (uint32_t*)(b + L.off[2]);
    w.run_node = (int32_t*)(b + L.off[3]);
    w.parent = (int32_t*)(b + L.off[4]);
    w.area = (int32_t*)(b + L.off[5]);
    w.first = (unsigned long long*)(b + L.off[6]);
    w.peak = (uint32_t*)(b + L.off[7]);
    w.xmin = (int32_t*)(b + L.off[8]);
    w.xmax = (int32_t*)(b + L.off[9]);
    w.ymin = (int32_t*)(b + L.off[10]);
    w.ymax = (int32_t*)(b + L.off[11]);
    w.sum = (long long*)(b + L.off[12]);
    w.sx = (long long*)(b + L.off[13]);
    w.sy = (long long*)(b + L.off[14]);
    w.label = (int32_t*)(b + L.off[15]);
    w.btop = (int32_t*)(b + L.off[16]);
    w.bbot = (int32_t*)(b + L.off[17]);
    w.blef = (int32_t*)(b + L.off[18]);
    w.brig = (int32_t*)(b + L.off[19]);
    w.counters = (int32_t*)(b + L.off[20]);
    w.trcnt = w.counters + CT_WORDS;
    w.klist = (int32_t*)(b + L.off[21]);
    w.lpos = (int32_t*)(b + L.off[22]);
    w.pk = (int32_t*)(b + L.off[23]);
    w.rowcnt = (int32_t*)(b + L.off[25]);
    w.ovf = (int32_t*)(b + L.off[26]);
    return w;
}

size_t ipp_ccl_workspace_size(int64_t W, int64_t H) { return ccl_layout(W, H).total; }


int ipp_launch_detect(const DetectArgs& A, cudaStream_t s) {
    CclLayout L = ccl_layout(A.W, A.H);
    if (L.nodes >= (int64_t)INT32_MAX) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "frame too large for 32-bit node ids");
    CclWs w = ccl_ws(L, A.ws);
    TileJob J;
    J.W = A.W; J.H = A.H; J.ntx = L.ntx; J.nty = L.nty;
    J.sub = A.sub; J.sub_pitch = A.sub_pitch;
    J.mw = cdiv(A.W, 32);
    J.min_area = A.min_area;
    J.ws = w;
    if (A.mode == MODE_MASK) {
        J.mask = A.mask_in;
    } else {  // subtract (fused) and threshold into the workspace's bit rows
        SubThreshJob T;
        T.W = A.W; T.H = A.H; T.fused = A.mode == MODE_FUSED;
        T.img = A.img; T.dtype = A.dtype; T.pitch = A.pitch;
        T.bias_map = A.bias_map; T.bias = A.bias; T.inv_flat = A.inv_flat;
        T.mesh_bkg = A.mesh_bkg; T.sub = A.sub; T.sub_pitch = A.sub_pitch;
        T.mesh_rms = A.mesh_rms; T.nx = A.nx; T.ny = A.ny; T.mesh_w = A.mesh_w; T.mesh_h = A.mesh_h;
        T.k = A.k; T.thresh_abs = A.thresh_abs; T.filter = false;
        T.mask = (uint32_t*)((unsigned char*)A.ws + L.off[24]);
        T.mw = J.mw;
        dim3 sg((unsigned)cdiv(A.W, ST_TW), (unsigned)cdiv(A.H, ST_TH));
        if (A.interp == 1) {
            if (A.filter) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "detection filter with the spline reading");
            if (!A.bnodes || !A.rnodes) return ipp_set_error(IPP_ERR_INVALID_ARG, "spline node tables missing");
            dim3 spg((unsigned)cdiv(A.W, 128), (unsigned)cdiv(A.H, 8));
            k_sub_thresh_spline<<<spg, 256, 0, s>>>(T, A.bnodes, A.rnodes);
        } else if (A.mesh_w >= 16) {
            k_sub_thresh_poly<<<sg, ST_THREADS, 0, s>>>(T);
        } else {
            k_sub_thresh<<<sg, ST_THREADS, 0, s>>>(T);
        }
        if (int e = ipp_check_launch("k_sub_thresh")) return e;
        if (A.filter) {  // detection filter: threshold again, on the smoothed sub just written
            SubThreshJob Tf = T;
            Tf.fused = false;
            Tf.filter = true;
            k_sub_thresh<<<sg, ST_THREADS, 0, s>>>(Tf);
            if (int e = ipp_check_launch("k_sub_thresh (filtered)")) return e;
        }
        J.mask = T.mask;
    }
    cudaFuncSetAttribute(k_tile_label, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileFast));
    cudaFuncSetAttribute(k_tile_label_full, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileFull));
    dim3 tg(L.ntx, L.nty);
    // the kept-node counter, the overflow count and the per-tile-row counts start at zero
    if (cudaMemsetAsync(w.counters, 0, (size_t)(L.nty + CT_WORDS) * 4, s) != cudaSuccess) return ipp_check_launch("memset");
    k_tile_label<<<tg, T_THREADS, sizeof(TileFast), s>>>(J);
    if (int e = ipp_check_launch("k_tile_label")) return e;
    {
        int dev0 = 0, nsm = 0;
        cudaGetDevice(&dev0);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev0);
        const int64_t fg = std::min<int64_t>(L.ntiles, (int64_t)std::max(nsm, 1) * 4);
        k_tile_label_full<<<(unsigned)fg, T_THREADS, sizeof(TileFull), s>>>(J);
        if (int e = ipp_check_launch("k_tile_label_full")) return e;
    }
    const unsigned nt = (unsigned)L.ntiles;
    k_ccl_union<<<nt, G_THREADS, 0, s>>>(w, L.ntx, L.nty);
    if (int e = ipp_check_launch("k_ccl_union")) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned pg = (unsigned)std::max(sms, 1) * 4;  // grid-stride over the kept nodes
    k_ccl_resolve<<<pg, G_THREADS, 0, s>>>(w);
    if (int e = ipp_check_launch("k_ccl_resolve")) return e;
    k_ccl_count<<<nt, G_THREADS, 0, s>>>(w, A.W, L.ntx, A.min_area);
    if (int e = ipp_check_launch("k_ccl_count")) return e;
    const size_t lsm = (size_t)2 * T_TH * L.ntx * sizeof(int);
    if (lsm > 200 * 1024) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "frame too wide for the labeling pass");
    cudaFuncSetAttribute(k_ccl_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
    k_ccl_scan<<<L.nty, G_THREADS, lsm, s>>>(w, L.ntx, L.nty, A.n_src_dev);
    if (int e = ipp_check_launch("k_ccl_scan")) return e;
    k_ccl_emit<<<pg, G_THREADS, 0, s>>>(w, A.max_src, A.stats);
    if (int e = ipp_check_launch("k_ccl_emit")) return e;
    k_tile_final<<<nt, G_THREADS, 0, s>>>(w, A.W, A.H, L.ntx, A.labels);
    return ipp_check_launch("k_tile_final");
}

// ---- batched form: tables and launches ----------------------------------------
int ipp_detect_multi_pack(const DetectArgs* A, int nf, HostBlob& hb, DetMultiPlan* p) {
    if (nf < 1 || nf > 1024) return ipp_set_error(IPP_ERR_INVALID_ARG, "1..1024 frames");
    std::vector<SubThreshJob> T(nf), Tf(nf);
    std::vector<TileJob> J(nf);
    std::vector<CclJob> C(nf);
    std::vector<ZeroJob> Z(nf);
    std::vector<int> nb(nf);
    int max_ntx = 0;
    p->poly = true;
    p->filter = A[0].filter != 0;
    for (int f = 0; f < nf; f++) {
        const DetectArgs& a = A[f];
        if (a.mode == MODE_MASK) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "batched detection from a mask");
        if (a.interp != 0) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "the table form with the spline reading");
        if ((a.filter != 0) != p->filter) return ipp_set_error(IPP_ERR_INVALID_ARG, "mixed detection filters");
        const CclLayout L = ccl_layout(a.W, a.H);
        if (L.nodes >= (int64_t)INT32_MAX) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "frame too large");
        const CclWs w = ccl_ws(L, a.ws);
        SubThreshJob& t = T[f];
        t.W = a.W; t.H = a.H; t.fused = a.mode == MODE_FUSED;
        t.img = a.img; t.dtype = a.dtype; t.pitch = a.pitch;
        t.bias_map = a.bias_map; t.bias = a.bias; t.inv_flat = a.inv_flat;
        t.mesh_bkg = a.mesh_bkg; t.sub = a.sub; t.sub_pitch = a.sub_pitch;
        t.mesh_rms = a.mesh_rms; t.nx = a.nx; t.ny = a.ny; t.mesh_w = a.mesh_w; t.mesh_h = a.mesh_h;
        t.k = a.k; t.thresh_abs = a.thresh_abs; t.filter = false;
        t.mask = (uint32_t*)((unsigned char*)a.ws + L.off[24]);
        t.mw = (int)cdiv(a.W, 32);
        Tf[f] = t;
        Tf[f].fused = false;
        Tf[f].filter = true;
        p->poly = p->poly && a.mesh_w >= 16;
        TileJob& j = J[f];
        j.W = a.W; j.H = a.H; j.ntx = L.ntx; j.nty = L.nty;
        j.sub = a.sub; j.sub_pitch = a.sub_pitch; j.mw = t.mw; j.min_area = a.min_area;
        j.ws = w; j.mask = t.mask;
        CclJob& c = C[f];
        c.ws = w; c.ntx = L.ntx; c.nty = L.nty; c.W = a.W; c.H = a.H; c.min_area = a.min_area;
        c.n_src_dev = a.n_src_dev; c.max_src = a.max_src; c.stats = a.stats; c.labels = a.labels;
        Z[f].p = w.counters;
        Z[f].words = L.nty + CT_WORDS;
        max_ntx = std::max(max_ntx, L.ntx);
    }
    for (int f = 0; f < nf; f++) nb[f] = 1;
    p->zero = ipp_put_stage(hb, Z.data(), nb.data(), nf);
    for (int f = 0; f < nf; f++) nb[f] = (int)(cdiv(T[f].W, ST_TW) * cdiv(T[f].H, ST_TH));
    p->thresh = ipp_put_stage(hb, T.data(), nb.data(), nf);
    if (p->filter) p->filt = ipp_put_stage(hb, Tf.data(), nb.data(), nf);
    for (int f = 0; f < nf; f++) nb[f] = J[f].ntx * J[f].nty;
    p->tile = ipp_put_stage(hb, J.data(), nb.data(), nf);
    for (int f = 0; f < nf; f++) nb[f] = std::min(J[f].ntx * J[f].nty, 8);
    p->tile_full = ipp_put_stage(hb, J.data(), nb.data(), nf);
    for (int f = 0; f < nf; f++) nb[f] = C[f].ntx * C[f].nty;
    p->unions = ipp_put_stage(hb, C.data(), nb.data(), nf);
    p->count = p->unions;
    p->fin = p->unions;
    for (int f = 0; f < nf; f++) nb[f] = std::max(1, (C[f].ntx * C[f].nty + 3) / 4);
    p->resolve = ipp_put_stage(hb, C.data(), nb.data(), nf);
    p->emit = p->resolve;
    for (int f = 0; f < nf; f++) nb[f] = C[f].nty;
    p->scan = ipp_put_stage(hb, C.data(), nb.data(), nf);
    p->scan_smem = (size_t)2 * T_TH * max_ntx * sizeof(int);
    if (p->scan_smem > 200 * 1024) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "frame too wide for the labeling pass");
    p->nf = nf;
    return hb.ok() ? IPP_OK : ipp_set_error(IPP_ERR_INVALID_ARG, "batch table overflow");
}

int ipp_detect_multi_launch(const DetMultiPlan& p, const unsigned char* t, cudaStream_t s) {
#define IPP_TAB(st, T) reinterpret_cast<const T*>(t + p.st.jobs), reinterpret_cast<const int*>(t + p.st.bs), p.nf
    cudaFuncSetAttribute(k_tile_label_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileFast));
    cudaFuncSetAttribute(k_tile_label_full_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileFull));
    cudaFuncSetAttribute(k_ccl_scan_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.scan_smem);
    k_zero_multi<<<(unsigned)p.zero.total, 256, 0, s>>>(IPP_TAB(zero, ZeroJob));
    if (int e = ipp_check_launch("k_zero_multi")) return e;
    if (p.poly) k_sub_thresh_poly_multi<<<(unsigned)p.thresh.total, ST_THREADS, 0, s>>>(IPP_TAB(thresh, SubThreshJob));
    else k_sub_thresh_multi<<<(unsigned)p.thresh.total, ST_THREADS, 0, s>>>(IPP_TAB(thresh, SubThreshJob));
    if (int e = ipp_check_launch("k_sub_thresh_multi")) return e;
    if (p.filter) {
        k_sub_thresh_multi<<<(unsigned)p.filt.total, ST_THREADS, 0, s>>>(IPP_TAB(filt, SubThreshJob));
        if (int e = ipp_check_launch("k_sub_thresh_multi (filtered)")) return e;
    }
    k_tile_label_multi<<<(unsigned)p.tile.total, T_THREADS, sizeof(TileFast), s>>>(IPP_TAB(tile, TileJob));
    if (int e = ipp_check_launch("k_tile_label_multi")) return e;
    k_tile_label_full_multi<<<(unsigned)p.tile_full.total, T_THREADS, sizeof(TileFull), s>>>(
        IPP_TAB(tile_full, TileJob));
    if (int e = ipp_check_launch("k_tile_label_full_multi")) return e;
    k_ccl_union_multi<<<(unsigned)p.unions.total, G_THREADS, 0, s>>>(IPP_TAB(unions, CclJob));
    if (int e = ipp_check_launch("k_ccl_union_multi")) return e;
    k_ccl_resolve_multi<<<(unsigned)p.resolve.total, G_THREADS, 0, s>>>(IPP_TAB(resolve, CclJob));
    if (int e = ipp_check_launch("k_ccl_resolve_multi")) return e;
    k_ccl_count_multi<<<(unsigned)p.count.total, G_THREADS, 0, s>>>(IPP_TAB(count, CclJob));
    if (int e = ipp_check_launch("k_ccl_count_multi")) return e;
    k_ccl_scan_multi<<<(unsigned)p.scan.total, G_THREADS, p.scan_smem, s>>>(IPP_TAB(scan, CclJob));
    if (int e = ipp_check_launch("k_ccl_scan_multi")) return e;
    k_ccl_emit_multi<<<(unsigned)p.emit.total, G_THREADS, 0, s>>>(IPP_TAB(emit, CclJob));
    if (int e = ipp_check_launch("k_ccl_emit_multi")) return e;
    k_tile_final_multi<<<(unsigned)p.fin.total, G_THREADS, 0, s>>>(IPP_TAB(fin, CclJob));
#undef IPP_TAB
    return ipp_check_launch("k_tile_final_multi");
}
