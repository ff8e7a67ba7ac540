// detect.cu -- pixel detection and connection into candidates, with the
// per-candidate pre-analysis of Sec. 2.2.5 (peak, total flux, ...).
//
// Tiles of TH x TW pixels.  k_tile_label thresholds a tile (or takes a given
// mask), packs it into bits, labels it with a shared-memory union-find whose
// roots are the smallest local raster index, and emits one node per component
// that touches the tile border or is large enough, with its partial stats.
// Border pixels record their node.  The global phase unites nodes across tile
// seams, folds the stats into the roots, keeps roots of at least min_area pixels
// and numbers them by the raster index of their first pixel (per-row counts,
// an exclusive scan, a rank inside each row).  k_tile_final re-derives the
// identical local labels from the bit mask and writes the label map once.
// Nothing depends on the tile shape except the work split.
#include "jobs.cuh"

namespace ipp {

constexpr int T_TH = 32, T_TW = 128;
constexpr int T_WPR = T_TW / 32;                 // mask words per tile row
constexpr int T_WORDS = T_TH * T_WPR;            // 128
constexpr int T_PIX = T_TH * T_TW;               // 4096
constexpr int T_CAP = (T_TH / 2) * (T_TW / 2);   // max 8-connected components in a tile
constexpr int T_THREADS = 256;
constexpr int T_NQ = 40;

enum TileMode { MODE_SUB_THRESH = 0, MODE_MASK = 1, MODE_FUSED = 2 };

// Global scratch of the labeling (all indices by node = tile * T_CAP + cid).
struct CclWs {
    uint32_t* mask;      // padded bit mask: (nty*T_TH) rows x (ntx*T_WPR) words
    int32_t* ncomp;      // [ntiles]
    int32_t* parent;     // [ntiles*T_CAP], -1 = dropped component
    int32_t* area;
    unsigned long long* first;
    uint32_t* peak;      // order-preserving key
    int32_t* xmin; int32_t* xmax; int32_t* ymin; int32_t* ymax;
    double* sum; double* sx; double* sy;
    int32_t* label;
    int32_t* btop; int32_t* bbot;    // [ntiles*T_TW]
    int32_t* blef; int32_t* brig;    // [ntiles*T_TH]
    int32_t* rowcnt; int32_t* rowfill; int32_t* rowbase;  // [H], [H], [H+1]
    unsigned long long* slist_first; int32_t* slist_node;  // [ntiles*T_CAP]
};

struct TileJob {
    int mode;
    int64_t W, H;
    int ntx, nty;
    // MODE_FUSED input
    const void* img; int dtype; int64_t pitch;
    const float* bias_map; float bias; const float* inv_flat;
    const float* mesh_bkg;
    // sub: input (SUB_THRESH / MASK) or output (FUSED)
    float* sub; int64_t sub_pitch;
    const float* mesh_rms;
    int nx, ny, mesh_w, mesh_h;
    float k, thresh_abs;
    int min_area;
    const uint32_t* mask_in;  // MODE_MASK: row stride ceil(W/32) words
    CclWs ws;
};

struct TileShared {
    uint32_t mask[T_TH][T_WPR];
    int32_t lab[T_PIX];
    uint32_t rootw[T_WORDS];
    int32_t rootpre[T_WORDS];
    int32_t nc;
    int32_t c_area[T_CAP];
    uint32_t c_peak[T_CAP];
    double c_sum[T_CAP], c_sx[T_CAP], c_sy[T_CAP];
    int32_t c_xmin[T_CAP], c_xmax[T_CAP], c_ymin[T_CAP], c_ymax[T_CAP];
    int32_t c_border[T_CAP];
    int32_t c_root[T_CAP];
    float cvb[T_TH][T_NQ];
    float cvr[T_TH][T_NQ];
};

__device__ __forceinline__ int lfind(const int32_t* L, int x) {
    int p = L[x];
    while (p != x) { x = p; p = L[x]; }
    return x;
}
// lock-free union by atomicMin: the larger root is linked under the smaller
__device__ __forceinline__ void lunite(int32_t* L, int a, int b) {
    while (true) {
        a = lfind(L, a);
        b = lfind(L, b);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicMin(&L[b], a);
        if (old == b) return;
        b = old;
    }
}
__device__ __forceinline__ bool mbit(const TileShared& S, int r, int c) {
    return (S.mask[r][c >> 5] >> (c & 31)) & 1u;
}

// Local union-find over the bit mask in S.mask, then compaction of the roots
// (component ids in raster order of their roots).  Identical in both tile
// passes, so component ids agree.
__device__ void tile_ccl(TileShared& S) {
    const int t = threadIdx.x;
    if (t < T_WORDS) {
        int r = t / T_WPR, wi = t % T_WPR;
        uint32_t bits = S.mask[r][wi];
        while (bits) {
            int b = __ffs(bits) - 1;
            bits &= bits - 1;
            int p = r * T_TW + wi * 32 + b;
            S.lab[p] = p;
        }
    }
    __syncthreads();
    if (t < T_WORDS) {
        int r = t / T_WPR, wi = t % T_WPR;
        uint32_t bits = S.mask[r][wi];
        while (bits) {
            int b = __ffs(bits) - 1;
            bits &= bits - 1;
            int c = wi * 32 + b, p = r * T_TW + c;
            if (c > 0 && mbit(S, r, c - 1)) lunite(S.lab, p, p - 1);
            if (r > 0) {
                if (mbit(S, r - 1, c)) {
                    lunite(S.lab, p, p - T_TW);
                } else {
                    if (c > 0 && mbit(S, r - 1, c - 1)) lunite(S.lab, p, p - T_TW - 1);
                    if (c < T_TW - 1 && mbit(S, r - 1, c + 1)) lunite(S.lab, p, p - T_TW + 1);
                }
            }
        }
    }
    __syncthreads();
    if (t < T_WORDS) {
        int r = t / T_WPR, wi = t % T_WPR;
        uint32_t bits = S.mask[r][wi], rb = 0;
        while (bits) {
            int b = __ffs(bits) - 1;
            bits &= bits - 1;
            int p = r * T_TW + wi * 32 + b;
            int root = lfind(S.lab, p);
            S.lab[p] = root;
            if (root == p) rb |= 1u << b;
        }
        S.rootw[t] = rb;
    }
    __syncthreads();
    if (t < 32) {  // exclusive popcount prefix over the 128 root words
        int c[4], tot = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) { c[k] = __popc(S.rootw[t * 4 + k]); tot += c[k]; }
        int inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (t >= o) inc += v;
        }
        int run = inc - tot;
#pragma unroll
        for (int k = 0; k < 4; k++) { S.rootpre[t * 4 + k] = run; run += c[k]; }
        if (t == 31) S.nc = inc;
    }
    __syncthreads();
}

__device__ __forceinline__ int cid_of(const TileShared& S, int root) {
    int w = root >> 5, b = root & 31;
    return S.rootpre[w] + __popc(S.rootw[w] & ((1u << b) - 1u));
}

__device__ __forceinline__ float tile_load_pix(const TileJob& J, int64_t y, int64_t x) {
    if (J.dtype == IPP_F32) return __ldg(reinterpret_cast<const float*>(J.img) + y * J.pitch + x);
    float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(J.img) + y * J.pitch + x);
    float b = J.bias_map ? __ldg(J.bias_map + y * J.W + x) : J.bias;
    return (raw - b) * __ldg(J.inv_flat + y * J.W + x);
}

__global__ void __launch_bounds__(T_THREADS, 3) k_tile_label(TileJob J) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileShared& S = *reinterpret_cast<TileShared*>(smem_raw);
    const int tx = blockIdx.x, ty = blockIdx.y, tile = ty * J.ntx + tx;
    const int64_t tx0 = (int64_t)tx * T_TW, ty0 = (int64_t)ty * T_TH;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t mpitch = (int64_t)J.ntx * T_WPR;

    // zero the per-row counters of the numbering (any block may do it)
    for (int64_t i = (int64_t)tile * T_THREADS + threadIdx.x; i < J.H; i += (int64_t)J.ntx * J.nty * T_THREADS) {
        J.ws.rowcnt[i] = 0;
        J.ws.rowfill[i] = 0;
    }

    // ---- phase A: values, threshold, bit mask ------------------------------
    const bool thresh = J.mode != MODE_MASK;
    const bool fused = J.mode == MODE_FUSED;
    int qbase = 0;
    float refb = 0.f, refr = 0.f;
    if (thresh) {
        const int qa = (int)floorf(((float)tx0 + 0.5f) / J.mesh_w - 0.5f) - 1;
        qbase = max(qa, 0);
        refr = J.mesh_rms[0];
        if (fused) refb = J.mesh_bkg[0];
        for (int t = threadIdx.x; t < T_TH * T_NQ; t += T_THREADS) {
            int r = t / T_NQ, qq = t - r * T_NQ;
            int q = min(qbase + qq, J.nx - 1);
            float vy = ((float)(ty0 + r) + 0.5f) / J.mesh_h - 0.5f;
            float pf = floorf(vy);
            float w[4];
            keys_weights(vy - pf, w);
            int p0 = (int)pf;
            float ab = 0.f, ar = 0.f;
#pragma unroll
            for (int a = 0; a < 4; a++) {
                int p = clampi(p0 - 1 + a, 0, J.ny - 1);
                ar = fmaf(w[a], J.mesh_rms[p * J.nx + q] - refr, ar);
                if (fused) ab = fmaf(w[a], J.mesh_bkg[p * J.nx + q] - refb, ab);
            }
            S.cvr[r][qq] = ar;
            S.cvb[r][qq] = ab;
        }
        __syncthreads();
    }
    {
        const int64_t xc = tx0 + lane * 4;
        float wx[4][4];
        int qi[4][4];
        if (thresh) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                float u = ((float)(xc + c) + 0.5f) / J.mesh_w - 0.5f;
                float qf = floorf(u);
                keys_weights(u - qf, wx[c]);
                int q0 = (int)qf;
#pragma unroll
                for (int b = 0; b < 4; b++) qi[c][b] = min(clampi(q0 - 1 + b, 0, J.nx - 1) - qbase, T_NQ - 1);
            }
        }
        const bool vin = (J.pitch % 4 == 0) && (((uintptr_t)J.img & 15) == 0) && J.dtype == IPP_F32;
        const bool vsub = (J.sub_pitch % 4 == 0) && (((uintptr_t)J.sub & 15) == 0);
        const bool full4 = xc + 4 <= J.W;
        for (int r = warp; r < T_TH; r += T_THREADS / 32) {
            const int64_t y = ty0 + r;
            uint32_t nib = 0;
            if (y < J.H && xc < J.W) {
                if (J.mode == MODE_MASK) {
                    const int64_t mw = (J.W + 31) / 32;
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        int64_t x = xc + c;
                        if (x < J.W && ((J.mask_in[y * mw + (x >> 5)] >> (x & 31)) & 1u)) nib |= 1u << c;
                    }
                } else {
                    float f[4];
                    if (fused) {
                        if (vin && full4) {
                            float4 t4 = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(J.img) + y * J.pitch + xc));
                            f[0] = t4.x; f[1] = t4.y; f[2] = t4.z; f[3] = t4.w;
                        } else {
#pragma unroll
                            for (int c = 0; c < 4; c++) f[c] = (xc + c < J.W) ? tile_load_pix(J, y, xc + c) : 0.f;
                        }
#pragma unroll
                        for (int c = 0; c < 4; c++) {
                            float acc = 0.f;
#pragma unroll
                            for (int b = 0; b < 4; b++) acc = fmaf(wx[c][b], S.cvb[r][qi[c][b]], acc);
                            f[c] = f[c] - (refb + acc);
                        }
                        if (vsub && full4) {
                            *reinterpret_cast<float4*>(J.sub + y * J.sub_pitch + xc) = make_float4(f[0], f[1], f[2], f[3]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 4; c++)
                                if (xc + c < J.W) J.sub[y * J.sub_pitch + xc + c] = f[c];
                        }
                    } else {
                        if (vsub && full4) {
                            float4 t4 = __ldg(reinterpret_cast<const float4*>(J.sub + y * J.sub_pitch + xc));
                            f[0] = t4.x; f[1] = t4.y; f[2] = t4.z; f[3] = t4.w;
                        } else {
#pragma unroll
                            for (int c = 0; c < 4; c++) f[c] = (xc + c < J.W) ? __ldg(J.sub + y * J.sub_pitch + xc + c) : 0.f;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        float acc = 0.f;
#pragma unroll
                        for (int b = 0; b < 4; b++) acc = fmaf(wx[c][b], S.cvr[r][qi[c][b]], acc);
                        float thr = fmaxf(J.k * (refr + acc), J.thresh_abs);
                        if (xc + c < J.W && f[c] > thr) nib |= 1u << c;
                    }
                }
            }
            // 8 lanes x 4 bits -> one 32-bit word
            uint32_t wv = nib << (4 * (lane & 7));
            wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
            wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
            wv |= __shfl_xor_sync(0xffffffffu, wv, 4);
            if ((lane & 7) == 0) S.mask[r][lane >> 3] = wv;
        }
    }
    __syncthreads();
    if (threadIdx.x < T_WORDS) {
        int r = threadIdx.x / T_WPR, wi = threadIdx.x % T_WPR;
        J.ws.mask[(ty0 + r) * mpitch + (int64_t)tx * T_WPR + wi] = S.mask[r][wi];
    }

    // ---- phase B/C: local components ---------------------------------------
    tile_ccl(S);
    const int nc = S.nc;
    for (int c = threadIdx.x; c < nc; c += T_THREADS) {
        S.c_area[c] = 0;
        S.c_peak[c] = 0u;
        S.c_sum[c] = 0.0; S.c_sx[c] = 0.0; S.c_sy[c] = 0.0;
        S.c_xmin[c] = T_TW; S.c_xmax[c] = -1; S.c_ymin[c] = T_TH; S.c_ymax[c] = -1;
        S.c_border[c] = 0;
    }
    __syncthreads();

    // ---- phase D: per-component partial stats -------------------------------
    // Each thread walks its word's pixels in order and aggregates runs of the
    // same component before one set of shared atomics per run; the sums are
    // FP64, so the result does not depend on the order of the atomics.
    if (threadIdx.x < T_WORDS) {
        const int r = threadIdx.x / T_WPR, wi = threadIdx.x % T_WPR;
        uint32_t bits = S.mask[r][wi];
        int cur = -1, n = 0, cmin = 0, cmax = 0;
        float s0 = 0.f, s1 = 0.f, pk = 0.f;
        bool border = false;
        auto flush = [&]() {
            if (cur < 0) return;
            atomicAdd(&S.c_area[cur], n);
            atomicAdd(&S.c_sum[cur], (double)s0);
            atomicAdd(&S.c_sx[cur], (double)s1);
            atomicAdd(&S.c_sy[cur], (double)s0 * (double)r);
            atomicMax(&S.c_peak[cur], fkey(pk));
            atomicMin(&S.c_xmin[cur], cmin);
            atomicMax(&S.c_xmax[cur], cmax);
            atomicMin(&S.c_ymin[cur], r);
            atomicMax(&S.c_ymax[cur], r);
            if (border) S.c_border[cur] = 1;
        };
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int col = wi * 32 + b, p = r * T_TW + col;
            const int root = S.lab[p];
            const int c = cid_of(S, root);
            if (root == p) S.c_root[c] = p;
            const float f = __ldcg(J.sub + (ty0 + r) * J.sub_pitch + tx0 + col);
            if (c != cur) {
                flush();
                cur = c; n = 0; s0 = 0.f; s1 = 0.f; pk = f; cmin = col; border = false;
            }
            n++;
            s0 += f;
            s1 = fmaf(f, (float)col, s1);
            pk = fmaxf(pk, f);
            cmax = col;
            border |= (r == 0 || r == T_TH - 1 || col == 0 || col == T_TW - 1);
        }
        flush();
    }
    __syncthreads();

    // ---- phase E: emit nodes --------------------------------------------------
    for (int c = threadIdx.x; c < nc; c += T_THREADS) {
        const int node = tile * T_CAP + c;
        const bool kept = S.c_border[c] || S.c_area[c] >= J.min_area;
        if (!kept) { J.ws.parent[node] = -1; continue; }
        const int root = S.c_root[c];
        const int rr = root / T_TW, rc = root % T_TW;
        J.ws.parent[node] = node;
        J.ws.area[node] = S.c_area[c];
        J.ws.first[node] = (unsigned long long)((ty0 + rr) * J.W + tx0 + rc);
        J.ws.peak[node] = S.c_peak[c];
        J.ws.xmin[node] = (int)tx0 + S.c_xmin[c];
        J.ws.xmax[node] = (int)tx0 + S.c_xmax[c];
        J.ws.ymin[node] = (int)ty0 + S.c_ymin[c];
        J.ws.ymax[node] = (int)ty0 + S.c_ymax[c];
        const double sm = S.c_sum[c];
        J.ws.sum[node] = sm;
        J.ws.sx[node] = S.c_sx[c] + (double)tx0 * sm;
        J.ws.sy[node] = S.c_sy[c] + (double)ty0 * sm;
    }
    if (threadIdx.x == 0) J.ws.ncomp[tile] = nc;

    // ---- phase F: node of each border pixel -----------------------------------
    for (int t = threadIdx.x; t < 2 * T_TW + 2 * T_TH; t += T_THREADS) {
        int r, c;
        int32_t* dst;
        if (t < T_TW) { r = 0; c = t; dst = J.ws.btop + (int64_t)tile * T_TW + c; }
        else if (t < 2 * T_TW) { r = T_TH - 1; c = t - T_TW; dst = J.ws.bbot + (int64_t)tile * T_TW + c; }
        else if (t < 2 * T_TW + T_TH) { r = t - 2 * T_TW; c = 0; dst = J.ws.blef + (int64_t)tile * T_TH + r; }
        else { r = t - 2 * T_TW - T_TH; c = T_TW - 1; dst = J.ws.brig + (int64_t)tile * T_TH + r; }
        *dst = mbit(S, r, c) ? tile * T_CAP + cid_of(S, S.lab[r * T_TW + c]) : -1;
    }
}

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

__global__ void k_ccl_union(CclWs ws, int ntx, int nty) {
    const int tx = blockIdx.x, ty = blockIdx.y, tile = ty * ntx + tx;
    const int t = threadIdx.x;  // 128 threads
    if (ty + 1 < nty) {  // bottom seam, including the diagonal corners
        const int below = tile + ntx;
        int a = __ldcg(ws.bbot + (int64_t)tile * T_TW + t);
        if (a >= 0) {
            for (int d = -1; d <= 1; d++) {
                int j = t + d;
                int b;
                if (j < 0) b = (tx > 0) ? __ldcg(ws.btop + (int64_t)(below - 1) * T_TW + T_TW - 1) : -1;
                else if (j >= T_TW) b = (tx + 1 < ntx) ? __ldcg(ws.btop + (int64_t)(below + 1) * T_TW) : -1;
                else b = __ldcg(ws.btop + (int64_t)below * T_TW + j);
                if (b >= 0) gunite(ws.parent, a, b);
            }
        }
    }
    if (tx + 1 < ntx && t < T_TH) {  // right seam
        const int right = tile + 1;
        int a = __ldcg(ws.brig + (int64_t)tile * T_TH + t);
        if (a >= 0) {
            for (int d = -1; d <= 1; d++) {
                int i = t + d;
                if (i < 0 || i >= T_TH) continue;
                int b = __ldcg(ws.blef + (int64_t)right * T_TH + i);
                if (b >= 0) gunite(ws.parent, a, b);
            }
        }
    }
}

// fold every kept node into its root
__global__ void k_ccl_resolve(CclWs ws) {
    const int tile = blockIdx.x;
    const int nc = ws.ncomp[tile];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int node = tile * T_CAP + c;
        if (__ldcg(ws.parent + node) < 0) continue;
        const int r = gfind(ws.parent, node);
        if (r == node) continue;
        ws.parent[node] = r;
        atomicAdd(&ws.area[r], ws.area[node]);
        atomicMin(&ws.first[r], ws.first[node]);
        atomicMax(&ws.peak[r], ws.peak[node]);
        atomicMin(&ws.xmin[r], ws.xmin[node]);
        atomicMax(&ws.xmax[r], ws.xmax[node]);
        atomicMin(&ws.ymin[r], ws.ymin[node]);
        atomicMax(&ws.ymax[r], ws.ymax[node]);
        atomicAdd(&ws.sum[r], ws.sum[node]);
        atomicAdd(&ws.sx[r], ws.sx[node]);
        atomicAdd(&ws.sy[r], ws.sy[node]);
    }
}

__global__ void k_ccl_count(CclWs ws, int64_t W, int min_area) {
    const int tile = blockIdx.x;
    const int nc = ws.ncomp[tile];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int node = tile * T_CAP + c;
        if (ws.parent[node] != node) continue;
        if (ws.area[node] >= min_area) atomicAdd(&ws.rowcnt[ws.first[node] / W], 1);
        else ws.label[node] = 0;
    }
}

constexpr int SCAN_THREADS = 1024;
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_rows(CclWs ws, int64_t H, int32_t* n_src_dev) {
    __shared__ int wsum[SCAN_THREADS / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < H; base += SCAN_THREADS) {
        int64_t i = base + threadIdx.x;
        int v = i < H ? ws.rowcnt[i] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            int s = wsum[lane];
            int si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o) si += t;
            }
            wsum[lane] = si - s;
        }
        __syncthreads();
        int excl = carry + wsum[warp] + inc - v;
        if (i < H) ws.rowbase[i] = excl;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ws.rowbase[H] = carry;
        *n_src_dev = carry;
    }
}

__global__ void k_ccl_place(CclWs ws, int64_t W, int min_area) {
    const int tile = blockIdx.x;
    const int nc = ws.ncomp[tile];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int node = tile * T_CAP + c;
        if (ws.parent[node] != node || ws.area[node] < min_area) continue;
        const unsigned long long f = ws.first[node];
        const int64_t row = (int64_t)(f / (unsigned long long)W);
        const int slot = ws.rowbase[row] + atomicAdd(&ws.rowfill[row], 1);
        ws.slist_first[slot] = f;
        ws.slist_node[slot] = node;
    }
}

__global__ void k_ccl_number(CclWs ws, int64_t W, int min_area, int32_t max_src, ipp_src_stats out) {
    const int tile = blockIdx.x;
    const int nc = ws.ncomp[tile];
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int node = tile * T_CAP + c;
        if (ws.parent[node] != node || ws.area[node] < min_area) continue;
        const unsigned long long f = ws.first[node];
        const int64_t row = (int64_t)(f / (unsigned long long)W);
        const int s0 = ws.rowbase[row], s1 = ws.rowbase[row] + ws.rowcnt[row];
        int rank = 0;
        for (int s = s0; s < s1; s++) rank += ws.slist_first[s] < f;
        const int lab = s0 + rank + 1;
        ws.label[node] = lab;
        if (lab <= max_src) {
            const int k = lab - 1;
            const double sm = ws.sum[node];
            out.area[k] = ws.area[node];
            out.first[k] = (int64_t)f;
            out.xmin[k] = ws.xmin[node];
            out.xmax[k] = ws.xmax[node];
            out.ymin[k] = ws.ymin[node];
            out.ymax[k] = ws.ymax[node];
            out.peak[k] = fkey_inv(ws.peak[node]);
            out.flux[k] = (float)sm;
            out.xbar[k] = (float)(ws.sx[node] / sm);
            out.ybar[k] = (float)(ws.sy[node] / sm);
        }
    }
}

// Second tile pass: rebuild the local components from the bit mask and write
// the final label of every pixel of the tile (0 for background and dropped).
__global__ void __launch_bounds__(T_THREADS, 3) k_tile_final(CclWs ws, int64_t W, int64_t H, int ntx,
                                                           int32_t* labels) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileShared& S = *reinterpret_cast<TileShared*>(smem_raw);
    const int tx = blockIdx.x, ty = blockIdx.y, tile = ty * ntx + tx;
    const int64_t tx0 = (int64_t)tx * T_TW, ty0 = (int64_t)ty * T_TH;
    const int64_t mpitch = (int64_t)ntx * T_WPR;
    if (threadIdx.x < T_WORDS) {
        int r = threadIdx.x / T_WPR, wi = threadIdx.x % T_WPR;
        S.mask[r][wi] = ws.mask[(ty0 + r) * mpitch + (int64_t)tx * T_WPR + wi];
    }
    __syncthreads();
    tile_ccl(S);
    // component id -> final label
    const int nc = S.nc;
    for (int c = threadIdx.x; c < nc; c += T_THREADS) {
        const int node = tile * T_CAP + c;
        const int p = __ldcg(ws.parent + node);
        S.c_area[c] = p < 0 ? 0 : __ldcg(ws.label + p);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t xc = tx0 + lane * 4;
    const bool vec = (W % 4 == 0) && (((uintptr_t)labels & 15) == 0) && (xc + 4 <= W);
    for (int r = warp; r < T_TH; r += T_THREADS / 32) {
        const int64_t y = ty0 + r;
        if (y >= H || xc >= W) continue;
        int out[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            int col = lane * 4 + c;
            out[c] = mbit(S, r, col) ? S.c_area[cid_of(S, S.lab[r * T_TW + col])] : 0;
        }
        if (vec) {
            *reinterpret_cast<int4*>(labels + y * W + xc) = make_int4(out[0], out[1], out[2], out[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; c++)
                if (xc + c < W) labels[y * W + xc + c] = out[c];
        }
    }
}

}  // namespace ipp

// ------------------------------------------------------------------ host side
using namespace ipp;

struct CclLayout {
    int ntx, nty;
    int64_t ntiles, nodes;
    size_t off[24];
    size_t total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static CclLayout ccl_layout(int64_t W, int64_t H) {
    CclLayout L;
    L.ntx = (int)cdiv(W, T_TW);
    L.nty = (int)cdiv(H, T_TH);
    L.ntiles = (int64_t)L.ntx * L.nty;
    L.nodes = L.ntiles * T_CAP;
    size_t sizes[] = {
        (size_t)(L.nty * T_TH) * (size_t)(L.ntx * T_WPR) * 4,  // mask
        (size_t)L.ntiles * 4,                                  // ncomp
        (size_t)L.nodes * 4, (size_t)L.nodes * 4,              // parent, area
        (size_t)L.nodes * 8, (size_t)L.nodes * 4,              // first, peak
        (size_t)L.nodes * 4, (size_t)L.nodes * 4, (size_t)L.nodes * 4, (size_t)L.nodes * 4,  // bbox
        (size_t)L.nodes * 8, (size_t)L.nodes * 8, (size_t)L.nodes * 8,  // sum sx sy
        (size_t)L.nodes * 4,                                   // label
        (size_t)L.ntiles * T_TW * 4, (size_t)L.ntiles * T_TW * 4,  // btop bbot
        (size_t)L.ntiles * T_TH * 4, (size_t)L.ntiles * T_TH * 4,  // blef brig
        (size_t)H * 4, (size_t)H * 4, (size_t)(H + 1) * 4,     // rowcnt rowfill rowbase
        (size_t)L.nodes * 8, (size_t)L.nodes * 4,              // slist
    };
    size_t o = 0;
    for (int k = 0; k < 23; k++) { L.off[k] = o; o += align256(sizes[k]); }
    L.total = o;
    return L;
}

static CclWs ccl_ws(const CclLayout& L, void* ws) {
    unsigned char* b = (unsigned char*)ws;
    CclWs w;
    w.mask = (uint32_t*)(b + L.off[0]);
    w.ncomp = (int32_t*)(b + L.off[1]);
    w.parent = (int32_t*)(b + L.off[2]);
    w.area = (int32_t*)(b + L.off[3]);
    w.first = (unsigned long long*)(b + L.off[4]);
    w.peak = (uint32_t*)(b + L.off[5]);
    w.xmin = (int32_t*)(b + L.off[6]);
    w.xmax = (int32_t*)(b + L.off[7]);
    w.ymin = (int32_t*)(b + L.off[8]);
    w.ymax = (int32_t*)(b + L.off[9]);
    w.sum = (double*)(b + L.off[10]);
    w.sx = (double*)(b + L.off[11]);
    w.sy = (double*)(b + L.off[12]);
    w.label = (int32_t*)(b + L.off[13]);
    w.btop = (int32_t*)(b + L.off[14]);
    w.bbot = (int32_t*)(b + L.off[15]);
    w.blef = (int32_t*)(b + L.off[16]);
    w.brig = (int32_t*)(b + L.off[17]);
    w.rowcnt = (int32_t*)(b + L.off[18]);
    w.rowfill = (int32_t*)(b + L.off[19]);
    w.rowbase = (int32_t*)(b + L.off[20]);
    w.slist_first = (unsigned long long*)(b + L.off[21]);
    w.slist_node = (int32_t*)(b + L.off[22]);
    return w;
}

size_t ipp_ccl_workspace_size(int64_t W, int64_t H) { return ccl_layout(W, H).total; }


int ipp_launch_detect(const DetectArgs& A, cudaStream_t s) {
    CclLayout L = ccl_layout(A.W, A.H);
    if (L.nodes >= (int64_t)INT32_MAX) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "frame too large for 32-bit node ids");
    CclWs w = ccl_ws(L, A.ws);
    TileJob J;
    J.mode = A.mode; J.W = A.W; J.H = A.H; J.ntx = L.ntx; J.nty = L.nty;
    J.img = A.img; J.dtype = A.dtype; J.pitch = A.pitch;
    J.bias_map = A.bias_map; J.bias = A.bias; J.inv_flat = A.inv_flat;
    J.mesh_bkg = A.mesh_bkg; J.sub = A.sub; J.sub_pitch = A.sub_pitch;
    J.mesh_rms = A.mesh_rms; J.nx = A.nx; J.ny = A.ny; J.mesh_w = A.mesh_w; J.mesh_h = A.mesh_h;
    J.k = A.k; J.thresh_abs = A.thresh_abs; J.min_area = A.min_area; J.mask_in = A.mask_in;
    J.ws = w;
    const size_t sm = sizeof(TileShared);
    cudaFuncSetAttribute(k_tile_label, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_tile_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 tg(L.ntx, L.nty);
    k_tile_label<<<tg, T_THREADS, sm, s>>>(J);
    if (int e = ipp_check_launch("k_tile_label")) return e;
    k_ccl_union<<<tg, 128, 0, s>>>(w, L.ntx, L.nty);
    if (int e = ipp_check_launch("k_ccl_union")) return e;
    const unsigned nt = (unsigned)L.ntiles;
    k_ccl_resolve<<<nt, 128, 0, s>>>(w);
    if (int e = ipp_check_launch("k_ccl_resolve")) return e;
    k_ccl_count<<<nt, 128, 0, s>>>(w, A.W, A.min_area);
    if (int e = ipp_check_launch("k_ccl_count")) return e;
    k_scan_rows<<<1, SCAN_THREADS, 0, s>>>(w, A.H, A.n_src_dev);
    if (int e = ipp_check_launch("k_scan_rows")) return e;
    k_ccl_place<<<nt, 128, 0, s>>>(w, A.W, A.min_area);
    if (int e = ipp_check_launch("k_ccl_place")) return e;
    k_ccl_number<<<nt, 128, 0, s>>>(w, A.W, A.min_area, A.max_src, A.stats);
    if (int e = ipp_check_launch("k_ccl_number")) return e;
    k_tile_final<<<tg, T_THREADS, sm, s>>>(w, A.W, A.H, L.ntx, A.labels);
    return ipp_check_launch("k_tile_final");
}
