// subtract.cu -- the convolution and difference of HOTPANTS-style image
// subtraction (Sec. 2.2.4, Eqs. 8-10): with fitted coefficients c_{n,s} and
// background d_b, the kernel of each (2 hw + 1)^2 output tile is
// K(u, v) = sum_n a_n(tile centre) K_n(u, v), a_n = sum_s c_{n,s} P_s (Eq. 8),
// K_n = exp(-(u^2 + v^2) / (2 sig^2)) u^i v^j (Eq. 9), and the difference is
// D = I + B - R (x) K (the residual of Eq. 10), NaN where the kernel's support
// leaves the frame.
//
// One block per output tile, as in the paper's stamp-per-block convolution:
// the tile's kernel and the template window (tile + 2 hw border) are staged in
// shared memory; each thread computes a strip of 7 output pixels of one row,
// holding the strip's window row in registers for each kernel row, so that a
// kernel tap costs one shared load (broadcast) per 7 FMAs.
#include <math.h>

#include <algorithm>

#include "jobs.cuh"

namespace ipp {

constexpr int SB_STRIP = 7;
constexpr int SB_MAXB = 64;    // basis functions
constexpr int SB_MAXT = 16;    // spatial terms (order <= 4)

struct SubBasisDesc {
    int nk;
    float sig[8];
    int deg[8];
};

// basis function n on the (2 hw + 1)^2 grid: one block per function
__global__ void k_sub_basis(SubBasisDesc d, int hw, float* __restrict__ basis) {
    int n = blockIdx.x, k = 0, i = 0, j = 0, acc = 0;
    for (int kk = 0; kk < d.nk; kk++) {
        const int cnt = (d.deg[kk] + 1) * (d.deg[kk] + 2) / 2;
        if (n < acc + cnt) {
            k = kk;
            int r = n - acc;
            for (i = 0; i <= d.deg[kk]; i++) {
                const int row = d.deg[kk] - i + 1;
                if (r < row) {
                    j = r;
                    break;
                }
                r -= row;
            }
            break;
        }
        acc += cnt;
    }
    const int S = 2 * hw + 1;
    const double s2 = 2.0 * (double)d.sig[k] * (double)d.sig[k];
    for (int t = threadIdx.x; t < S * S; t += blockDim.x) {
        const int u = t % S - hw, v = t / S - hw;
        double p = exp(-(double)(u * u + v * v) / s2);
        for (int q = 0; q < i; q++) p *= (double)u;
        for (int q = 0; q < j; q++) p *= (double)v;
        basis[(size_t)n * S * S + t] = (float)p;
    }
}

__device__ __forceinline__ void sub_terms(float xs, float ys, int order, float* t) {
    int n = 0;
    float xp = 1.f;
    for (int p = 0; p <= order; p++) {
        float yq = 1.f;
        for (int q = 0; q <= order - p; q++) {
            t[n++] = xp * yq;
            yq *= ys;
        }
        xp *= xs;
    }
}

template <int HW>
__global__ void __launch_bounds__(((2 * HW + 1) / SB_STRIP + ((2 * HW + 1) % SB_STRIP != 0)) * (2 * HW + 1))
    k_sub_apply(const float* __restrict__ I, const float* __restrict__ R, int64_t W, int64_t H, int64_t pitch,
                const float* __restrict__ basis, int nb, const float* __restrict__ cs, int sord,
                const float* __restrict__ cb, int bord, float* __restrict__ D, int64_t opitch) {
    constexpr int S = 2 * HW + 1, WIN = S + 2 * HW, SPR = (S + SB_STRIP - 1) / SB_STRIP;
    __shared__ float Ks[S * S];
    __shared__ float Rw[WIN][WIN + 1];
    __shared__ float an[SB_MAXB];
    const int ntx = (int)((W + S - 1) / S);
    const int64_t tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int64_t x0 = tx * S, y0 = ty * S;
    const float sx = W > 1 ? 2.f / (float)(W - 1) : 0.f, sy = H > 1 ? 2.f / (float)(H - 1) : 0.f;
    // Eq. 8 at the tile centre
    {
        float P[SB_MAXT];
        const float xs = W > 1 ? (float)((double)x0 + 0.5 * (S - 1)) * sx - 1.f : 0.f;
        const float ys = H > 1 ? (float)((double)y0 + 0.5 * (S - 1)) * sy - 1.f : 0.f;
        sub_terms(xs, ys, sord, P);
        const int ns = (sord + 1) * (sord + 2) / 2;
        for (int n = threadIdx.x; n < nb; n += blockDim.x) {
            float a = 0.f;
            for (int t = 0; t < ns; t++) a = fmaf(__ldg(cs + n * ns + t), P[t], a);
            an[n] = a;
        }
    }
    // template window: rows y0 - HW .. y0 + S - 1 + HW (0 outside the frame)
    for (int t = threadIdx.x; t < WIN * WIN; t += blockDim.x) {
        const int a = t / WIN, b = t % WIN;
        const int64_t yy = y0 - HW + a, xx = x0 - HW + b;
        Rw[a][b] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? __ldg(R + yy * pitch + xx) : 0.f;
    }
    __syncthreads();
    // Eq. 9 summed with the tile's amplitudes
    for (int t = threadIdx.x; t < S * S; t += blockDim.x) {
        float k = 0.f;
        for (int n = 0; n < nb; n++) k = fmaf(an[n], __ldg(basis + (size_t)n * S * S + t), k);
        Ks[t] = k;
    }
    __syncthreads();
    const int oy = threadIdx.x / SPR, ox0 = (threadIdx.x % SPR) * SB_STRIP;
    if (oy >= S) return;
    float acc[SB_STRIP];
#pragma unroll
    for (int q = 0; q < SB_STRIP; q++) acc[q] = 0.f;
    // out(oy, ox) = sum_{v', u'} K[v'][u'] Rw[oy + 2HW - v'][ox + 2HW - u']
    for (int vp = 0; vp < S; vp++) {
        const int a = oy + 2 * HW - vp;
        float rr[SB_STRIP + 2 * HW];
#pragma unroll
        for (int q = 0; q < SB_STRIP + 2 * HW; q++) rr[q] = (ox0 + q < WIN) ? Rw[a][ox0 + q] : 0.f;
#pragma unroll
        for (int up = 0; up < S; up++) {
            const float k = Ks[vp * S + up];
#pragma unroll
            for (int q = 0; q < SB_STRIP; q++) acc[q] = fmaf(k, rr[q + 2 * HW - up], acc[q]);
        }
    }
    const int64_t y = y0 + oy;
    if (y >= H) return;
    const float ys = H > 1 ? (float)y * sy - 1.f : 0.f;
    const int ng = bord >= 0 ? (bord + 1) * (bord + 2) / 2 : 0;
#pragma unroll
    for (int q = 0; q < SB_STRIP; q++) {
        const int ox = ox0 + q;
        const int64_t x = x0 + ox;
        if (ox >= S || x >= W) continue;
        float r = NAN;
        if (x >= HW && y >= HW && x <= W - 1 - HW && y <= H - 1 - HW) {
            float b = 0.f;
            if (ng) {
                float P[SB_MAXT];
                const float xs = W > 1 ? (float)x * sx - 1.f : 0.f;
                sub_terms(xs, ys, bord, P);
                for (int t = 0; t < ng; t++) b = fmaf(cb[t], P[t], b);
            }
            r = __ldg(I + y * pitch + x) + b - acc[q];
        }
        D[y * opitch + x] = r;
    }
}

}  // namespace ipp

using namespace ipp;

size_t ipp_sub_ws_bytes(int nb, int hw) {
    return (size_t)nb * (2 * hw + 1) * (2 * hw + 1) * sizeof(float);
}

int ipp_launch_sub_apply(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int hw, int nk,
                         const float* sig, const int* deg, int nb, const float* cs, int sord, const float* cb,
                         int bord, float* D, int64_t opitch, void* ws, cudaStream_t s) {
    SubBasisDesc d;
    d.nk = nk;
    for (int k = 0; k < nk; k++) {
        d.sig[k] = sig[k];
        d.deg[k] = deg[k];
    }
    float* basis = (float*)ws;
    k_sub_basis<<<nb, 128, 0, s>>>(d, hw, basis);
    if (int e = ipp_check_launch("k_sub_basis")) return e;
    const int S = 2 * hw + 1;
    const int64_t ntiles = ((W + S - 1) / S) * ((H + S - 1) / S);
    const int threads = ((S + SB_STRIP - 1) / SB_STRIP) * S;
    switch (hw) {
#define SB_CASE(HWV)                                                                                       \
    case HWV:                                                                                              \
        k_sub_apply<HWV><<<(unsigned)ntiles, threads, 0, s>>>(I, R, W, H, pitch, basis, nb, cs, sord, cb, \
                                                              bord, D, opitch);                            \
        break;
        SB_CASE(4)
        SB_CASE(6)
        SB_CASE(8)
        SB_CASE(10)
        SB_CASE(12)
#undef SB_CASE
        default: return IPP_ERR_NOT_SUPPORTED;
    }
    return ipp_check_launch("k_sub_apply");
}
