// phot.cu -- per-source measurements of Sec. 2.2.5: windowed centroid and
// circular-aperture photometry with a local sky annulus.  One warp per source,
// persistent grid-stride over the device-resident source count (the count never
// leaves the GPU).  Positions are carried as an integer anchor plus a small
// offset so that pixel offsets keep full FP32 precision anywhere in the frame.
#include <math.h>

#include "jobs.cuh"

namespace ipp {

constexpr int P_THREADS = 256;
constexpr int P_WARPS = P_THREADS / 32;
constexpr int ANN_MAXR = 16;                               // r_out limit
constexpr int ANN_BOX = 2 * (ANN_MAXR + 1) + 1;            // 35
constexpr int ANN_CAP = ANN_BOX * ANN_BOX;                 // 1225


__global__ void __launch_bounds__(P_THREADS) k_centroid(CenJob J) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * P_THREADS + threadIdx.x) >> 5;
    const int nw = (gridDim.x * P_THREADS) >> 5;
    const int n = min(*J.n_src_dev, J.max_src);
    const float rad2 = J.rad * J.rad;
    const float inv2s2 = 1.0f / (2.0f * J.sw * J.sw);
    const int R = (int)ceilf(J.rad) + 1;
    const int box = 2 * R + 1;
    for (int s = gw; s < n; s += nw) {
        const float sx0 = J.x0[s], sy0 = J.y0[s];
        float ax = rintf(sx0), ay = rintf(sy0);
        float ox = sx0 - ax, oy = sy0 - ay;
        int fl = IPP_FLAG_WIN_NOT_CONVERGED, it;
        for (it = 0; it < J.max_iter; it++) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            const int64_t ia = (int64_t)ay, ja = (int64_t)ax;
            for (int idx = lane; idx < box * box; idx += 32) {
                int di = idx / box - R, dj = idx % box - R;
                float dx = (float)dj - ox, dy = (float)di - oy;
                float d2 = fmaf(dx, dx, dy * dy);
                int64_t i = ia + di, j = ja + dj;
                if (d2 < rad2 && i >= 0 && i < J.H && j >= 0 && j < J.W) {
                    float w = expf(-d2 * inv2s2) * __ldg(J.sub + i * J.pitch + j);
                    s0 += w;
                    s1 = fmaf(w, dx, s1);
                    s2 = fmaf(w, dy, s2);
                }
            }
            s0 = warp_sum(s0);
            s1 = warp_sum(s1);
            s2 = warp_sum(s2);
            if (!(s0 > 0.f)) {  // keep the seed
                ax = rintf(sx0); ay = rintf(sy0); ox = sx0 - ax; oy = sy0 - ay;
                it++;
                break;
            }
            float ddx = 2.0f * s1 / s0, ddy = 2.0f * s2 / s0;
            ox += ddx;
            oy += ddy;
            float rx = rintf(ox), ry = rintf(oy);  // re-anchor: |offset| <= 1/2
            ax += rx; ox -= rx;
            ay += ry; oy -= ry;
            if (ddx * ddx + ddy * ddy < J.tol2) { fl = 0; it++; break; }
        }
        const float xf = ax + ox, yf = ay + oy;
        if (xf - J.rad < -0.5f || xf + J.rad > (float)J.W - 0.5f || yf - J.rad < -0.5f ||
            yf + J.rad > (float)J.H - 0.5f)
            fl |= IPP_FLAG_EDGE;
        if (lane == 0) {
            J.x[s] = xf;
            J.y[s] = yf;
            if (J.niter) J.niter[s] = it;
            J.flags[s] = fl;
        }
    }
}

// ---------------------------------------------------------------- aperture
// Area of the disk of radius r centred at (cx, cy) -- coordinates relative to
// the pixel centre -- intersected with the pixel [-1/2, 1/2]^2.  In disk-centred
// coordinates the pixel is [X0, X1] x [Y0, Y1]; the area is the integral over x
// of the chord clipped to [Y0, Y1], split where the circle meets y = Y0, Y1.
// On a piece [p, q] a limit is either the box edge or the circle, whose integral
// is G(q) - G(p), G(t) = (t s(t) + r^2 atan2(t, s(t))) / 2, s(t) = sqrt(r^2 - t^2);
// the angle difference is taken as one atan2 of the cross/dot products, which
// keeps it accurate for the narrow pieces of edge pixels.
__device__ float circle_pixel_area(float cx, float cy, float r) {
    const float ax = fabsf(cx), ay = fabsf(cy);
    const float nx = fmaxf(ax - 0.5f, 0.f), ny = fmaxf(ay - 0.5f, 0.f);
    const float r2 = r * r;
    if (nx * nx + ny * ny >= r2) return 0.f;
    const float fx = ax + 0.5f, fy = ay + 0.5f;
    if (fx * fx + fy * fy <= r2) return 1.f;
    // disk-centred box (by symmetry use |cx|, |cy|: the box is then at -a-1/2..-a+1/2)
    const float X0 = -ax - 0.5f, X1 = -ax + 0.5f, Y0 = -ay - 0.5f, Y1 = -ay + 0.5f;
    float a = fmaxf(X0, -r), b = fminf(X1, r);
    if (!(a < b)) return 0.f;
    float pts[6];
    int np = 0;
    pts[np++] = a;
    const float ys[2] = {Y0, Y1};
#pragma unroll
    for (int k = 0; k < 2; k++) {
        float yy = fabsf(ys[k]);
        if (yy < r) {
            float h = sqrtf((r - yy) * (r + yy));
            if (-h > a && -h < b) pts[np++] = -h;
            if (h > a && h < b) pts[np++] = h;
        }
    }
    pts[np++] = b;
    // sort (at most 6 values)
    for (int i = 1; i < np; i++) {
        float v = pts[i];
        int j = i - 1;
        while (j >= 0 && pts[j] > v) { pts[j + 1] = pts[j]; j--; }
        pts[j + 1] = v;
    }
    float area = 0.f;
    for (int k = 0; k + 1 < np; k++) {
        float p = pts[k], q = pts[k + 1];
        if (!(q > p)) continue;
        float m = 0.5f * (p + q);
        float am = fabsf(m);
        float hm = am < r ? sqrtf((r - am) * (r + am)) : 0.f;
        bool up_circ = hm < Y1, lo_circ = -hm > Y0;
        float upv = up_circ ? hm : Y1, lov = lo_circ ? -hm : Y0;
        if (!(upv > lov)) continue;
        float dG = 0.f;
        if (up_circ || lo_circ) {
            float ap = fabsf(p), aq = fabsf(q);
            float sp = ap < r ? sqrtf((r - ap) * (r + ap)) : 0.f;
            float sq = aq < r ? sqrtf((r - aq) * (r + aq)) : 0.f;
            float dth = atan2f(sp * q - p * sq, sp * sq + p * q);
            dG = 0.5f * ((q * sq - p * sp) + r2 * dth);
        }
        float w = q - p;
        float iu = up_circ ? dG : Y1 * w;
        float il = lo_circ ? -dG : Y0 * w;
        area += iu - il;
    }
    return fminf(fmaxf(area, 0.f), 1.f);
}


// Annulus membership r_in^2 <= d^2 < r_out^2 decided exactly as an FP64
// evaluation ((j - x)^2 + (i - y)^2 with no fused operations): FP32 first, and the
// FP64 expression only when the FP32 value is within 1e-5 relative of a bound.
__device__ __forceinline__ bool in_annulus(float dx, float dy, int64_t i, int64_t j, float x, float y,
                                           float rin2, float rout2, double rin2d, double rout2d) {
    float d2 = fmaf(dx, dx, dy * dy);
    const float m_in = 1e-5f * rin2, m_out = 1e-5f * rout2;
    bool near = fabsf(d2 - rin2) <= m_in || fabsf(d2 - rout2) <= m_out;
    if (!near) return d2 >= rin2 && d2 < rout2;
    double ddx = __dsub_rn((double)j, (double)x), ddy = __dsub_rn((double)i, (double)y);
    double e2 = __dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy));
    return e2 >= rin2d && e2 < rout2d;
}

__global__ void __launch_bounds__(P_THREADS) k_aperture(PhotJob J) {
    __shared__ float ann[P_WARPS][ANN_CAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = (blockIdx.x * P_THREADS + threadIdx.x) >> 5;
    const int nw = (gridDim.x * P_THREADS) >> 5;
    const int n = min(*J.n_src_dev, J.max_src);
    float* buf = ann[wib];
    const int R1 = (int)ceilf(J.r_ap + 0.5f), box1 = 2 * R1 + 1;
    const int R2 = (int)ceilf(J.r_out) + 1, box2 = 2 * R2 + 1;
    const double rin2d = __dmul_rn((double)J.r_in, (double)J.r_in);
    const double rout2d = __dmul_rn((double)J.r_out, (double)J.r_out);
    const float rin2 = (float)rin2d, rout2 = (float)rout2d;
    for (int s = gw; s < n; s += nw) {
        const float x = J.x[s], y = J.y[s];
        const float ax = rintf(x), ay = rintf(y);
        const float ox = x - ax, oy = y - ay;
        const int64_t ia = (int64_t)ay, ja = (int64_t)ax;
        // aperture sum with exact overlap weights
        float sw = 0.f, swf = 0.f;
        for (int idx = lane; idx < box1 * box1; idx += 32) {
            int di = idx / box1 - R1, dj = idx % box1 - R1;
            int64_t i = ia + di, j = ja + dj;
            if (i < 0 || i >= J.H || j < 0 || j >= J.W) continue;
            float w = circle_pixel_area(ox - (float)dj, oy - (float)di, J.r_ap);
            if (w > 0.f) {
                sw += w;
                swf = fmaf(w, __ldg(J.sub + i * J.pitch + j), swf);
            }
        }
        sw = warp_sum(sw);
        swf = warp_sum(swf);
        // annulus values into the warp's buffer
        int na = 0;
        for (int base = 0; base < box2 * box2; base += 32) {
            int idx = base + lane;
            bool take = false;
            float v = 0.f;
            if (idx < box2 * box2) {
                int di = idx / box2 - R2, dj = idx % box2 - R2;
                int64_t i = ia + di, j = ja + dj;
                if (i >= 0 && i < J.H && j >= 0 && j < J.W &&
                    in_annulus((float)dj - ox, (float)di - oy, i, j, x, y, rin2, rout2, rin2d, rout2d)) {
                    take = true;
                    v = __ldg(J.sub + i * J.pitch + j);
                }
            }
            unsigned bal = __ballot_sync(0xffffffffu, take);
            if (take) buf[na + __popc(bal & ((1u << lane) - 1u))] = v;
            na += __popc(bal);
        }
        __syncwarp();
        float skyv = 0.f;
        int fl = 0;
        if (na < J.min_ann) {
            fl |= IPP_FLAG_ANN_FEW;
        } else {
            // median (Eq. 1) by bisection over order-preserving keys
            const int k0 = (na - 1) / 2, k1 = na / 2;
            uint32_t lo = 0u, hi = 0xffffffffu;
            while (lo < hi) {
                uint32_t mid = lo + ((hi - lo) >> 1);
                int c = 0;
                for (int t = lane; t < na; t += 32) c += fkey(buf[t]) <= mid;
                c = __reduce_add_sync(0xffffffffu, c);
                if (c > k0) hi = mid; else lo = mid + 1;
            }
            const uint32_t ka = lo;
            int cle = 0;
            uint32_t nxt = 0xffffffffu;
            for (int t = lane; t < na; t += 32) {
                uint32_t kk = fkey(buf[t]);
                cle += kk <= ka;
                if (kk > ka && kk < nxt) nxt = kk;
            }
            cle = __reduce_add_sync(0xffffffffu, cle);
            nxt = __reduce_min_sync(0xffffffffu, nxt);
            const uint32_t kb = (cle > k1) ? ka : nxt;
            skyv = (float)(0.5 * ((double)fkey_inv(ka) + (double)fkey_inv(kb)));
        }
        __syncwarp();
        const float Rm = fmaxf(J.r_ap, J.r_out);
        if (x - Rm < -0.5f || x + Rm > (float)J.W - 0.5f || y - Rm < -0.5f || y + Rm > (float)J.H - 0.5f)
            fl |= IPP_FLAG_EDGE;
        if (lane == 0) {
            J.flux[s] = swf - skyv * sw;
            if (J.sky) J.sky[s] = skyv;
            if (J.area) J.area[s] = sw;
            if (J.n_ann) J.n_ann[s] = na;
            if (J.flags) J.flags[s] = fl;
        }
    }
}

}  // namespace ipp

using namespace ipp;

static int persistent_blocks(cudaStream_t) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms * 4 : 512;
}

int ipp_launch_centroid(const CenJob& J, cudaStream_t s) {
    k_centroid<<<persistent_blocks(s), P_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_centroid");
}

int ipp_launch_aperture(const PhotJob& J, cudaStream_t s) {
    if (J.r_out > (float)ANN_MAXR) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "r_out above %d px", ANN_MAXR);
    k_aperture<<<persistent_blocks(s), P_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_aperture");
}
