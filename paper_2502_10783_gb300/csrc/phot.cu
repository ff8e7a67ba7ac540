// phot.cu -- per-source measurements of Sec. 2.2.5: windowed centroid and
// circular-aperture photometry with a local sky annulus.  One warp per source,
// persistent grid-stride over the device-resident source count (the count never
// leaves the GPU).  Positions are carried as an integer anchor plus a small
// offset so that pixel offsets keep full FP32 precision anywhere in the frame.
#include <math.h>

#include <algorithm>
#include <vector>

#include "jobs.cuh"

namespace ipp {

constexpr int P_THREADS = 256;
constexpr int P_WARPS = P_THREADS / 32;
constexpr int ANN_MAXR = 16;                               // r_out limit
constexpr int ANN_BOX = 2 * (ANN_MAXR + 1) + 1;            // 35
constexpr int ANN_CAP = ANN_BOX * ANN_BOX;                 // 1225


// Window pixels of one source: the box of half-width R = floor(rad + 1/2)
// around the integer anchor covers every pixel within rad of a position whose
// offset from the anchor is at most 1/2.  With NPL > 0 each lane caches its
// NPL box pixels in registers and reloads them only when the anchor moves.
template <int NPL>
__global__ void __launch_bounds__(P_THREADS) k_centroid(CenJob J) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * P_THREADS + threadIdx.x) >> 5;
    const int nw = (gridDim.x * P_THREADS) >> 5;
    const int n = min(*J.n_src_dev, J.max_src);
    const float rad2 = J.rad * J.rad;
    const float inv2s2 = 1.0f / (2.0f * J.sw * J.sw);
    const float Wf = (float)(int)J.W, Hf = (float)(int)J.H;
    const int R = (int)floorf(J.rad + 0.5f);
    const int box = 2 * R + 1, nbox = box * box;
    // this lane's box offsets, fixed for the whole kernel
    constexpr int NC = NPL > 0 ? NPL : 1;
    float dif[NC], djf[NC];
    int dii[NC], dji[NC];
#pragma unroll
    for (int m = 0; m < NC; m++) {
        const int idx = lane + 32 * m;
        dii[m] = idx / box - R;
        dji[m] = idx % box - R;
        dif[m] = (float)dii[m];
        djf[m] = (float)dji[m];
    }
    for (int s = gw; s < n; s += nw) {
        const float sx0 = J.x0[s], sy0 = J.y0[s];
        float ax = rintf(sx0), ay = rintf(sy0);
        float ox = sx0 - ax, oy = sy0 - ay;
        int fl = IPP_FLAG_WIN_NOT_CONVERGED, it;
        float cache[NC];
        uint32_t valid = 0;
        float cax = NAN, cay = NAN;  // anchor of the cached pixels
        for (it = 0; it < J.max_iter; it++) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            if (NPL > 0) {
                if (ax != cax || ay != cay) {  // (re)load the box around the anchor
                    const int64_t ia = (int)ay, ja = (int)ax;
                    valid = 0;
#pragma unroll
                    for (int m = 0; m < NC; m++) {
                        const int64_t i = ia + dii[m], j = ja + dji[m];
                        const bool ok = (lane + 32 * m < nbox) && i >= 0 && i < J.H && j >= 0 && j < J.W;
                        cache[m] = ok ? __ldg(J.sub + i * J.pitch + j) : 0.f;
                        valid |= (uint32_t)ok << m;
                    }
                    cax = ax;
                    cay = ay;
                }
#pragma unroll
                for (int m = 0; m < NC; m++) {
                    const float dx = djf[m] - ox, dy = dif[m] - oy;
                    const float d2 = fmaf(dx, dx, dy * dy);
                    if (((valid >> m) & 1u) && d2 < rad2) {
                        const float w = __expf(-d2 * inv2s2) * cache[m];
                        s0 += w;
                        s1 = fmaf(w, dx, s1);
                        s2 = fmaf(w, dy, s2);
                    }
                }
            } else {
                const int64_t ia = (int)ay, ja = (int)ax;
                for (int idx = lane; idx < nbox; idx += 32) {
                    const int di = idx / box - R, dj = idx % box - R;
                    const float dx = (float)dj - ox, dy = (float)di - oy;
                    const float d2 = fmaf(dx, dx, dy * dy);
                    const int64_t i = ia + di, j = ja + dj;
                    if (d2 < rad2 && i >= 0 && i < J.H && j >= 0 && j < J.W) {
                        const float w = __expf(-d2 * inv2s2) * __ldg(J.sub + i * J.pitch + j);
                        s0 += w;
                        s1 = fmaf(w, dx, s1);
                        s2 = fmaf(w, dy, s2);
                    }
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
            const float ddx = 2.0f * s1 / s0, ddy = 2.0f * s2 / s0;
            ox += ddx;
            oy += ddy;
            const float rx = rintf(ox), ry = rintf(oy);  // re-anchor: |offset| <= 1/2
            ax += rx; ox -= rx;
            ay += ry; oy -= ry;
            if (ddx * ddx + ddy * ddy < J.tol2) { fl = 0; it++; break; }
        }
        const float xf = ax + ox, yf = ay + oy;
        if (xf - J.rad < -0.5f || xf + J.rad > Wf - 0.5f || yf - J.rad < -0.5f || yf + J.rad > Hf - 0.5f)
            fl |= IPP_FLAG_EDGE;
        if (lane == 0) {
            J.x[s] = xf;
            J.y[s] = yf;
            if (J.niter) J.niter[s] = it;
            J.flags[s] = fl;
        }
    }
}

// Separable form, half a warp per source: the window weight is
// g(dx) g(dy) with g(t) = exp(-t^2 / (2 sw^2)), and the disk |d| < rad keeps in
// row i the columns with dx_j^2 < rad^2 - dy_i^2.  Lane r of the half holds box
// row r in registers; lane j computes column j's (g, dx, dx^2), shared through
// shared memory; each row sums g(dx) f and g(dx) dx f, and the rows' sums are
// weighted by g(dy) and reduced over the half.  Same iteration and stopping
// rule as k_centroid; about a third of its instructions per pass.
constexpr int CR_BOX = 15;  // box of 2R + 1 <= 15 pixels (rad < 7.5)

__device__ __forceinline__ void centroid_rows_body(const CenJob& J, int vb, int nvb) {
    __shared__ float4 colv[P_THREADS / 16][CR_BOX];
    const int lane = threadIdx.x & 31, sub = lane & 15, half = threadIdx.x >> 4;
    const unsigned hmask = 0xffffu << (lane & 16);
    const int gid = (vb * P_THREADS + threadIdx.x) >> 4;
    const int ng = (nvb * P_THREADS) >> 4;
    const int n = min(*J.n_src_dev, J.max_src);
    const float rad2 = J.rad * J.rad;
    const float inv2s2 = 1.0f / (2.0f * J.sw * J.sw);
    const float Wf = (float)(int)J.W, Hf = (float)(int)J.H;
    const int R = (int)floorf(J.rad + 0.5f);
    const int box = 2 * R + 1;
    const bool rowlane = sub < box;
    const float dyr = (float)(sub - R);
    for (int s = gid; s < n; s += ng) {
        const float sx0 = J.x0[s], sy0 = J.y0[s];
        float ax = rintf(sx0), ay = rintf(sy0);
        float ox = sx0 - ax, oy = sy0 - ay;
        int fl = IPP_FLAG_WIN_NOT_CONVERGED, it;
        float row[CR_BOX];
        uint32_t valid = 0;
        float cax = NAN, cay = NAN;  // anchor of the cached row
        for (it = 0; it < J.max_iter; it++) {
            if (ax != cax || ay != cay) {  // (re)load this lane's box row around the anchor
                const int64_t i = (int64_t)(int)ay + (sub - R), ja = (int)ax;
                valid = 0;
#pragma unroll
                for (int c = 0; c < CR_BOX; c++) {
                    const int64_t j = ja + (c - R);
                    const bool ok = rowlane && c < box && i >= 0 && i < J.H && j >= 0 && j < J.W;
                    row[c] = ok ? __ldg(J.sub + i * J.pitch + j) : 0.f;
                    valid |= (uint32_t)ok << c;
                }
                cax = ax;
                cay = ay;
            }
            if (rowlane) {
                const float dx = dyr - ox;  // column sub's offset (dyr = sub - R)
                colv[half][sub] = make_float4(__expf(-dx * dx * inv2s2), dx, dx * dx, 0.f);
            }
            __syncwarp(hmask);
            float r0 = 0.f, r1 = 0.f;
            const float dy = dyr - oy;
            const float lim = rad2 - dy * dy;
#pragma unroll
            for (int c = 0; c < CR_BOX; c++) {
                const float4 cv = colv[half][c < box ? c : 0];
                if (((valid >> c) & 1u) && cv.z < lim) {
                    const float gf = cv.x * row[c];
                    r0 += gf;
                    r1 = fmaf(gf, cv.y, r1);
                }
            }
            const float gy = rowlane ? __expf(-dy * dy * inv2s2) : 0.f;
            float s0 = gy * r0, s1 = gy * r1, s2 = gy * dy * r0;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(hmask, s0, o);
                s1 += __shfl_xor_sync(hmask, s1, o);
                s2 += __shfl_xor_sync(hmask, s2, o);
            }
            __syncwarp(hmask);  // colv is rewritten by the next pass
            if (!(s0 > 0.f)) {  // keep the seed
                ax = rintf(sx0); ay = rintf(sy0); ox = sx0 - ax; oy = sy0 - ay;
                it++;
                break;
            }
            const float ddx = 2.0f * s1 / s0, ddy = 2.0f * s2 / s0;
            ox += ddx;
            oy += ddy;
            const float rx = rintf(ox), ry = rintf(oy);  // re-anchor: |offset| <= 1/2
            ax += rx; ox -= rx;
            ay += ry; oy -= ry;
            if (ddx * ddx + ddy * ddy < J.tol2) { fl = 0; it++; break; }
        }
        const float xf = ax + ox, yf = ay + oy;
        if (xf - J.rad < -0.5f || xf + J.rad > Wf - 0.5f || yf - J.rad < -0.5f || yf + J.rad > Hf - 0.5f)
            fl |= IPP_FLAG_EDGE;
        if (sub == 0) {
            J.x[s] = xf;
            J.y[s] = yf;
            if (J.niter) J.niter[s] = it;
            J.flags[s] = fl;
        }
    }
}

__global__ void __launch_bounds__(P_THREADS) k_centroid_rows(CenJob J) { centroid_rows_body(J, blockIdx.x, gridDim.x); }

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
        if (yy <= r) {  // |y| = r: the circle touches the edge line at x = 0
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

// Median (Eq. 1) of buf[0..na) by one histogram pass: 30 equal bins over
// [mean - 2 sd, mean + 2 sd) plus one bin below and one above; the bin index
// is monotone in the value, so the bins holding the middle order statistics
// x_k0, x_k1 (k0 = (na-1)/2, k1 = na/2) hold a contiguous range of the sorted
// values.  When at most 32 values fall in those bins they are ranked directly;
// otherwise the bisection of warp_median below takes over.
__device__ float warp_median(const float* buf, int na, float* cand, int lane);

__device__ float warp_median_hist(const float* buf, int na, int* hist, float* cand, int lane) {
    const int k0 = (na - 1) / 2, k1 = na / 2;
    float s = 0.f;
    for (int t = lane; t < na; t += 32) s += buf[t];
    s = warp_sum(s);
    const float mean = s / na;
    float q = 0.f;
    for (int t = lane; t < na; t += 32) { const float d = buf[t] - mean; q = fmaf(d, d, q); }
    q = warp_sum(q);
    const float sd = sqrtf(q / na);
    const float lo = mean - 2.0f * sd, width = (4.0f * sd) / 30.0f;
    const float inv = 1.0f / width;
    if (!(width > 0.f) || !isfinite(inv) || !isfinite(lo)) return warp_median(buf, na, cand, lane);
    auto bin = [&](float v) {  // 0: below lo, 1..30, 31: at or above lo + 30 width
        const float u = (v - lo) * inv;
        return u < 0.f ? 0 : (u >= 30.0f ? 31 : 1 + min((int)u, 29));
    };
    hist[lane] = 0;
    __syncwarp();
    for (int t = lane; t < na; t += 32) atomicAdd(&hist[bin(buf[t])], 1);
    __syncwarp();
    const int c = hist[lane];
    int cum = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, cum, o);
        if (lane >= o) cum += t;
    }
    const int before = cum - c;
    const unsigned m0 = __ballot_sync(0xffffffffu, before <= k0 && k0 < cum);
    const unsigned m1 = __ballot_sync(0xffffffffu, before <= k1 && k1 < cum);
    const int b0 = __ffs(m0) - 1, b1 = __ffs(m1) - 1;
    const int base = __shfl_sync(0xffffffffu, before, b0);
    const int m = __shfl_sync(0xffffffffu, cum, b1) - base;
    if (m > 32) return warp_median(buf, na, cand, lane);
    int nc = 0;
    for (int t0 = 0; t0 < na; t0 += 32) {
        const int t = t0 + lane;
        float v = 0.f;
        bool in = false;
        if (t < na) { v = buf[t]; const int b = bin(v); in = b >= b0 && b <= b1; }
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (in) cand[nc + __popc(bal & ((1u << lane) - 1u))] = v;
        nc += __popc(bal);
    }
    __syncwarp();
    const float mine = lane < m ? cand[lane] : INFINITY;
    int rank = 0;
    for (int u = 0; u < m; u++) {
        const float x = cand[u];
        rank += (x < mine) || (x == mine && u < lane);
    }
    const unsigned r0 = __ballot_sync(0xffffffffu, lane < m && rank == k0 - base);
    const unsigned r1 = __ballot_sync(0xffffffffu, lane < m && rank == k1 - base);
    const float v0 = __shfl_sync(0xffffffffu, mine, r0 ? __ffs(r0) - 1 : 0);
    const float v1 = __shfl_sync(0xffffffffu, mine, r1 ? __ffs(r1) - 1 : 0);
    __syncwarp();
    return (float)(0.5 * ((double)v0 + (double)v1));
}

// Median (Eq. 1) of the na values buf[0..na) held by one warp's shared buffer,
// exact.  Both middle order statistics x_k0, x_k1 (k0 = (na-1)/2, k1 = na/2)
// minimise sum |x - m|, so they lie within one standard deviation of the mean:
// the search starts from [mean - sd, mean + sd] (checked by counting, else the
// full range), halves the value interval while both ranks stay on one side, and
// finishes with a rank count over the at most 32 values left in the interval.
__device__ float warp_median(const float* buf, int na, float* cand, int lane) {
    const int k0 = (na - 1) / 2, k1 = na / 2;
    float s = 0.f, q = 0.f, mn = INFINITY, mx = -INFINITY;
    for (int t = lane; t < na; t += 32) {
        const float v = buf[t];
        s += v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    s = warp_sum(s);
    const float mean = s / na;
    for (int t = lane; t < na; t += 32) { const float d = buf[t] - mean; q = fmaf(d, d, q); }
    q = warp_sum(q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const float sd = sqrtf(q / na);
    auto count_lt = [&](float x) {
        int c = 0;
        for (int t = lane; t < na; t += 32) c += buf[t] < x;
        return __reduce_add_sync(0xffffffffu, c);
    };
    auto count_le = [&](float x) {
        int c = 0;
        for (int t = lane; t < na; t += 32) c += buf[t] <= x;
        return __reduce_add_sync(0xffffffffu, c);
    };
    // invariant: c_lt = #(v < L) <= k0 and k1 < c_le = #(v <= U)
    float L = fmaxf(mn, mean - sd * 1.001f - 1e-30f), U = fminf(mx, mean + sd * 1.001f + 1e-30f);
    int c_lt = count_lt(L), c_le = count_le(U);
    if (!(c_lt <= k0 && k1 < c_le)) { L = mn; U = mx; c_lt = 0; c_le = na; }
    for (int step = 0; step < 64 && c_le - c_lt > 32 && L < U; step++) {
        const float M = 0.5f * (L + U);
        if (!(M > L && M <= U)) break;
        const int c_m = count_lt(M);
        if (k1 < c_m) { U = nextafterf(M, -INFINITY); c_le = c_m; }
        else if (k0 >= c_m) { L = M; c_lt = c_m; }
        else {  // x_k0 < M <= x_k1: the two neighbours of M
            float a = -INFINITY, b = INFINITY;
            for (int t = lane; t < na; t += 32) {
                const float v = buf[t];
                if (v < M) a = fmaxf(a, v); else b = fminf(b, v);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
                b = fminf(b, __shfl_xor_sync(0xffffffffu, b, o));
            }
            return (float)(0.5 * ((double)a + (double)b));
        }
    }
    if (!(L < U)) return L;  // all values of the interval are equal
    if (c_le - c_lt > 32) {  // L and U adjacent floats: only the two values L and U are left
        const int cl = count_le(L);
        const float v0 = k0 < cl ? L : U, v1 = k1 < cl ? L : U;
        return (float)(0.5 * ((double)v0 + (double)v1));
    }
    // gather the values of [L, U] (at most 32 when the loop ends normally)
    int nc = 0;
    for (int base = 0; base < na; base += 32) {
        const int t = base + lane;
        const bool in = t < na && buf[t] >= L && buf[t] <= U;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        const int pos = nc + __popc(bal & ((1u << lane) - 1u));
        if (in && pos < 32) cand[pos] = buf[t];
        nc += __popc(bal);
    }
    __syncwarp();
    nc = min(nc, 32);
    const float mine = lane < nc ? cand[lane] : INFINITY;
    int rank = 0;
    for (int u = 0; u < nc; u++) {
        const float x = cand[u];
        rank += (x < mine) || (x == mine && u < lane);
    }
    const int r0 = k0 - c_lt, r1 = k1 - c_lt;
    const unsigned b0 = __ballot_sync(0xffffffffu, lane < nc && rank == r0);
    const unsigned b1 = __ballot_sync(0xffffffffu, lane < nc && rank == r1);
    const float v0 = __shfl_sync(0xffffffffu, mine, b0 ? __ffs(b0) - 1 : 0);
    const float v1 = __shfl_sync(0xffffffffu, mine, b1 ? __ffs(b1) - 1 : 0);
    __syncwarp();
    return (float)(0.5 * ((double)v0 + (double)v1));
}

// Warp 0: ordered list (row-major box order) of the offsets (di, dj), |di|,
// |dj| <= R, that satisfy pred; returns the count.  Deterministic order keeps
// the FP32 sums reproducible.
template <class P>
__device__ int build_offsets(int R, int16_t* out, int cap, int lane, P pred) {
    const int box = 2 * R + 1;
    int cnt = 0;
    for (int base = 0; base < box * box; base += 32) {
        const int idx = base + lane;
        const int di = idx / box - R, dj = idx % box - R;
        const bool take = idx < box * box && pred(di, dj);
        const unsigned bal = __ballot_sync(0xffffffffu, take);
        const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
        if (take && pos < cap) out[pos] = (int16_t)((di << 8) | (dj & 0xff));
        cnt += __popc(bal);
    }
    return min(cnt, cap);
}
// offsets packed as two signed bytes (|di|, |dj| <= 17)
__device__ __forceinline__ int off_di(int16_t o) { return o >> 8; }
__device__ __forceinline__ int off_dj(int16_t o) { return (int)(int8_t)(o & 0xff); }

// Area of the disk of radius r centred at the origin beyond the corner (u, v),
// u, v >= 0 (the region X >= u, Y >= v).  With a = sqrt(r^2 - u^2) and
// b = sqrt(r^2 - v^2) it is the right triangle (u, v), (u, a), (b, v) plus the
// circular segment between (u, a) and (b, v), whose angle phi has
// r^2 sin(phi) = a b - u v and r^2 cos(phi) = u b + a v:
//   K = (a - v)(b - u) / 2 + (r^2 phi - r^2 sin(phi)) / 2.
// A pixel's overlap is K(near corner) - K(x-far) - K(y-far) + K(far corner)
// after reflecting it into the first quadrant (splitting it at an axis it
// straddles), so one table of K over the corner grid of a source serves all its
// edge pixels.
__device__ __forceinline__ float corner_area(float u, float v, float r, float r2) {
    if (fmaf(u, u, v * v) >= r2) return 0.f;
    const float a = sqrtf((r - u) * (r + u)), b = sqrtf((r - v) * (r + v));
    const float sn = fmaf(a, b, -u * v), cs = fmaf(u, b, a * v);
    return 0.5f * ((a - v) * (b - u) + fmaf(r2, atan2f(sn, cs), -sn));
}

constexpr int AG_RMAX = 7;                    // corner grid for apertures with R1 <= 7 (r_ap < 7)
constexpr int AG_N = 2 * AG_RMAX + 2;         // grid lines per axis
constexpr int AG_SIZE = AG_N * AG_N + 2 * AG_N + 1;

// Overlap of edge pixel (di, dj) from a source's corner table: G[r][c] =
// K(|X_c|, |Y_r|) at the pixel-corner lines X_c = c - R1 - 1/2 - ox,
// Y_r = r - R1 - 1/2 - oy; A[r] = K(0, |Y_r|), B[c] = K(|X_c|, 0), K00 = K(0, 0).
__device__ __forceinline__ float grid_pixel_area(const float* tab, int R1, int di, int dj, float ox, float oy) {
    const int n = 2 * R1 + 2;
    const float* G = tab;
    const float* A = tab + n * n;
    const float* B = A + n;
    const float K00 = B[n];
    const int c0 = dj + R1, r0 = di + R1;
    const float xa = (float)dj - 0.5f - ox, ya = (float)di - 0.5f - oy;
    const bool xs = xa < 0.f && xa + 1.0f > 0.f, ys = ya < 0.f && ya + 1.0f > 0.f;  // straddles an axis
    const int cn = xa >= 0.f ? c0 : c0 + 1, cf = xa >= 0.f ? c0 + 1 : c0;
    const int rn = ya >= 0.f ? r0 : r0 + 1, rf = ya >= 0.f ? r0 + 1 : r0;
    float area;
    if (!xs && !ys) {
        area = (G[rn * n + cn] - G[rn * n + cf]) - (G[rf * n + cn] - G[rf * n + cf]);
    } else if (xs && !ys) {  // halves [0, |X_c0|] and [0, |X_c1|] in x
        area = 2.0f * (A[rn] - A[rf]) - (G[rn * n + c0] - G[rf * n + c0]) - (G[rn * n + c0 + 1] - G[rf * n + c0 + 1]);
    } else if (!xs && ys) {
        area = 2.0f * (B[cn] - B[cf]) - (G[r0 * n + cn] - G[r0 * n + cf]) - (G[(r0 + 1) * n + cn] - G[(r0 + 1) * n + cf]);
    } else {
        area = 4.0f * K00 - 2.0f * (B[c0] + B[c0 + 1]) - 2.0f * (A[r0] + A[r0 + 1]) +
               (G[r0 * n + c0] + G[r0 * n + c0 + 1] + G[(r0 + 1) * n + c0] + G[(r0 + 1) * n + c0 + 1]);
    }
    return fminf(fmaxf(area, 0.f), 1.f);
}

__device__ __forceinline__ void aperture_body(const PhotJob& J, int vb, int nvb) {
    extern __shared__ float ann_dyn[];        // [P_WARPS][J.ann_cap] annulus values
    __shared__ float cand[P_WARPS][32];
    __shared__ int hist[P_WARPS][32];
    __shared__ float ktab[P_WARPS][AG_SIZE];  // per-source corner table (apertures with R1 <= AG_RMAX)
    // pixel lists shared by the block, for any centre within 1/2 px of the anchor:
    // aperture pixels always inside the disk (weight 1), pixels the disk edge may
    // cross, and pixels whose centre may lie in the annulus
    __shared__ int16_t l_ap[ANN_CAP], l_ann[ANN_CAP];  // aperture: inner pixels, then edge pixels
    __shared__ int n_lists[3];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = (vb * P_THREADS + threadIdx.x) >> 5;
    const int nw = (nvb * P_THREADS) >> 5;
    const int n = min(*J.n_src_dev, J.max_src);
    float* buf = ann_dyn + (size_t)wib * J.ann_cap;
    const float Wf = (float)(int)J.W, Hf = (float)(int)J.H;
    const int R1 = (int)ceilf(J.r_ap + 1.0f) - 1;  // pixels reaching within r_ap
    const int R2 = (int)floorf(J.r_out + 0.5f);    // centres within r_out of any offset <= 1/2
    const double rin2d = __dmul_rn((double)J.r_in, (double)J.r_in);
    const double rout2d = __dmul_rn((double)J.r_out, (double)J.r_out);
    const float rin2 = (float)rin2d, rout2 = (float)rout2d;
    if (wib == 0) {
        const float r = J.r_ap, r2 = r * r;
        // nearest / farthest point of the pixel square from a centre within 1/2 px
        auto near2 = [](int di, int dj) {
            const float a = fmaxf(fabsf((float)dj) - 1.0f, 0.f), b = fmaxf(fabsf((float)di) - 1.0f, 0.f);
            return a * a + b * b;
        };
        auto far2 = [](int di, int dj) {
            const float a = fabsf((float)dj) + 1.0f, b = fabsf((float)di) + 1.0f;
            return a * a + b * b;
        };
        const int ni = build_offsets(R1, l_ap, ANN_CAP, lane, [&](int di, int dj) { return far2(di, dj) <= r2; });
        const int ne = build_offsets(R1, l_ap + ni, ANN_CAP - ni, lane, [&](int di, int dj) {
            return far2(di, dj) > r2 && near2(di, dj) < r2;
        });
        // annulus: the pixel centre's distance ranges over |p| +- sqrt(2)/2
        const int na = build_offsets(R2, l_ann, min(ANN_CAP, J.ann_cap), lane, [&](int di, int dj) {
            const float a = fmaxf(fabsf((float)dj) - 0.5f, 0.f), b = fmaxf(fabsf((float)di) - 0.5f, 0.f);
            const float c = fabsf((float)dj) + 0.5f, d = fabsf((float)di) + 0.5f;
            return a * a + b * b < rout2 * 1.0001f && c * c + d * d >= rin2 * 0.9999f;
        });
        if (lane == 0) { n_lists[0] = ni; n_lists[1] = ne; n_lists[2] = na; }
    }
    __syncthreads();
    const int ni = n_lists[0], ne = n_lists[1], nac = n_lists[2];
    for (int s = gw; s < n; s += nw) {
        const float x = J.x[s], y = J.y[s];
        const float ax = rintf(x), ay = rintf(y);
        const float ox = x - ax, oy = y - ay;
        const int64_t ia = (int)ay, ja = (int)ax;
        // aperture sum with exact overlap weights: inner pixels weigh 1; the
        // edge pixels' overlaps come from a table of corner areas of this source
        // (one K per grid corner instead of four per pixel), or, for large
        // apertures, pixel by pixel
        float sw = 0.f, swf = 0.f;
        const bool tab = R1 <= AG_RMAX;
        if (tab) {
            float* kt = ktab[wib];
            const int n = 2 * R1 + 2;
            const float r = J.r_ap, r2 = r * r;
            for (int t = lane; t < n * n + 2 * n + 1; t += 32) {
                float u, v;
                if (t < n * n) {
                    const int rr = t / n, cc = t - rr * n;
                    u = fabsf((float)(cc - R1) - 0.5f - ox);
                    v = fabsf((float)(rr - R1) - 0.5f - oy);
                } else if (t < n * n + n) {
                    u = 0.f; v = fabsf((float)(t - n * n - R1) - 0.5f - oy);
                } else if (t < n * n + 2 * n) {
                    u = fabsf((float)(t - n * n - n - R1) - 0.5f - ox); v = 0.f;
                } else {
                    u = 0.f; v = 0.f;
                }
                kt[t] = corner_area(u, v, r, r2);
            }
            __syncwarp();
        }
        for (int t = lane; t < ni + ne; t += 32) {
            const int16_t o = l_ap[t];
            const int di = off_di(o), dj = off_dj(o);
            const int64_t i = ia + di, j = ja + dj;
            if (i < 0 || i >= J.H || j < 0 || j >= J.W) continue;
            const float v = __ldg(J.sub + i * J.pitch + j);
            const float w = t < ni ? 1.0f
                            : (tab ? grid_pixel_area(ktab[wib], R1, di, dj, ox, oy)
                                   : circle_pixel_area(ox - (float)dj, oy - (float)di, J.r_ap));
            if (w > 0.f) {  // pixels outside the aperture never touch the sums
                sw += w;
                swf = fmaf(w, v, swf);
            }
        }
        __syncwarp();  // the table is rebuilt for the next source
        sw = warp_sum(sw);
        swf = warp_sum(swf);
        // annulus values into the warp's buffer, NCH loads per lane in flight
        int na = 0;
        {
            constexpr int NCH = 4;
            for (int base = 0; base < nac; base += 32 * NCH) {
                float v[NCH];
                bool take[NCH];
#pragma unroll
                for (int c = 0; c < NCH; c++) {
                    const int t = base + 32 * c + lane;
                    const int16_t o = t < nac ? l_ann[t] : (int16_t)0;
                    const int di = off_di(o), dj = off_dj(o);
                    const int64_t i = ia + di, j = ja + dj;
                    take[c] = t < nac && i >= 0 && i < J.H && j >= 0 && j < J.W &&
                              in_annulus((float)dj - ox, (float)di - oy, i, j, x, y, rin2, rout2, rin2d, rout2d);
                    v[c] = take[c] ? __ldg(J.sub + i * J.pitch + j) : 0.f;
                }
#pragma unroll
                for (int c = 0; c < NCH; c++) {
                    const unsigned bal = __ballot_sync(0xffffffffu, take[c]);
                    if (take[c]) buf[na + __popc(bal & ((1u << lane) - 1u))] = v[c];
                    na += __popc(bal);
                }
            }
        }
        __syncwarp();
        float skyv = 0.f;
        int fl = 0;
        if (na < J.min_ann) {
            fl |= IPP_FLAG_ANN_FEW;
        } else {
            skyv = warp_median_hist(buf, na, hist[wib], cand[wib], lane);
        }
        __syncwarp();
        const float Rm = fmaxf(J.r_ap, J.r_out);
        if (x - Rm < -0.5f || x + Rm > Wf - 0.5f || y - Rm < -0.5f || y + Rm > Hf - 0.5f)
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

__global__ void __launch_bounds__(P_THREADS) k_aperture(PhotJob J) { aperture_body(J, blockIdx.x, gridDim.x); }

// batched form: the same bodies over a table of frames
__global__ void __launch_bounds__(P_THREADS) k_centroid_rows_multi(const CenJob* J, const int* bs, int nf) {
    const int f = frame_of(bs, nf, blockIdx.x);
    centroid_rows_body(J[f], blockIdx.x - bs[f], bs[f + 1] - bs[f]);
}

__global__ void __launch_bounds__(P_THREADS) k_aperture_multi(const PhotJob* J, const int* bs, int nf) {
    const int f = frame_of(bs, nf, blockIdx.x);
    aperture_body(J[f], blockIdx.x - bs[f], bs[f + 1] - bs[f]);
}

// Stamp cut: one thread per stamp pixel, grid-stride over the device-resident
// count.  Consecutive threads take consecutive columns of a stamp row, so each
// stamp row is one short contiguous read of the frame.
__global__ void __launch_bounds__(P_THREADS) k_stamp_cut(const float* __restrict__ sub, int64_t W, int64_t H,
                                                          int64_t pitch, const int32_t* n_src_dev, int32_t max_src,
                                                          const float* __restrict__ x, const float* __restrict__ y,
                                                          int S, float* __restrict__ stamps,
                                                          float* __restrict__ weights, int32_t* __restrict__ origin,
                                                          int32_t* __restrict__ flags) {
    const int64_t n = min(*n_src_dev, max_src);
    const int SS = S * S, half = S / 2;
    const int64_t total = n * SS;
    for (int64_t t = (int64_t)blockIdx.x * P_THREADS + threadIdx.x; t < total; t += (int64_t)gridDim.x * P_THREADS) {
        const int64_t s = t / SS;
        const int pix = (int)(t - s * SS);
        const int r = pix / S, c = pix - r * S;
        const float xs = x[s], ys = y[s];
        const float lim = 1073741824.0f + (float)max(W, H);  // 2^30 px beyond the frame
        const bool pos_ok = isfinite(xs) && isfinite(ys) && fabsf(xs) < lim && fabsf(ys) < lim;
        int64_t ox = 0, oy = 0;
        if (pos_ok) {  // floor(v + 1/2) without the rounding of v + 0.5f: v - floor(v) is exact
            const float fx0 = floorf(xs), fy0 = floorf(ys);
            ox = (int64_t)fx0 + (xs - fx0 >= 0.5f) - half;
            oy = (int64_t)fy0 + (ys - fy0 >= 0.5f) - half;
        }
        const int64_t fy = oy + r, fx = ox + c;
        const bool in = pos_ok && fy >= 0 && fy < H && fx >= 0 && fx < W;
        stamps[t] = in ? __ldg(sub + fy * pitch + fx) : 0.f;
        if (weights) weights[t] = in ? 1.f : 0.f;
        if (pix == 0) {
            if (origin) { origin[2 * s] = (int32_t)ox; origin[2 * s + 1] = (int32_t)oy; }
            if (flags) {
                const bool inside = pos_ok && ox >= 0 && oy >= 0 && ox + S <= W && oy + S <= H;
                flags[s] = inside ? 0 : IPP_FLAG_EDGE;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Auto (Kron) photometry (Sec. 2.2.5 lists it; method paper-silent), three
// passes over small boxes of the subtracted frame (read through the caches
// right after the frame is written):
//   1. second moments of sub over the isophotal footprint (labels == k+1 in the
//      source's bounding box) about its barycentre; 1/12 is added to x2 and y2
//      when x2 y2 - xy^2 < 1/144 (a footprint thinner than a pixel);
//   2. Kron radius r1 = sum r f / sum f over in-frame pixels with elliptical
//      (Mahalanobis) radius r <= r_kmax,
//      r^2 = (y2 dx^2 - 2 xy dx dy + x2 dy^2) / (x2 y2 - xy^2);
//   3. flux and pixel count within r <= max(k_kron r1, r_min); EDGE when a
//      pixel centre inside that ellipse lies in the one-pixel border around
//      the frame.
// A warp takes a source whose footprint box has at most AUTO_BIG_BOX pixels;
// larger sources, whose Kron and aperture boxes run to tens of thousands of
// pixels, take a whole block, so that no single warp carries the tail of the
// launch.  Each thread sums its pixels in FP32 and
// the group adds them in a fixed order, leaving identical totals in every
// thread, so all threads take the same decisions afterwards.
constexpr int AUTO_BIG_BOX = 128;

// Integer points examined for an ellipse of half-widths `half` about c: one
// beyond each rounded end (the oracle's box), clipped to [lo_clip, hi_clip].
__device__ __forceinline__ void auto_box(float c, float half, int lo_clip, int hi_clip, int& lo, int& hi) {
    lo = max((int)fmaxf(floorf(c - half) - 1.0f, (float)lo_clip), lo_clip);
    hi = min((int)fminf(ceilf(c + half) + 1.0f, (float)hi_clip), hi_clip);
}

// Sum over the NT threads of a group (a warp, or a block of NT threads with
// `red` holding NT/32 floats of shared memory); every thread gets the total.
template <int NT>
__device__ __forceinline__ float auto_sum(float v, float* red) {
    v = warp_sum(v);
    if constexpr (NT == 32) {
        return v;
    } else {
        __syncthreads();  // earlier readers of red are done
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < NT / 32; w++) t += red[w];
        return t;
    }
}
template <int NT>
__device__ __forceinline__ bool auto_any(bool v) {
    if constexpr (NT == 32) return __any_sync(0xffffffffu, v);
    else return __syncthreads_or(v) != 0;
}

// The w x h box at (x0, y0), visited by the NT threads of a group (rank me) in
// raster order, four pixels a thread in flight: the values (and, for the
// footprint pass, the labels) of a step are loaded before any is used.  The
// box lies within the frame plus a one-pixel border, so 32-bit coordinates
// hold it (frames below 2^31 pixels).  (A column per thread, which keeps the
// column terms in registers, measured slower: narrow boxes leave most of a
// warp idle.)  fn(i, j, f, in_frame, in_footprint).
template <int NT, bool LAB, class Fn>
__device__ __forceinline__ void auto_visit(const AutoJob& J, int x0, int y0, int w, int h, int me, int32_t lab,
                                           Fn&& fn) {
    if (w <= 0 || h <= 0) return;
    const int n = w * h;
    const int dq = NT / w, dc = NT - dq * w;  // index + NT: dq rows and dc columns on
    const int W = (int)J.W, H = (int)J.H, pitch = (int)J.pitch;
    int r = me / w, c = me - r * w;
    for (int t0 = me; t0 < n; t0 += 4 * NT) {
        int ii[4], jj[4];
        bool ok[4], inf[4], inl[4];
        float f[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            ok[u] = t0 + u * NT < n;
            ii[u] = y0 + r;
            jj[u] = x0 + c;
            c += dc;
            r += dq;
            if (c >= w) { c -= w; r++; }
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            inf[u] = ok[u] && (unsigned)ii[u] < (unsigned)H && (unsigned)jj[u] < (unsigned)W;
            f[u] = inf[u] ? __ldg(J.sub + ((int64_t)ii[u] * pitch + jj[u])) : 0.f;
            inl[u] = LAB && inf[u] && __ldg(J.labels + ((int64_t)ii[u] * W + jj[u])) == lab;
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (ok[u]) fn(ii[u], jj[u], f[u], inf[u], inl[u]);
    }
}

template <int NT>
__device__ __forceinline__ void auto_source(const AutoJob& J, int64_t k, int me, float* red) {
    const float xb = __ldg(J.xbar + k), yb = __ldg(J.ybar + k);
    const int bx0 = __ldg(J.xmin + k), by0 = __ldg(J.ymin + k);
    const int bw = __ldg(J.xmax + k) - bx0 + 1, bh = __ldg(J.ymax + k) - by0 + 1;
    const int W = (int)J.W, H = (int)J.H;
    const int32_t lab = (int32_t)(k + 1);
    int fl = 0;
    // 1. footprint moments
    float s0 = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
    auto_visit<NT, true>(J, bx0, by0, bw, bh, me, lab, [&](int i, int j, float f, bool, bool inl) {
        if (!inl) return;
        const float dx = (float)j - xb, dy = (float)i - yb;
        s0 += f;
        sxx = fmaf(f * dx, dx, sxx);
        syy = fmaf(f * dy, dy, syy);
        sxy = fmaf(f * dx, dy, sxy);
    });
    s0 = auto_sum<NT>(s0, red); sxx = auto_sum<NT>(sxx, red);
    syy = auto_sum<NT>(syy, red); sxy = auto_sum<NT>(sxy, red);
    float x2, y2, xy;
    if (s0 > 0.f) {
        x2 = sxx / s0; y2 = syy / s0; xy = sxy / s0;
        if (x2 * y2 - xy * xy < 1.0f / 144.0f) { x2 += 1.0f / 12.0f; y2 += 1.0f / 12.0f; }
    } else {
        x2 = 1.0f / 12.0f; y2 = 1.0f / 12.0f; xy = 0.f;
        fl |= IPP_FLAG_KRON_BAD;
    }
    const float det = x2 * y2 - xy * xy;
    const float ca = y2 / det, cb = -2.0f * xy / det, cc = x2 / det;
    // 2. Kron radius (in-frame pixels only)
    float r1 = 0.f;
    if (!(fl & IPP_FLAG_KRON_BAD)) {
        int x0, x1, y0, y1;
        auto_box(xb, J.r_kmax * sqrtf(x2), 0, W - 1, x0, x1);
        auto_box(yb, J.r_kmax * sqrtf(y2), 0, H - 1, y0, y1);
        const float rk2 = J.r_kmax * J.r_kmax;
        float sr = 0.f, sf = 0.f;
        auto_visit<NT, false>(J, x0, y0, x1 - x0 + 1, y1 - y0 + 1, me, lab,
                              [&](int i, int j, float f, bool, bool) {
            const float dx = (float)j - xb, dy = (float)i - yb;
            const float q = fmaf(ca * dx, dx, fmaf(cb * dx, dy, cc * dy * dy));
            if (q > rk2) return;
            sr = fmaf(sqrtf(q), f, sr);
            sf += f;
        });
        sr = auto_sum<NT>(sr, red); sf = auto_sum<NT>(sf, red);
        if (sf > 0.f && sr > 0.f) r1 = sr / sf;
        else fl |= IPP_FLAG_KRON_BAD;
    }
    // 3. the automatic aperture (the frame and its one-pixel border)
    const float R = fmaxf(J.k_kron * r1, J.r_min), R2 = R * R;
    int x0, x1, y0, y1;
    auto_box(xb, R * sqrtf(x2), -1, W, x0, x1);
    auto_box(yb, R * sqrtf(y2), -1, H, y0, y1);
    float fs = 0.f, na = 0.f;
    bool edge = false;
    auto_visit<NT, false>(J, x0, y0, x1 - x0 + 1, y1 - y0 + 1, me, lab,
                          [&](int i, int j, float f, bool inf, bool) {
        const float dx = (float)j - xb, dy = (float)i - yb;
        const float q = fmaf(ca * dx, dx, fmaf(cb * dx, dy, cc * dy * dy));
        if (q > R2) return;
        if (!inf) { edge = true; return; }
        fs += f;
        na += 1.0f;
    });
    fs = auto_sum<NT>(fs, red); na = auto_sum<NT>(na, red);
    if (auto_any<NT>(edge)) fl |= IPP_FLAG_EDGE;
    if (me == 0) {
        J.flux[k] = fs;
        if (J.area) J.area[k] = na;
        if (J.kron) J.kron[k] = r1;
        if (J.shape) { J.shape[3 * k] = x2; J.shape[3 * k + 1] = y2; J.shape[3 * k + 2] = xy; }
        if (J.flags) J.flags[k] = fl;
    }
}

__device__ __forceinline__ bool auto_is_big(const AutoJob& J, int64_t k) {
    const int64_t bw = (int64_t)__ldg(J.xmax + k) - __ldg(J.xmin + k) + 1;
    const int64_t bh = (int64_t)__ldg(J.ymax + k) - __ldg(J.ymin + k) + 1;
    return bw * bh > AUTO_BIG_BOX;
}

// One launch: each block first takes the large sources of its grid-stride
// share as a block, then its warps take the small sources of theirs, so the
// blocks that meet no large source start on the small ones at once.
__global__ void __launch_bounds__(P_THREADS) k_auto_phot(AutoJob J) {
    __shared__ float red[P_WARPS];
    const int64_t nsrc = min((int64_t)__ldg(J.n_src_dev), (int64_t)J.max_src);
    for (int64_t k = blockIdx.x; k < nsrc; k += gridDim.x)
        if (auto_is_big(J, k)) auto_source<P_THREADS>(J, k, threadIdx.x, red);
    const int64_t nwarps = ((int64_t)gridDim.x * P_THREADS) >> 5;
    for (int64_t k = (((int64_t)blockIdx.x * P_THREADS) + threadIdx.x) >> 5; k < nsrc; k += nwarps)
        if (!auto_is_big(J, k)) auto_source<32>(J, k, threadIdx.x & 31, nullptr);
}

}  // namespace ipp

using namespace ipp;

static int persistent_blocks(cudaStream_t) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms * 4 : 512;
}

// A persistent grid of exactly the blocks that fit at once (one wave).
template <class K>
static int resident_blocks(K kernel, size_t smem) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, P_THREADS, smem) != cudaSuccess || per < 1) per = 1;
    return (sms > 0 ? sms : 132) * per;
}

int ipp_launch_centroid(const CenJob& J, cudaStream_t s) {
    const int R = (int)floorf(J.rad + 0.5f);
    const int nbox = (2 * R + 1) * (2 * R + 1);
    if (2 * R + 1 <= CR_BOX) k_centroid_rows<<<resident_blocks(k_centroid_rows, 0), P_THREADS, 0, s>>>(J);
    else if (nbox <= 32 * 4) k_centroid<4><<<resident_blocks(k_centroid<4>, 0), P_THREADS, 0, s>>>(J);
    else if (nbox <= 32 * 8) k_centroid<8><<<resident_blocks(k_centroid<8>, 0), P_THREADS, 0, s>>>(J);
    else k_centroid<0><<<persistent_blocks(s), P_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_centroid");
}

// annulus buffer per warp: the number of pixels whose centre can lie in the
// annulus for a centre within 1/2 px of the anchor (same test as the device list)
static int annulus_cap(const PhotJob& J) {
    const float rin2 = (float)((double)J.r_in * (double)J.r_in), rout2 = (float)((double)J.r_out * (double)J.r_out);
    const int R2 = (int)floorf(J.r_out + 0.5f);
    int cap = 0;
    for (int di = -R2; di <= R2; di++)
        for (int dj = -R2; dj <= R2; dj++) {
            const float a = fmaxf(fabsf((float)dj) - 0.5f, 0.f), b = fmaxf(fabsf((float)di) - 0.5f, 0.f);
            const float c = fabsf((float)dj) + 0.5f, d = fabsf((float)di) + 0.5f;
            cap += (a * a + b * b < rout2 * 1.0001f && c * c + d * d >= rin2 * 0.9999f);
        }
    return cap + 32;  // slack for host/device rounding differences of the test
}

int ipp_launch_aperture(const PhotJob& J0, cudaStream_t s) {
    if (J0.r_out > (float)ANN_MAXR) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "r_out above %d px", ANN_MAXR);
    PhotJob J = J0;
    J.ann_cap = annulus_cap(J);
    const size_t dyn = (size_t)P_WARPS * J.ann_cap * sizeof(float);
    cudaFuncSetAttribute(k_aperture, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    k_aperture<<<resident_blocks(k_aperture, dyn), P_THREADS, dyn, s>>>(J);
    return ipp_check_launch("k_aperture");
}

int ipp_launch_auto_phot(const AutoJob& J, cudaStream_t s) {
    if (J.max_src <= 0) return IPP_OK;
    k_auto_phot<<<resident_blocks(k_auto_phot, 0), P_THREADS, 0, s>>>(J);
    return ipp_check_launch("k_auto_phot");
}

int ipp_launch_stamp_cut(const float* sub, int64_t W, int64_t H, int64_t pitch, const int32_t* n_src_dev,
                         int32_t max_src, const float* x, const float* y, int S, float* stamps, float* weights,
                         int32_t* origin, int32_t* flags, cudaStream_t s) {
    if (max_src <= 0) return IPP_OK;
    const int64_t total = (int64_t)max_src * S * S;
    const int64_t blocks = std::min<int64_t>((total + P_THREADS - 1) / P_THREADS, (int64_t)persistent_blocks(s) * 4);
    k_stamp_cut<<<(unsigned)blocks, P_THREADS, 0, s>>>(sub, W, H, pitch, n_src_dev, max_src, x, y, S, stamps,
                                                        weights, origin, flags);
    return ipp_check_launch("k_stamp_cut");
}


// ---- batched form: tables and launches ----------------------------------------
// Per frame, blocks in proportion to its area (one per 64 K pixels, at least
// one), each striding over the frame's device-resident source count.
int ipp_phot_multi_pack(const CenJob* C, const PhotJob* P, int nf, HostBlob& hb, PhotMultiPlan* p) {
    if (nf < 1 || nf > 1024) return ipp_set_error(IPP_ERR_INVALID_ARG, "1..1024 frames");
    std::vector<PhotJob> Pj(P, P + nf);
    std::vector<int> nb(nf);
    for (int f = 0; f < nf; f++) {
        const int R = (int)floorf(C[f].rad + 0.5f);
        if (2 * R + 1 > CR_BOX) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "batched centroid window above 15 px");
        if (P[f].r_out > (float)ANN_MAXR) return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "r_out above %d px", ANN_MAXR);
        Pj[f].ann_cap = annulus_cap(P[f]);
        if (Pj[f].ann_cap != Pj[0].ann_cap) return ipp_set_error(IPP_ERR_INVALID_ARG, "mixed aperture params");
        nb[f] = (int)std::max<int64_t>(1, (C[f].W * C[f].H) >> 16);
    }
    p->cen = ipp_put_stage(hb, C, nb.data(), nf);
    p->ap = ipp_put_stage(hb, Pj.data(), nb.data(), nf);
    p->ap_smem = (size_t)P_WARPS * Pj[0].ann_cap * sizeof(float);
    p->nf = nf;
    return hb.ok() ? IPP_OK : ipp_set_error(IPP_ERR_INVALID_ARG, "batch table overflow");
}

int ipp_phot_multi_launch(const PhotMultiPlan& p, const unsigned char* t, cudaStream_t s) {
    k_centroid_rows_multi<<<(unsigned)p.cen.total, P_THREADS, 0, s>>>(
        reinterpret_cast<const CenJob*>(t + p.cen.jobs), reinterpret_cast<const int*>(t + p.cen.bs), p.nf);
    if (int e = ipp_check_launch("k_centroid_rows_multi")) return e;
    cudaFuncSetAttribute(k_aperture_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.ap_smem);
    k_aperture_multi<<<(unsigned)p.ap.total, P_THREADS, p.ap_smem, s>>>(
        reinterpret_cast<const PhotJob*>(t + p.ap.jobs), reinterpret_cast<const int*>(t + p.ap.bs), p.nf);
    return ipp_check_launch("k_aperture_multi");
}
