// spline.cuh -- evaluation of the natural tensor-product spline of the mesh
// nodes (Sec. 2.2.2's spline interpolation; the node table {f, Mx, My, Mxy} is
// built by k_spline_nodes in spline.cu).  Shared by the stand-alone map
// (spline.cu) and the fused subtraction / threshold pass (detect.cu).
#pragma once
#include "common.cuh"

namespace ipp {

// A 1-D natural spline at offset b from node k: (f0, M0) value and second
// derivative at node k, (f1, M1) at node k + 1; the cubic between them, and
// beyond the first (below) or last (above) node the line with the end slope.
__device__ __forceinline__ float nat_piece(float f0, float M0, float f1, float M1, float b) {
    const float a = 1.0f - b;
    return fmaf(a, f0, b * f1) + ((a * a * a - a) * M0 + (b * b * b - b) * M1) * (1.0f / 6.0f);
}
__device__ __forceinline__ float nat_eval(float f0, float M0, float f1, float M1, float b, bool below, bool above) {
    if (below) return f0 + b * ((f1 - f0) - (2.0f * M0 + M1) * (1.0f / 6.0f));            // b < 0
    if (above) return f1 + (b - 1.0f) * ((f1 - f0) + (M0 + 2.0f * M1) * (1.0f / 6.0f));  // b > 1
    return nat_piece(f0, M0, f1, M1, b);
}

// cell and offset along one axis: node k (0 <= k <= n - 2) and b = u - k, with
// the flags for u beyond the first or last node; n = 1 gives k = 0, b = 0
__device__ __forceinline__ void nat_cell(float u, int n, int* k, float* b, bool* below, bool* above) {
    if (n < 2) { *k = 0; *b = 0.f; *below = *above = false; return; }
    const int kk = min(max((int)floorf(u), 0), n - 2);
    *k = kk;
    *b = u - (float)kk;
    *below = u < 0.f;
    *above = u > (float)(n - 1);
}

__device__ __forceinline__ float spline_at(const float4* nodes, int nx, int ny, float u, float v) {
    int q, p;
    float bx, by;
    bool xb, xa, yb, ya;
    nat_cell(u, nx, &q, &bx, &xb, &xa);
    nat_cell(v, ny, &p, &by, &yb, &ya);
    const int q1 = min(q + 1, nx - 1), p1 = min(p + 1, ny - 1);
    float R[2], Ry[2];
#pragma unroll
    for (int s = 0; s < 2; s++) {
        const int pp = s ? p1 : p;
        const float4 A = __ldg(nodes + pp * nx + q), B = __ldg(nodes + pp * nx + q1);
        if (nx < 2) { R[s] = A.x; Ry[s] = A.z; continue; }
        R[s] = nat_eval(A.x, A.y, B.x, B.y, bx, xb, xa);     // along x: values with Mx
        Ry[s] = nat_eval(A.z, A.w, B.z, B.w, bx, xb, xa);    // along x: My with Mxy
    }
    if (ny < 2) return R[0];
    return nat_eval(R[0], Ry[0], R[1], Ry[1], by, yb, ya);   // along y
}

}  // namespace ipp
