// spline.cu -- the natural-spline background map (Sec. 2.2.2: the filtered mesh
// is scaled back to full resolution by spline interpolation; this is the
// natural cubic spline reading, beside the default Keys cubic of bg.cu).
//
// The map is the tensor product of 1-D natural cubic splines through the mesh
// nodes (node (p, q) at pixel ((q + 1/2) mesh_w - 1/2, (p + 1/2) mesh_h - 1/2),
// unit spacing in node coordinates, zero second derivative at the end nodes,
// continued beyond them as the line with the end slope).  On a cell it is fixed
// by four numbers at each of its four corner nodes: the value f, the second
// derivatives Mx (along x) and My (along y), and the mixed fourth derivative
// Mxy.  k_spline_nodes computes that table once per call (tridiagonal solves,
// a thread per node row or column); k_bg_subtract_spline then evaluates the map
// at each pixel from its cell's sixteen numbers and writes f - B.
#include "jobs.cuh"
#include "spline.cuh"

namespace ipp {

constexpr int SP_THREADS = 256;

// Thomas coefficients of the natural-spline system of n nodes (they depend on
// the position only): c_1 = 1/4, c_k = 1 / (4 - c_{k-1}).
__device__ void nat_coef(int n, float* c) {
    float pc = 0.f;
    for (int k = 1; k <= n - 2; k++) {
        c[k] = 1.0f / (4.0f - (k > 1 ? pc : 0.f));
        pc = c[k];
    }
}

// Natural-spline second derivatives of n values y[k * ys] into M[k * ms]:
// M_0 = M_{n-1} = 0, M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1})
// (Thomas algorithm with the shared coefficients c of nat_coef).
__device__ void nat_m(const float* y, int ys, int n, float* M, int ms, const float* c) {
    for (int k = 0; k < n; k++) M[k * ms] = 0.f;
    if (n < 3) return;
    float pd = 0.f;
    for (int k = 1; k <= n - 2; k++) {
        const float r = 6.0f * ((y[(k + 1) * ys] - y[k * ys]) - (y[k * ys] - y[(k - 1) * ys]));
        const float dk = (r - (k > 1 ? pd : 0.f)) * c[k];
        M[k * ms] = dk;
        pd = dk;
    }
    for (int k = n - 3; k >= 1; k--) M[k * ms] -= c[k] * M[(k + 1) * ms];
}

// One block: node table {f, Mx, My, Mxy} of an ny x nx grid (row-major).
// scratch: nx ny + nx + ny floats (Mx, then the coefficients along x and y).
__global__ void __launch_bounds__(SP_THREADS) k_spline_nodes(const float* mesh, int nx, int ny, float4* nodes,
                                                             float* scratch) {
    float* mx = scratch;            // Mx, row-major [ny][nx]
    float* cx = scratch + nx * ny;  // coefficients along x [nx]
    float* cy = cx + nx;            // coefficients along y [ny]
    if (threadIdx.x == 0) nat_coef(nx, cx);
    if (threadIdx.x == 32) nat_coef(ny, cy);
    __syncthreads();
    float* nf = reinterpret_cast<float*>(nodes);
    // Mx along each node row, My (node .z) along each node column
    for (int t = threadIdx.x; t < ny + nx; t += SP_THREADS) {
        if (t < ny) nat_m(mesh + t * nx, 1, nx, mx + t * nx, 1, cx);
        else nat_m(mesh + (t - ny), nx, ny, nf + 2 + 4 * (t - ny), 4 * nx, cy);
    }
    __syncthreads();
    // Mxy (node .w): second derivatives along y of the Mx values of each column
    for (int q = threadIdx.x; q < nx; q += SP_THREADS) nat_m(mx + q, nx, ny, nf + 3 + 4 * q, 4 * nx, cy);
    __syncthreads();
    for (int k = threadIdx.x; k < nx * ny; k += SP_THREADS) {
        nf[4 * k] = mesh[k];
        nf[4 * k + 1] = mx[k];
    }
}

__device__ __forceinline__ float spline_pix(const SubJob& J, int64_t y, int64_t x) {
    if (J.dtype == IPP_F32) return __ldg(reinterpret_cast<const float*>(J.img) + y * J.pitch + x);
    const float raw = (float)__ldg(reinterpret_cast<const uint16_t*>(J.img) + y * J.pitch + x);
    const float b = J.bias_map ? __ldg(J.bias_map + y * J.W + x) : J.bias;
    return (raw - b) * __ldg(J.inv_flat + y * J.W + x);
}

// a thread per 4 consecutive pixels of a row, 8 rows per block of 256
__global__ void __launch_bounds__(SP_THREADS) k_bg_subtract_spline(SubJob J, const float4* nodes) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t y = (int64_t)blockIdx.y * (SP_THREADS / 32) + warp;
    const int64_t x0 = ((int64_t)blockIdx.x * 32 + lane) * 4;
    if (y >= J.H || x0 >= J.W) return;
    const float v = ((float)y + 0.5f) / J.mesh_h - 0.5f;
    float B[4], f[4];
    const bool vec = J.dtype == IPP_F32 && (J.pitch % 4 == 0) && (J.sub_pitch % 4 == 0) &&
                     (((uintptr_t)J.img & 15) == 0) && (((uintptr_t)J.sub & 15) == 0) &&
                     (!J.bkg_map || ((uintptr_t)J.bkg_map & 15) == 0) && x0 + 4 <= J.W;
    if (vec) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(J.img) + y * J.pitch + x0));
        f[0] = t.x; f[1] = t.y; f[2] = t.z; f[3] = t.w;
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int64_t x = x0 + c;
        if (x >= J.W) continue;
        if (!vec) f[c] = spline_pix(J, y, x);
        B[c] = spline_at(nodes, J.nx, J.ny, ((float)x + 0.5f) / J.mesh_w - 0.5f, v);
    }
    if (vec) {
        *reinterpret_cast<float4*>(J.sub + y * J.sub_pitch + x0) =
            make_float4(f[0] - B[0], f[1] - B[1], f[2] - B[2], f[3] - B[3]);
        if (J.bkg_map) *reinterpret_cast<float4*>(J.bkg_map + y * J.sub_pitch + x0) = make_float4(B[0], B[1], B[2], B[3]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int64_t x = x0 + c;
            if (x >= J.W) continue;
            J.sub[y * J.sub_pitch + x] = f[c] - B[c];
            if (J.bkg_map) J.bkg_map[y * J.sub_pitch + x] = B[c];
        }
    }
}

}  // namespace ipp

using namespace ipp;

size_t ipp_spline_ws_bytes(int nx, int ny) {
    const size_t n = (size_t)nx * ny;
    return ((n * sizeof(float4) + 255) & ~(size_t)255) + (n + nx + ny) * sizeof(float);
}

// the node table of an nx x ny grid at the head of ws (ipp_spline_ws_bytes)
int ipp_launch_spline_nodes(const float* mesh, int nx, int ny, void* ws, cudaStream_t s) {
    const size_t n = (size_t)nx * ny;
    float4* nodes = static_cast<float4*>(ws);
    float* scratch = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + ((n * sizeof(float4) + 255) & ~(size_t)255));
    k_spline_nodes<<<1, SP_THREADS, 0, s>>>(mesh, nx, ny, nodes, scratch);
    return ipp_check_launch("k_spline_nodes");
}

int ipp_launch_bg_subtract_spline(const SubJob& J, void* ws, cudaStream_t s) {
    const size_t n = (size_t)J.nx * J.ny;
    float4* nodes = static_cast<float4*>(ws);
    float* scratch = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + ((n * sizeof(float4) + 255) & ~(size_t)255));
    k_spline_nodes<<<1, SP_THREADS, 0, s>>>(J.mesh, J.nx, J.ny, nodes, scratch);
    if (int e = ipp_check_launch("k_spline_nodes")) return e;
    dim3 g((unsigned)((J.W + 127) / 128), (unsigned)((J.H + SP_THREADS / 32 - 1) / (SP_THREADS / 32)));
    k_bg_subtract_spline<<<g, SP_THREADS, 0, s>>>(J, nodes);
    return ipp_check_launch("k_bg_subtract_spline");
}
