// noalloc.cu -- ipp_bg_estimate_noalloc: the mesh background call without a
// caller-provided workspace, for callers that cannot allocate device memory.
//
// Its scratch (unfiltered mesh values and the filled grids, four float arrays
// of up to IPP_BG_NOALLOC_MAX_MESHES nodes) lives in one file-scope device array.
// Every GPU that loads this library holds that array (256 KiB) until the
// process exits.  Host code cannot use the array's name as a device address, so
// the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <mutex>

#include "checks.cuh"

namespace {

constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_bg_scratch[4 * IPP_BG_NOALLOC_MAX_MESHES];

std::mutex g_lock;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_bg_scratch on the current device (looked up once per device).
int scratch_for_current_device(float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "device ordinal %d above %d", dev, kMaxDevices - 1);
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bg_scratch);
        if (e != cudaSuccess || !p)
            return ipp_set_error(IPP_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return IPP_OK;
}

}  // namespace

extern "C" int ipp_bg_estimate_noalloc(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch,
                                       const uint8_t* mask, const ipp_calib* cal, const ipp_bg_params* p,
                                       float* mesh_bkg, float* mesh_rms, int32_t* status_dev, void* stream) {
    if (int e = check_frame(img, dtype, W, H, pitch, cal)) return e;
    if (int e = check_bg(p)) return e;
    if (!mesh_bkg || !mesh_rms) return ipp_set_error(IPP_ERR_INVALID_ARG, "mesh outputs NULL");
    const int64_t nx = ipp::cdiv(W, p->mesh_w), ny = ipp::cdiv(H, p->mesh_h);
    if (nx * ny > IPP_BG_NOALLOC_MAX_MESHES)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED,
                             "mesh grid of %lld x %lld = %lld nodes exceeds the no-allocation limit of %d nodes",
                             (long long)nx, (long long)ny, (long long)(nx * ny), IPP_BG_NOALLOC_MAX_MESHES);
    float* scratch = nullptr;
    if (int e = scratch_for_current_device(&scratch)) return e;
    float* raw_bkg = scratch;
    float* raw_rms = scratch + IPP_BG_NOALLOC_MAX_MESHES;
    float* fill_bkg = scratch + 2 * IPP_BG_NOALLOC_MAX_MESHES;
    float* fill_rms = scratch + 3 * IPP_BG_NOALLOC_MAX_MESHES;
    // nothing here must start at zero: each call writes every scratch element it reads
    ipp::MeshJob J;
    J.img = img; J.dtype = dtype; J.W = W; J.H = H; J.pitch = pitch; J.mask = mask;
    J.bias_map = cal ? cal->bias_map : nullptr; J.bias = cal ? cal->bias : 0.f;
    J.inv_flat = cal ? cal->inv_flat : nullptr;
    J.mesh_w = p->mesh_w; J.mesh_h = p->mesh_h; J.nx = (int)nx; J.ny = (int)ny;
    J.maxiters = p->maxiters; J.min_valid = p->min_valid; J.estimator = p->estimator;
    J.nsigma = p->nsigma; J.mf = p->median_factor; J.mnf = p->mean_factor;
    J.raw_bkg = raw_bkg; J.raw_rms = raw_rms;
    cudaStream_t s = (cudaStream_t)stream;
    if (int e = ipp_launch_mesh_stats(J, s)) return e;
    return ipp_launch_mesh_filter(raw_bkg, raw_rms, fill_bkg, fill_rms, (int)nx, (int)ny, p->filter_w, p->filter_h,
                                  mesh_bkg, mesh_rms, status_dev, s);
}
