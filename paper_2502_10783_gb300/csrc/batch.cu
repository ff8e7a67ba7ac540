// batch.cu -- the catalog path over a batch of independent frames: a runner
// that spreads frames over its own CUDA streams (largest frames first, each to
// the least-loaded lane), fork/join with events around the caller's stream, an
// optional CUDA graph of a whole batch, and a lane-count autotuner.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "jobs.cuh"

struct ipp_batch_s {
    int lanes = 0;
    cudaStream_t st[IPP_BATCH_MAX_LANES] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[IPP_BATCH_MAX_LANES] = {};
    cudaGraphExec_t exec = nullptr;
};

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int check_frames(const ipp_frame_desc* f, int32_t n, int64_t* maxW, int64_t* maxH) {
    if (!f || n < 0) return ipp_set_error(IPP_ERR_INVALID_ARG, "frames NULL or n < 0");
    int64_t mw = 0, mh = 0;
    for (int i = 0; i < n; i++) {
        if (!f[i].img || f[i].W <= 0 || f[i].H <= 0 || f[i].pitch < f[i].W)
            return ipp_set_error(IPP_ERR_INVALID_ARG, "frame %d: bad image or size", i);
        mw = std::max(mw, f[i].W);
        mh = std::max(mh, f[i].H);
    }
    *maxW = mw;
    *maxH = mh;
    return IPP_OK;
}

// frames in descending pixel count, each to the lane with the fewest pixels so far
std::vector<int> assign_lanes(const ipp_frame_desc* f, int32_t n, int lanes) {
    std::vector<int> order(n), lane(n, 0);
    for (int i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return f[a].W * f[a].H > f[b].W * f[b].H; });
    std::vector<int64_t> load(lanes, 0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane[i] = l;
        load[l] += f[i].W * f[i].H;
    }
    return lane;
}

int run(ipp_batch b, const ipp_frame_desc* f, int32_t n, const ipp_bg_params* bp, const ipp_det_params* dp,
        const ipp_cen_params* cp, const ipp_phot_params* pp, int32_t max_src, void* ws, size_t ws_bytes,
        cudaStream_t s) {
    int64_t mw = 0, mh = 0;
    if (int e = check_frames(f, n, &mw, &mh)) return e;
    if (n == 0) return IPP_OK;
    const size_t per = a256(ipp_extract_workspace_size(mw, mh, bp));
    if (!ws || ws_bytes < per * (size_t)b->lanes)
        return ipp_set_error(IPP_ERR_INVALID_ARG, "workspace of %zu bytes needed", per * (size_t)b->lanes);
    const std::vector<int> lane = assign_lanes(f, n, b->lanes);
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (int l = 0; l < b->lanes && e == cudaSuccess; l++) e = cudaStreamWaitEvent(b->st[l], b->fork, 0);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "batch fork: %s", cudaGetErrorString(e));
    int status = IPP_OK;
    for (int i = 0; i < n && status == IPP_OK; i++) {
        unsigned char* w = (unsigned char*)ws + per * (size_t)lane[i];
        status = ipp_extract(f[i].img, f[i].dtype, f[i].W, f[i].H, f[i].pitch, f[i].cal, bp, dp, cp, pp, max_src,
                             &f[i].out, w, per, b->st[lane[i]]);
        if (status != IPP_OK) {
            char msg[512];
            snprintf(msg, sizeof(msg), "%s", ipp_last_error_detail());
            ipp_set_error(status, "frame %d: %s", i, msg);
        }
    }
    // join every lane back to the caller's stream (also after an error, so
    // that a capture in progress stays well formed)
    for (int l = 0; l < b->lanes; l++) {
        cudaEventRecord(b->join[l], b->st[l]);
        cudaStreamWaitEvent(s, b->join[l], 0);
    }
    return status;
}

}  // namespace

extern "C" size_t ipp_batch_workspace_size(int64_t max_W, int64_t max_H, const ipp_bg_params* bp, int32_t lanes) {
    if (!bp || max_W <= 0 || max_H <= 0 || lanes < 1 || lanes > IPP_BATCH_MAX_LANES) return 0;
    return a256(ipp_extract_workspace_size(max_W, max_H, bp)) * (size_t)lanes;
}

extern "C" int ipp_batch_create(int32_t lanes, ipp_batch* out) {
    if (!out || lanes < 1 || lanes > IPP_BATCH_MAX_LANES)
        return ipp_set_error(IPP_ERR_INVALID_ARG, "lanes must be 1..%d", IPP_BATCH_MAX_LANES);
    ipp_batch b = new ipp_batch_s;
    b->lanes = lanes;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int l = 0; l < lanes && e == cudaSuccess; l++) {
        e = cudaStreamCreateWithFlags(&b->st[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[l], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        ipp_batch_destroy(b);
        return ipp_set_error(IPP_ERR_CUDA, "batch create: %s", cudaGetErrorString(e));
    }
    *out = b;
    return IPP_OK;
}

extern "C" int ipp_batch_destroy(ipp_batch b) {
    if (!b) return IPP_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (int l = 0; l < IPP_BATCH_MAX_LANES; l++) {
        if (b->join[l]) cudaEventDestroy(b->join[l]);
        if (b->st[l]) cudaStreamDestroy(b->st[l]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return IPP_OK;
}

extern "C" int ipp_batch_extract(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                                 const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                                 int32_t max_src, void* ws, size_t ws_bytes, void* stream) {
    if (!b) return ipp_set_error(IPP_ERR_INVALID_ARG, "batch runner NULL");
    return run(b, frames, n, bp, dp, cp, pp, max_src, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" int ipp_batch_capture(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                                 const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                                 int32_t max_src, void* ws, size_t ws_bytes, void* stream) {
    if (!b) return ipp_set_error(IPP_ERR_INVALID_ARG, "batch runner NULL");
    if (!stream) return ipp_set_error(IPP_ERR_INVALID_ARG, "capture needs a stream other than the legacy default");
    int64_t mw = 0, mh = 0;
    if (int e = check_frames(frames, n, &mw, &mh)) return e;
    cudaStream_t s = (cudaStream_t)stream;
    // kernels configured once before the capture (attributes are not stream work)
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    const int status = run(b, frames, n, bp, dp, cp, pp, max_src, ws, ws_bytes, s);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (status != IPP_OK) {
        if (g) cudaGraphDestroy(g);
        return status;
    }
    if (e != cudaSuccess || !g) return ipp_set_error(IPP_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = x;
    return IPP_OK;
}

extern "C" int ipp_batch_launch(ipp_batch b, void* stream) {
    if (!b || !b->exec) return ipp_set_error(IPP_ERR_INVALID_ARG, "no captured batch");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return IPP_OK;
}

extern "C" int ipp_batch_autotune(const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                                  const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                                  int32_t max_src, void* ws, size_t ws_bytes, void* stream, int32_t* best_lanes,
                                  float* ms_per_lanes) {
    if (!best_lanes) return ipp_set_error(IPP_ERR_INVALID_ARG, "best_lanes NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const int cand[4] = {1, 2, 4, 8};
    float best = 0.f;
    int bl = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int status = IPP_OK;
    for (int c = 0; c < 4 && status == IPP_OK; c++) {
        ipp_batch b = nullptr;
        if ((status = ipp_batch_create(cand[c], &b)) != IPP_OK) break;
        status = run(b, frames, n, bp, dp, cp, pp, max_src, ws, ws_bytes, s);  // warm-up
        if (status == IPP_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2 && status == IPP_OK; r++)
                status = run(b, frames, n, bp, dp, cp, pp, max_src, ws, ws_bytes, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms *= 0.5f;
            if (ms_per_lanes) ms_per_lanes[c] = ms;
            if (c == 0 || ms < best) { best = ms; bl = cand[c]; }
        }
        cudaStreamSynchronize(s);
        ipp_batch_destroy(b);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status == IPP_OK) *best_lanes = bl;
    return status;
}
