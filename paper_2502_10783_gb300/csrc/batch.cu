// batch.cu -- the catalog path over a batch of independent frames, in two forms:
//   streams: a runner that spreads frames over its own CUDA streams (largest
//     frames first, each to the least-loaded lane), fork/join with events around
//     the caller's stream, and a lane-count autotuner;
//   table: one launch per stage for a group of frames -- a device table holds
//     every frame's jobs, each block finds its frame by binary search over the
//     frames' first blocks and runs the per-frame kernel body on it; the frames
//     are split into one group per lane, each group's ~17 launches on the
//     lane's stream, so stages of different groups overlap.
// Either form can be recorded as one CUDA graph.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "jobs.cuh"

struct ipp_batch_s {
    int lanes = 0;
    cudaStream_t st[IPP_BATCH_MAX_LANES] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[IPP_BATCH_MAX_LANES] = {};
    cudaGraphExec_t exec = nullptr;
    // table form: pinned staging of the device table, and what was uploaded last
    unsigned char* stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t staged = nullptr;    // the last upload has left the staging buffer
    bool stage_busy = false;
    std::vector<unsigned char> last;
    const void* last_dev = nullptr;
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
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->stage) cudaFreeHost(b->stage);
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


// ---- table form -----------------------------------------------------------------
namespace {

size_t table_bytes(int32_t n) { return a256((size_t)n * 6144 + 65536 * IPP_BATCH_MAX_LANES); }

// Builds the batch's table in the runner's pinned staging buffer, uploads it
// to the head of ws unless it equals the table uploaded there last, and
// enqueues the stages.  upload_only: stop after the upload (capture set-up).
struct TablePlan {
    int nf = 0;
    ipp::BgMultiPlan bg;
    ipp::DetMultiPlan det;
    ipp::PhotMultiPlan ph;
};

// the groups' stages, each on its lane's stream, forked from and joined to s
int launch_table(ipp_batch b, const TablePlan* plans, const unsigned char* dtab, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (int l = 0; l < b->lanes && e == cudaSuccess; l++) e = cudaStreamWaitEvent(b->st[l], b->fork, 0);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "table fork: %s", cudaGetErrorString(e));
    int status = IPP_OK;
    for (int l = 0; l < b->lanes && status == IPP_OK; l++) {
        if (plans[l].nf == 0) continue;
        status = ipp_bg_multi_launch(plans[l].bg, dtab, b->st[l]);
        if (status == IPP_OK) status = ipp_detect_multi_launch(plans[l].det, dtab, b->st[l]);
        if (status == IPP_OK) status = ipp_phot_multi_launch(plans[l].ph, dtab, b->st[l]);
    }
    for (int l = 0; l < b->lanes; l++) {   // joined also after an error (a capture stays well formed)
        cudaEventRecord(b->join[l], b->st[l]);
        cudaStreamWaitEvent(s, b->join[l], 0);
    }
    return status;
}

int run_table(ipp_batch b, const ipp_frame_desc* f, int32_t n, const ipp_bg_params* bp, const ipp_det_params* dp,
              const ipp_cen_params* cp, const ipp_phot_params* pp, int32_t max_src, void* ws, size_t ws_bytes,
              cudaStream_t s, bool upload_only, TablePlan* plans) {
    using namespace ipp;
    int64_t mw = 0, mh = 0;
    if (int e = check_frames(f, n, &mw, &mh)) return e;
    if (n == 0) return IPP_OK;
    if (n > 1024) return ipp_set_error(IPP_ERR_INVALID_ARG, "at most 1024 frames in the table form");
    if (!ws || ((uintptr_t)ws & 255)) return ipp_set_error(IPP_ERR_INVALID_ARG, "workspace NULL or misaligned");
    const size_t tb = table_bytes(n);
    std::vector<MeshJob> M(n);
    std::vector<MeshFilterJob> F(n);
    std::vector<DetectArgs> A(n);
    std::vector<CenJob> C(n);
    std::vector<PhotJob> P(n);
    size_t off = tb;
    for (int i = 0; i < n; i++) {
        const size_t need = a256(ipp_extract_workspace_size(f[i].W, f[i].H, bp));
        if (off + need > ws_bytes) return ipp_set_error(IPP_ERR_INVALID_ARG, "workspace too small at frame %d", i);
        int st = ipp_extract_jobs(f[i].img, f[i].dtype, f[i].W, f[i].H, f[i].pitch, f[i].cal, bp, dp, cp, pp, max_src,
                                  &f[i].out, (unsigned char*)ws + off, need, &M[i], &F[i], &A[i], &C[i], &P[i]);
        if (st != IPP_OK) {
            char msg[512];
            snprintf(msg, sizeof(msg), "%s", ipp_last_error_detail());
            return ipp_set_error(st, "frame %d: %s", i, msg);
        }
        off += need;
    }
    // the staging buffer is reused only once the previous upload has read it
    if (b->stage_busy) {
        cudaEventSynchronize(b->staged);
        b->stage_busy = false;
    }
    if (b->stage_cap < tb) {
        if (b->stage) cudaFreeHost(b->stage);
        b->stage = nullptr;
        b->stage_cap = 0;
        if (cudaMallocHost(&b->stage, tb) != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "pinned table staging");
        b->stage_cap = tb;
    }
    // frames in groups, one per lane (largest first to the least-loaded lane),
    // each group a table of its own on the lane's stream: the stages of one
    // group overlap those of the others
    const std::vector<int> lane = assign_lanes(f, n, b->lanes);
    HostBlob hb;
    hb.h = b->stage;
    hb.cap = tb;
    for (int l = 0; l < b->lanes; l++) {
        std::vector<MeshJob> gM;
        std::vector<MeshFilterJob> gF;
        std::vector<DetectArgs> gA;
        std::vector<CenJob> gC;
        std::vector<PhotJob> gP;
        for (int i = 0; i < n; i++) {
            if (lane[i] != l) continue;
            gM.push_back(M[i]); gF.push_back(F[i]); gA.push_back(A[i]); gC.push_back(C[i]); gP.push_back(P[i]);
        }
        TablePlan& tp = plans[l];
        tp.nf = (int)gM.size();
        if (tp.nf == 0) continue;
        if (int e = ipp_bg_multi_pack(gM.data(), gF.data(), tp.nf, hb, &tp.bg)) return e;
        if (int e = ipp_detect_multi_pack(gA.data(), tp.nf, hb, &tp.det)) return e;
        if (int e = ipp_phot_multi_pack(gC.data(), gP.data(), tp.nf, hb, &tp.ph)) return e;
    }
    const bool same = b->last_dev == ws && b->last.size() == hb.used && memcmp(b->last.data(), hb.h, hb.used) == 0;
    if (!same) {
        cudaError_t e = cudaMemcpyAsync(ws, hb.h, hb.used, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->staged, s);
        if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "table upload: %s", cudaGetErrorString(e));
        b->stage_busy = true;
        b->last.assign(hb.h, hb.h + hb.used);
        b->last_dev = ws;
    }
    if (upload_only) return IPP_OK;
    return launch_table(b, plans, static_cast<const unsigned char*>(ws), s);
}

int ensure_stage_event(ipp_batch b) {
    if (b->staged) return IPP_OK;
    if (cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess)
        return ipp_set_error(IPP_ERR_CUDA, "event create");
    return IPP_OK;
}

}  // namespace

extern "C" size_t ipp_batch_table_workspace_size(const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp) {
    if (!frames || !bp || n < 0 || n > 1024) return 0;
    size_t t = table_bytes(n);
    for (int i = 0; i < n; i++) {
        if (frames[i].W <= 0 || frames[i].H <= 0) return 0;
        t += a256(ipp_extract_workspace_size(frames[i].W, frames[i].H, bp));
    }
    return t;
}

extern "C" int ipp_batch_table_extract(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                                       const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                                       int32_t max_src, void* ws, size_t ws_bytes, void* stream) {
    if (!b) return ipp_set_error(IPP_ERR_INVALID_ARG, "batch runner NULL");
    if (int e = ensure_stage_event(b)) return e;
    TablePlan plans[IPP_BATCH_MAX_LANES];
    return run_table(b, frames, n, bp, dp, cp, pp, max_src, ws, ws_bytes, (cudaStream_t)stream, false, plans);
}

extern "C" int ipp_batch_table_capture(ipp_batch b, const ipp_frame_desc* frames, int32_t n, const ipp_bg_params* bp,
                                       const ipp_det_params* dp, const ipp_cen_params* cp, const ipp_phot_params* pp,
                                       int32_t max_src, void* ws, size_t ws_bytes, void* stream) {
    if (!b) return ipp_set_error(IPP_ERR_INVALID_ARG, "batch runner NULL");
    if (!stream) return ipp_set_error(IPP_ERR_INVALID_ARG, "capture needs a stream other than the legacy default");
    if (int e = ensure_stage_event(b)) return e;
    cudaStream_t s = (cudaStream_t)stream;
    // the table is uploaded before the capture, so the graph holds only the stages
    TablePlan plans[IPP_BATCH_MAX_LANES];
    if (int e = run_table(b, frames, n, bp, dp, cp, pp, max_src, ws, ws_bytes, s, true, plans)) return e;
    if (n == 0) return IPP_OK;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return ipp_set_error(IPP_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    const int status = launch_table(b, plans, static_cast<const unsigned char*>(ws), s);
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
    // a later upload to the same workspace must not be skipped: the graph reads
    // the table uploaded here, which stays in place
    return IPP_OK;
}
