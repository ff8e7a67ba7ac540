// jobs.cuh -- argument bundles passed from the C ABI (api.cu) to the kernel
// launchers of each translation unit, and the launchers' declarations.
#pragma once
#include <string.h>
#include "common.cuh"

namespace ipp {

struct MeshJob {
    const void* img;
    int dtype;
    int64_t W, H, pitch;
    const uint8_t* mask;
    const float* bias_map;
    float bias;
    const float* inv_flat;
    int mesh_w, mesh_h, nx, ny;
    int maxiters, min_valid, estimator;
    double nsigma, mf, mnf;
    float* raw_bkg;  // [ny*nx]
    float* raw_rms;  // [ny*nx], -1 marks an invalid mesh
};

struct SubJob {
    const void* img;
    int dtype;
    int64_t W, H, pitch;
    const float* bias_map;
    float bias;
    const float* inv_flat;
    const float* mesh;
    int nx, ny, mesh_w, mesh_h;
    float* sub;
    int64_t sub_pitch;
    float* bkg_map;
};

struct CenJob {
    const float* sub;
    int64_t W, H, pitch;
    const int32_t* n_src_dev;
    int32_t max_src;
    const float* x0;
    const float* y0;
    float sw, rad, tol2;
    int max_iter;
    float* x;
    float* y;
    int32_t* niter;
    int32_t* flags;
};

struct PhotJob {
    const float* sub;
    int64_t W, H, pitch;
    const int32_t* n_src_dev;
    int32_t max_src;
    const float* x;
    const float* y;
    float r_ap, r_in, r_out;
    int min_ann;
    int ann_cap;  // annulus values one warp can gather (set by the launcher)
    float* flux;
    float* sky;
    float* area;
    int32_t* n_ann;
    int32_t* flags;
};

struct AutoJob {
    const float* sub;
    const int32_t* labels;  // pitch W
    int64_t W, H, pitch;
    const int32_t* n_src_dev;
    int32_t max_src;
    const int32_t *xmin, *xmax, *ymin, *ymax;
    const float *xbar, *ybar;
    float k_kron, r_min, r_kmax;
    float* flux;
    float* area;
    float* kron;
    float* shape;  // nullable: x2, y2, xy per source
    int32_t* flags;
};

// Deblending workspace: per-candidate arrays of max_src entries and per-slot
// arrays of W*H entries (a candidate's pixels take slots [base, base + n)).
struct DeblendWs {
    int32_t *base, *nobj, *npx, *offs, *counters;
    int32_t* map;
    int32_t *pidx, *par, *nidA, *nidB, *core, *asg, *rootA, *rootB, *nobA, *nobB, *nsig, *tot, *sgc, *dec;
    float* f;
    double *fluxA, *fluxB, *o2, *o3, *o4, *o5;
};

struct DeblendJob {
    const float* sub;
    int64_t pitch;
    const int32_t* labels;  // pitch W
    int64_t W, H;
    const int32_t* n_src_dev;
    int32_t max_src;
    const int32_t *xmin, *xmax, *ymin, *ymax, *area;
    int32_t nthresh;
    double mincont;
    int32_t* out;        // [W*H] pitch W
    int32_t* n_out_dev;  // [1]
    DeblendWs ws;
};

// detection: mode 0 = threshold a given sub frame, 1 = given bit mask,
// 2 = fused with interpolation + subtraction of the raw frame
struct DetectArgs {
    int mode;
    int64_t W, H;
    const void* img;
    int dtype;
    int64_t pitch;
    const float* bias_map;
    float bias;
    const float* inv_flat;
    const float* mesh_bkg;
    float* sub;
    int64_t sub_pitch;
    const float* mesh_rms;
    int nx, ny, mesh_w, mesh_h;
    float k, thresh_abs;
    int min_area;
    int filter;  // 1: threshold the 3 x 3 pyramid-smoothed sub
    const uint32_t* mask_in;
    int32_t* labels;
    int32_t* n_src_dev;
    int32_t max_src;
    ipp_src_stats stats;
    void* ws;
    int interp;                 // IPP_INTERP_KEYS or IPP_INTERP_SPLINE
    const float4* bnodes;       // spline node tables of the mesh bkg and rms (interp = spline)
    const float4* rnodes;
};

struct FitJob {
    const float* stamps;
    int64_t N;               // stamps (with n_dev: the capacity)
    const int32_t* n_dev;    // nullable: the stamp count in device memory, min(*n_dev, N) are fitted
    int S;
    const float* weights;
    const float* init;
    int model;
    float beta;
    int max_iter;
    float lambda0;
    float* params;
    float* chi2;
    int32_t* iters;
    int32_t* flags;
};

}  // namespace ipp

// ---- the batched form: one launch per stage over a device table of frames ----
// A stage's table holds one job per frame and bs[nf + 1], the first virtual
// block of each frame; blocks find their frame by binary search (frame_of).
namespace ipp {
struct MeshFilterJob {
    const float* raw_bkg;
    const float* raw_rms;
    float* fill_bkg;
    float* fill_rms;
    int nx, ny, fw, fh;
    float* out_bkg;
    float* out_rms;
    int32_t* status_dev;
};

// host staging of a batch's device table (16-byte aligned entries)
struct HostBlob {
    unsigned char* h = nullptr;
    size_t used = 0, cap = 0;
    size_t put(const void* p, size_t bytes) {
        used = (used + 15) & ~(size_t)15;
        if (used + bytes > cap) { used = cap + 1; return 0; }   // overflow: the caller checks ok()
        memcpy(h + used, p, bytes);
        const size_t o = used;
        used += bytes;
        return o;
    }
    bool ok() const { return used <= cap; }
};

struct StageRef {
    size_t jobs = 0, bs = 0;   // offsets of the job array and of bs[] in the table
    int total = 0;             // virtual blocks over all frames
};

struct BgMultiPlan { StageRef stats, fill, median; int nf = 0; };
struct DetMultiPlan {
    StageRef zero, thresh, filt, tile, tile_full, unions, resolve, count, scan, emit, fin;
    int nf = 0;
    bool poly = true, filter = false;
    size_t scan_smem = 0;
};
struct PhotMultiPlan { StageRef cen, ap; int nf = 0; size_t ap_smem = 0; };
}  // namespace ipp

template <class T>
ipp::StageRef ipp_put_stage(ipp::HostBlob& hb, const T* jobs, const int* nblk, int nf) {
    ipp::StageRef r;
    r.jobs = hb.put(jobs, sizeof(T) * (size_t)nf);
    int bs[1025];
    bs[0] = 0;
    for (int f = 0; f < nf && f < 1024; f++) bs[f + 1] = bs[f] + nblk[f];
    r.bs = hb.put(bs, sizeof(int) * (size_t)(nf + 1));
    r.total = bs[nf];
    return r;
}

int ipp_extract_jobs(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch, const ipp_calib* cal,
                     const ipp_bg_params* bp, const ipp_det_params* dp, const ipp_cen_params* cp,
                     const ipp_phot_params* pp, int32_t max_src, const ipp_catalog_out* out, void* ws,
                     size_t ws_bytes, ipp::MeshJob* M, ipp::MeshFilterJob* F, ipp::DetectArgs* A, ipp::CenJob* C,
                     ipp::PhotJob* P);
int ipp_bg_multi_pack(const ipp::MeshJob* J, const ipp::MeshFilterJob* F, int nf, ipp::HostBlob& hb,
                      ipp::BgMultiPlan* p);
int ipp_bg_multi_launch(const ipp::BgMultiPlan& p, const unsigned char* dtab, cudaStream_t s);
int ipp_detect_multi_pack(const ipp::DetectArgs* A, int nf, ipp::HostBlob& hb, ipp::DetMultiPlan* p);
int ipp_detect_multi_launch(const ipp::DetMultiPlan& p, const unsigned char* dtab, cudaStream_t s);
int ipp_phot_multi_pack(const ipp::CenJob* C, const ipp::PhotJob* P, int nf, ipp::HostBlob& hb,
                        ipp::PhotMultiPlan* p);
int ipp_phot_multi_launch(const ipp::PhotMultiPlan& p, const unsigned char* dtab, cudaStream_t s);

int ipp_launch_mesh_stats(const ipp::MeshJob& J, cudaStream_t s);
size_t ipp_spline_ws_bytes(int nx, int ny);
int ipp_launch_bg_subtract_spline(const ipp::SubJob& J, void* ws, cudaStream_t s);
int ipp_launch_spline_nodes(const float* mesh, int nx, int ny, void* ws, cudaStream_t s);
size_t ipp_subfit_ws_bytes(int max_c, int nreg, int hw, int fh, int nk, const int32_t* deg, int sord, int bord);
size_t ipp_subfit_smem(int hw, int fh, int nk, const int32_t* deg, int sord, int bord);
int ipp_launch_sub_stamps(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int nsx, int nsy,
                          int hw, int fh, double nsig, int32_t* cx, int32_t* cy, int32_t* n_dev, void* ws,
                          cudaStream_t s);
int ipp_launch_sub_normal(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, const int32_t* cx,
                          const int32_t* cy, const int32_t* n_dev, int max_c, int nreg, int hw, int fh, int nk,
                          const double* sig, const int32_t* deg, int sord, int bord, double* AtA, double* Atb,
                          void* ws, cudaStream_t s);
int ipp_launch_sub_solve(double* AtA, double* Atb, int np, double* coef64, float* coef, int32_t* status,
                         cudaStream_t s);
int ipp_launch_sub_fit(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int nsx, int nsy,
                       double nsig, int hw, int fh, int nk, const double* sig, const int32_t* deg, int sord, int bord,
                       double* coef64, float* coef, int32_t* cx_out, int32_t* cy_out, int32_t* n_out,
                       int32_t* status, void* ws, cudaStream_t s);
size_t ipp_clean_ws_bytes(int32_t max_obj);
int ipp_launch_clean(const float* sub, int64_t pitch, const int32_t* labels, int64_t W, int64_t H,
                     const int32_t* n_dev, int32_t max_obj, const float* thr_map, const float* mesh_rms, int nx,
                     int ny, float mesh_w, float mesh_h, float k, float thresh_abs, float beta, int32_t* out,
                     int32_t* n_out, void* ws, cudaStream_t s);
int ipp_launch_mesh_filter(const float* raw_bkg, const float* raw_rms, float* fill_bkg, float* fill_rms,
                           int nx, int ny, int fw, int fh, float* out_bkg, float* out_rms,
                           int32_t* status_dev, cudaStream_t s);
int ipp_launch_bg_subtract(const ipp::SubJob& J, cudaStream_t s);
size_t ipp_ccl_workspace_size(int64_t W, int64_t H);
int ipp_launch_detect(const ipp::DetectArgs& A, cudaStream_t s);
int ipp_launch_centroid(const ipp::CenJob& J, cudaStream_t s);
int ipp_launch_stamp_cut(const float* sub, int64_t W, int64_t H, int64_t pitch, const int32_t* n_src_dev,
                         int32_t max_src, const float* x, const float* y, int S, float* stamps, float* weights,
                         int32_t* origin, int32_t* flags, cudaStream_t s);
int ipp_launch_aperture(const ipp::PhotJob& J, cudaStream_t s);
int ipp_launch_auto_phot(const ipp::AutoJob& J, cudaStream_t s);
int ipp_launch_deblend(const ipp::DeblendJob& J, cudaStream_t s);
size_t ipp_deblend_ws_carve(int64_t W, int64_t H, int32_t max_src, void* ws, ipp::DeblendWs* out);
int ipp_launch_psf_fit(const ipp::FitJob& J, cudaStream_t s);
int ipp_launch_gray(const float* img, int64_t W, int64_t H, int64_t pitch, int kind, float lo, float hi, float a,
                    float* out, int64_t opitch, cudaStream_t s);
size_t ipp_equalize_ws_bytes(int nbins);
size_t ipp_sub_ws_bytes(int nb, int hw);
int ipp_launch_sub_apply(const float* I, const float* R, int64_t W, int64_t H, int64_t pitch, int hw, int nk,
                         const float* sig, const int* deg, int nb, const float* cs, int sord, const float* cb,
                         int bord, float* D, int64_t opitch, void* ws, cudaStream_t s);
int ipp_launch_zscale(const float* img, int64_t W, int64_t H, int64_t pitch, int ns, double contrast, double krej,
                      int max_iter, double* z, int32_t* counts, cudaStream_t s);
int ipp_launch_wcs_map(const ipp_wcs& src, const ipp_wcs& tgt, int64_t nx, int64_t ny, int step, double* xo,
                       double* yo, cudaStream_t s);
size_t ipp_affine_ws_bytes();
int ipp_launch_affine_fit(const double* x, const double* y, const double* xt, const double* yt, int64_t n,
                          int64_t grid_nx, int step, double* M, int32_t* status, void* ws, cudaStream_t s);
int ipp_launch_reproject(const float* src, int64_t W, int64_t H, int64_t pitch, const double* Minv, int64_t Wo,
                         int64_t Ho, float fill, float* out, int64_t opitch, cudaStream_t s);
int ipp_launch_equalize(const float* img, int64_t W, int64_t H, int64_t pitch, int nbins, float* out,
                        int64_t opitch, void* ws, cudaStream_t s);
int ipp_launch_psf_fwd(const float* params, int64_t N, int S, int model, float beta, float* model_out, cudaStream_t s);
int ipp_launch_psf_adj(const float* params, int64_t N, int S, int model, float beta, const float* grad_model,
                       float* grad_params, cudaStream_t s);
