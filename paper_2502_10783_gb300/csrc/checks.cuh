// checks.cuh -- argument checks shared by the C-ABI entry points (host code).
#pragma once
#include "jobs.cuh"

#define REQUIRE(cond, ...) \
    do { if (!(cond)) return ipp_set_error(IPP_ERR_INVALID_ARG, __VA_ARGS__); } while (0)

static inline int check_frame(const void* img, int dtype, int64_t W, int64_t H, int64_t pitch, const ipp_calib* cal) {
    REQUIRE(img, "img is NULL");
    REQUIRE(W > 0 && H > 0, "W, H must be positive (got %lld, %lld)", (long long)W, (long long)H);
    REQUIRE(W < (1ll << 31) && H < (1ll << 31), "frame dimensions too large");
    REQUIRE(pitch >= W, "pitch %lld < W %lld", (long long)pitch, (long long)W);
    REQUIRE(dtype == IPP_F32 || dtype == IPP_U16, "unknown dtype %d", dtype);
    if (dtype == IPP_U16) REQUIRE(cal && cal->inv_flat, "IPP_U16 input needs cal->inv_flat");
    return IPP_OK;
}

static inline int check_bg(const ipp_bg_params* p) {
    REQUIRE(p, "bg params NULL");
    REQUIRE(p->mesh_w >= 4 && p->mesh_h >= 4, "mesh size must be >= 4 (got %d x %d)", p->mesh_w, p->mesh_h);
    REQUIRE((int64_t)p->mesh_w * p->mesh_h <= 16384, "mesh area %d > 16384", p->mesh_w * p->mesh_h);
    REQUIRE(p->filter_w >= 1 && p->filter_h >= 1 && (p->filter_w & 1) && (p->filter_h & 1) &&
                p->filter_w <= 7 && p->filter_h <= 7, "filter must be odd and <= 7");
    REQUIRE(p->maxiters >= 1, "maxiters must be >= 1");
    REQUIRE(p->min_valid >= 1, "min_valid must be >= 1");
    REQUIRE(p->estimator >= 0 && p->estimator <= 3, "unknown estimator %d", p->estimator);
    REQUIRE(p->nsigma > 0, "nsigma must be > 0");
    REQUIRE(p->interp == IPP_INTERP_KEYS || p->interp == IPP_INTERP_SPLINE, "unknown interp %d", p->interp);
    return IPP_OK;
}

// calls that interpolate with Keys only
static inline int check_keys_only(const ipp_bg_params* p, const char* what) {
    if (p && p->interp != IPP_INTERP_KEYS)
        return ipp_set_error(IPP_ERR_NOT_SUPPORTED, "%s interpolates with Keys only (interp = spline)", what);
    return IPP_OK;
}
