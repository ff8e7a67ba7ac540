// common.cuh -- small device helpers shared by the kernels of libipp.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ipp.h"

#define IPP_HD __host__ __device__ __forceinline__
#define IPP_D __device__ __forceinline__

namespace ipp {

constexpr int kWarp = 32;

// Float <-> order-preserving uint32 key (negative values reversed), so that
// integer comparisons and atomics order floats correctly.  NaNs map outside the
// keys of -inf..+inf.
IPP_D uint32_t fkey(float v) {
    uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
IPP_D float fkey_inv(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

IPP_D float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
IPP_D int warp_sum_i(int v) { return __reduce_add_sync(0xffffffffu, v); }

// ---- double-float (unevaluated sum hi + lo of two FP32 numbers) -----------
// Knuth's TwoSum and an FMA-based exact product; used for sums whose error
// must stay far below FP32 rounding without using the (slow) FP64 pipe.
struct df {
    float hi, lo;
};
IPP_D df df_make(float a) { return df{a, 0.0f}; }
IPP_D df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}
IPP_D df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo);
    return two_sum(s.hi, lo);
}
IPP_D df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
// exact square of a float as a double-float
IPP_D df sq_exact(float a) {
    float p = __fmul_rn(a, a);
    float e = __fmaf_rn(a, a, -p);
    return df{p, e};
}
IPP_D double df_to_d(df a) { return (double)a.hi + (double)a.lo; }
IPP_D df warp_sum_df(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, w);
    }
    return v;
}

// double-float arithmetic on the FP32 pipe (~48-bit significands)
IPP_D df df_neg(df a) { return df{-a.hi, -a.lo}; }
IPP_D df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
IPP_D df df_scale(df a, float p2) { return df{a.hi * p2, a.lo * p2}; }  // p2 a power of two
IPP_D df df_mul_f(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return two_sum(p, e);
}
IPP_D df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return two_sum(p, e);
}
IPP_D df df_div(df a, df b) {  // one correction step after the FP32 quotient
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df r = df_sub(a, df_mul_f(b, q1));
    return two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
IPP_D df df_sqrt(df a) {  // one Newton step after the FP32 root
    if (!(a.hi > 0.f)) return df{0.f, 0.f};
    const float r = __fsqrt_rn(a.hi);
    const df d = df_sub(a, sq_exact(r));
    return two_sum(r, __fdiv_rn(d.hi, 2.0f * r));
}
// exact split of an int64 into three pieces of at most 21 bits
IPP_D df df_from_i64(long long i) {
    const float c2 = (float)(int)(i >> 42);
    const float c1 = (float)(int)((i >> 21) & 0x1fffff);
    const float c0 = (float)(int)(i & 0x1fffff);
    return df_add_f(two_sum(c2 * 4398046511104.0f, c1 * 2097152.0f), c0);
}

// A float as two integers, v = c 2^-8 + f 2^-40 exactly for |v| >= 2^-17 (its
// bits below 2^-40 are dropped otherwise): c = rint(v 2^8), and f the residual
// v - c 2^-8 (|.| <= 2^-9, formed exactly in FP32) in units of 2^-40.  Sums of
// such pairs are exact and order-independent; the c sums stay in range while
// the totals stay below ~3.6e16 (values, or values times pixel coordinates).
IPP_D void fx_split(float v, long long out[2]) {
    const long long c = __float2ll_rn(v * 256.0f);
    const float rsd = fabsf(v) < 65536.0f ? v - (float)c * (1.0f / 256.0f) : 0.0f;
    out[0] = c;
    out[1] = __float2ll_rn(rsd * 1099511627776.0f);
}
// the pair's value in double-float
IPP_D df fx_value(const long long* p) {
    const df a = df_from_i64(__ldcg(p)), b = df_from_i64(__ldcg(p + 1));
    return df_add(df_scale(a, 1.0f / 256.0f), df_scale(b, 1.0f / 1099511627776.0f));
}
// add a float's pair to an integer-pair accumulator (global or shared memory)
IPP_D void fx_atomic_add(long long* acc, float v) {
    long long t[2];
    fx_split(v, t);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc), (unsigned long long)t[0]);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + 1), (unsigned long long)t[1]);
}

// Keys (1981) cubic-convolution weights, a = -1/2, for fractional offset s in
// [0, 1): nodes at distances 1 + s, s, 1 - s, 2 - s.
IPP_D void keys_weights(float s, float w[4]) {
    float s2 = s * s, s3 = s2 * s;
    w[0] = -0.5f * s3 + s2 - 0.5f * s;
    w[1] = 1.5f * s3 - 2.5f * s2 + 1.0f;
    w[2] = -1.5f * s3 + 2.0f * s2 + 0.5f * s;
    w[3] = 0.5f * s3 - 0.5f * s2;
}

// Frame of virtual block b in a multi-frame launch: bs[f] is the first block of
// frame f (bs[0] = 0, bs[nf] = the total); frames without blocks are skipped.
IPP_D int frame_of(const int* bs, int nf, int b) {
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(bs + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

IPP_HD int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
IPP_HD int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace ipp

// host-side error recording (api.cu)
int ipp_set_error(int status, const char* fmt, ...);
int ipp_check_launch(const char* what);

// Runs fn() (a host callable returning cudaError_t) once per (slot, device) for
// the current device, under a lock; later calls return at once.  For per-device
// kernel attributes.  Slots 0..15.  A failed fn() is retried on the next call.
int ipp_once_per_device_impl(int slot, cudaError_t (*fn)(void*), void* arg);
template <class F>
int ipp_once_per_device(int slot, F f) {
    return ipp_once_per_device_impl(slot, [](void* a) -> cudaError_t { return (*static_cast<F*>(a))(); }, &f);
}
