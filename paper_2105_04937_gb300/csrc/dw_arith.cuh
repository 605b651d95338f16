// Double-word (FP32 pair) arithmetic used by the emulated-FP64 products.
// Error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum (|a| >= |b|
// or a = 0), TwoProduct by FMA; the accurate double-word addition of Joldes,
// Muller and Popescu (ACM TOMS 2017, Alg. 6).  The __f*_rn intrinsics keep
// the compiler from contracting or reordering these operations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mhdc {
namespace dw {

static __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

static __device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (sh, sl) += (a.x + a.y) * (x.x + x.y)
static __device__ __forceinline__ void dw_fma(float &sh, float &sl, float2 a, float2 x)
{
    float ph = __fmul_rn(a.x, x.x);
    float pe = __fmaf_rn(a.x, x.x, -ph);
    pe = __fmaf_rn(a.x, x.y, pe);
    pe = __fmaf_rn(a.y, x.x, pe);
    fast_two_sum(ph, pe, ph, pe);
    float s, t, u, v;
    two_sum(sh, ph, s, t);
    two_sum(sl, pe, u, v);
    t = __fadd_rn(t, u);
    fast_two_sum(s, t, s, t);
    t = __fadd_rn(t, v);
    fast_two_sum(s, t, sh, sl);
}

// An FP32 number as FP64 without the FP64 pipe for normal numbers and zeros.
static __device__ __forceinline__ double f32_to_f64(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFF;
    if (e == 0 || e == 0xFF) {
        if ((b & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)(b & 0x80000000u) << 32);
        return (double)f;  // subnormal, inf, nan: rare
    }
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e - 127 + 1023) << 52) |
                                 ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}


}  // namespace dw
}  // namespace mhdc
