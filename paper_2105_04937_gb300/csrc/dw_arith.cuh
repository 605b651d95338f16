// Double-word (FP32 pair) arithmetic used by the emulated-FP64 products.
// Error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum, TwoProduct
// by FMA.  The __f*_rn intrinsics keep the compiler from contracting or
// reordering these operations.
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

// One step of an emulated row sum: (sh, sl) += (a.x + a.y) * (x.x + x.y).
// The high product a.x * x.x enters sh by TwoSum (exact); its exact error
// (TwoProduct) and the two cross products form pe; the TwoSum error plus pe
// join sl, and Fast2Sum renormalises the pair.  15 FP32 operations.
// Error of one step, relative to T = sum_j |a_j x_j| of the row (u = 2^-24):
// the product (a.y * x.y dropped, the splits of a and x, two roundings in
// pe) at most 8 u^2 |a x|; the two additions into sl and Fast2Sum (exact
// when |sh| >= |t|, else off by at most u |t|) at most u^2 (5.11 T + 9 |a x|),
// since |sl| stays within 1.02 u T.  A row of k terms therefore ends within
// (5.2 k + 18) u^2 T of its exact sum, including the final rounding of
// sh + sl to FP64 (2^-53 T).  Requires no overflow (|a|, |x| < 2^60, k <= 48)
// and products far above the subnormal range (|a|, |x| >= 2^-45, so that a
// rounding below 2^-126 costs at most 2^-12 u^2 T).
static __device__ __forceinline__ void dw_fma(float &sh, float &sl, float2 a, float2 x)
{
    const float ph = __fmul_rn(a.x, x.x);
    float pe = __fmaf_rn(a.x, x.x, -ph);
    pe = __fmaf_rn(a.x, x.y, pe);
    pe = __fmaf_rn(a.y, x.x, pe);
    float s, e;
    two_sum(sh, ph, s, e);
    const float t = __fadd_rn(sl, __fadd_rn(e, pe));
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
