// FP64 values as (hi, lo) FP32 pairs and compensated FP32 products: the
// arithmetic of the sweeps that apply FP64 inverses on the FP32 pipe (FP64
// FMAs run at 1/64 of the FP32 rate on this GPU).
#pragma once

#include <cuda_runtime.h>

namespace psr {

// v 2^-shift as a pair (hi, lo) of FP32 with integer operations only: hi is
// v's significand truncated to 24 bits, lo the next 23 bits (truncated), so
// |v 2^-shift - hi - lo| < 2^-46 |v 2^-shift|.  Scaled values below 2^-126
// (hi) or 2^-103 (lo) are dropped, which the caller's choice of shift (the
// largest exponent of the block) makes negligible; FP64 subnormals read as 0;
// Inf and NaN give NaN.
__device__ __forceinline__ float2 split_scaled(double v, int shift) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned h32 = (unsigned)(u >> 32), l32 = (unsigned)u;
    const unsigned sgn = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu);
    const int E = e - 1023 - shift;
    const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    const unsigned mlo = (l32 & 0x1fffffffu) >> 6;
    const int eh = E + 127, el = E - 23 + 127;
    float hi = (e != 0 && eh > 0) ? __uint_as_float(sgn | ((unsigned)eh << 23) | m23) : 0.f;
    float lo = 0.f;
    if (e != 0 && el > 0)
        lo = __fsub_rn(__uint_as_float(sgn | ((unsigned)el << 23) | mlo), __uint_as_float(sgn | ((unsigned)el << 23)));
    if (e == 0x7ff) { hi = __uint_as_float(0x7fc00000u); lo = 0.f; }
    return make_float2(hi, lo);
}

// (s, c) += (bh + bl)(xh + xl): the product bh xh exactly as p + e (FMA), p
// added to s exactly (TwoSum), the cross terms, e and the TwoSum error added
// to c.  Intrinsics keep every operation rounded as written (no contraction).
__device__ __forceinline__ void pair_fma(float& s, float& c, float bh, float bl, float xh, float xl) {
    const float p = __fmul_rn(bh, xh);
    const float e = __fmaf_rn(bh, xh, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    const float q = __fmaf_rn(bh, xl, __fmul_rn(bl, xh));
    c = __fadd_rn(c, __fadd_rn(err, __fadd_rn(e, q)));
    s = t;
}

}  // namespace psr
