// rmpcd_fixed.cuh -- FP32 values to the 2^-40 fixed point of the colloid and
// body force sums, without 64-bit conversions (float -> int64 conversion
// takes several times as long as two 32-bit ones on this GPU).
#pragma once

namespace rmpcd {

// round(f 2^40) to the nearest even integer, exactly as one float -> int64
// conversion would give it, by two 32-bit conversions: with h = f 2^9
// rounded to an integer, f - h 2^-9 is exact (Sterbenz) and at most 2^-10 in
// magnitude, and h 2^31 is even, so the ties round the same way.  Valid for
// |f| < 2^22.
__device__ __forceinline__ long long fx40(float f)
{
    const float h = rintf(f * 0x1p9f);
    const float r = f - h * 0x1p-9f;
    return ((long long)__float2int_rn(h) << 31) + (long long)__float2int_rn(r * 0x1p40f);
}

// The same for any f: the single 64-bit conversion where |f| >= 2^22.
__device__ __forceinline__ long long fx40_any(float f)
{
    return fabsf(f) < 0x1p22f ? fx40(f) : __float2ll_rn(f * 0x1p40f);
}

}  // namespace rmpcd
