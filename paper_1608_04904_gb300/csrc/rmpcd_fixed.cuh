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

// acc[idx] -= q for 64-bit fixed-point q, aggregated over the lanes that
// subtract into the same address at the same time: their values are summed
// first, exactly (each split into 32-bit parts hi 2^32 + mid 2^16 + lo, summed
// by warp reductions), and one lane of the group does the atomic.  Lanes
// that meet at one address serialise their atomics otherwise, and the
// particles of a warp often share a colloid.  Any |q| >= 2^56 in the active
// lanes: each lane subtracts its own value.
__device__ __forceinline__ void sub_fixed_agg(unsigned long long *acc, int idx, long long q)
{
    const unsigned act = __activemask();
    const long long aq = q < 0 ? -q : q;
    if (__any_sync(act, aq >= (1ll << 56))) {
        atomicAdd(acc + idx, (unsigned long long)(-q));
        return;
    }
    const unsigned grp = __match_any_sync(act, idx);
    const int lo = (int)(q & 0xFFFFll), mid = (int)((q >> 16) & 0xFFFFll), hi = (int)(q >> 32);
    const int slo = __reduce_add_sync(grp, lo);
    const int smid = __reduce_add_sync(grp, mid);
    const int shi = __reduce_add_sync(grp, hi);
    if ((int)(threadIdx.x & 31u) == __ffs(grp) - 1) {
        const long long sum = ((long long)shi << 32) + ((long long)smid << 16) + (long long)slo;
        atomicAdd(acc + idx, (unsigned long long)(-sum));
    }
}

}  // namespace rmpcd
