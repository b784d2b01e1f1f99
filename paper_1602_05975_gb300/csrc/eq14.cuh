// Section 5, eq. 14 in IEEE single precision for the strength-search
// kernels: one 8x8 block's value from its sums, in a fixed evaluation order
// shared by every kernel that forms eq. 14 tables.
#pragma once

#include <climits>
#include <cstdint>

namespace cdefgb {

// Eq. 14 for one 8x8 block from its sums over its n samples (source sum and
// sum of squares, filtered sum and sum of squares, squared error), in 1/256
// units rounded half away from zero.  Every operation is a correctly
// rounded IEEE single-precision operation, in a fixed order (no
// contraction): the value is exactly reproducible.  n is 64, 32 or 16 (4:2:0
// planes whose sizes are multiples of 4), so the division by n^2 is an
// exact scaling by a power of two.
// int64 -> float rounded to nearest: through the 32-bit conversion when the
// value fits (the same correctly rounded result, off the 64-bit path).
__device__ __forceinline__ float i64_to_float_rn(long long v)
{
    return (v >= INT_MIN && v <= INT_MAX) ? __int2float_rn((int)v) : __ll2float_rn(v);
}

// Round half away from zero to an integer (llroundf), through 32-bit
// conversions below 2^31: rintf rounds ties to even, and a tie is moved away
// from zero with one exact addition.
__device__ __forceinline__ long long round_half_away(float v)
{
    if (fabsf(v) < 2147483520.0f) {   // the largest float below 2^31
        const float r = rintf(v);
        const float q = fabsf(__fsub_rn(v, r)) == 0.5f ? __fadd_rn(v, copysignf(0.5f, v)) : r;
        return (long long)__float2int_rz(q);
    }
    return llroundf(v);
}

__device__ __forceinline__ long long eq14_value(int n, long long s1s, long long s2s, long long s1d,
                                long long s2d, long long sse, int bitdepth)
{
    const float c1 = __fmul_rn(6.25f, (float)(1 << (2 * (bitdepth - 8))));
    const float c2 = __fmul_rn(312.5f, (float)(1 << (4 * (bitdepth - 8))));
    const int nn = n * n;
    const float xs = i64_to_float_rn(n * s2s - s1s * s1s), xd = i64_to_float_rn(n * s2d - s1d * s1d);
    float vs, vd;
    if ((nn & (nn - 1)) == 0) {
        const float inv = __frcp_rn((float)nn);   // exact for a power of two
        vs = __fmul_rn(xs, inv);
        vd = __fmul_rn(xd, inv);
    } else {
        vs = __fdiv_rn(xs, (float)nn);
        vd = __fdiv_rn(xd, (float)nn);
    }
    const float num = __fadd_rn(__fadd_rn(vs, vd), c1);
    const float den = __fmul_rn(2.0f, __fsqrt_rn(__fadd_rn(__fmul_rn(vs, vd), c2)));
    const float d = __fmul_rn(__fdiv_rn(num, den), i64_to_float_rn(sse));
    return round_half_away(__fmul_rn(256.0f, d));
}

}  // namespace cdefgb
