// binary32 <-> binary64 conversions on the integer pipe.
//
// On GB300 the hardware conversions between float and double issue to the FP64 pipe at the
// rate of a DFMA, so in the FP64 residual kernels they cost as much as the arithmetic they
// feed.  These functions build the result from the IEEE 754 binary32 / binary64 encodings
// (sign, biased exponent, significand; IEEE 754-2008 Sec. 3.4) with integer operations only,
// so that no path through them issues an FP64 instruction, not even a predicated-off one:
//   * f2d_ieee is exact (every binary32 value is a binary64 value); subnormal inputs are
//     renormalised, infinities map to infinities, NaNs keep their payload;
//   * d2f_ieee rounds to nearest, ties to even (IEEE 754-2008 Sec. 4.3.1), with gradual
//     underflow to binary32 subnormals and overflow to infinity; NaNs map to quiet NaNs.
// Both agree bit for bit with the hardware conversions on every input except the payload of
// signalling NaNs; emfuse_selftest_fpconv checks that on the device.
#pragma once

#include <stdint.h>

namespace emfuse {

__device__ __forceinline__ double f2d_ieee(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t sgn = u & 0x80000000u;
    const bool zero = (u & 0x7fffffffu) == 0u;
    int ex = int((u >> 23) & 0xffu);  // biased binary32 exponent
    uint32_t man = u & 0x7fffffu;     // significand without the implicit bit
    if (ex == 0 && man != 0) {
        // subnormal: shift the leading one up to the implicit position, lower the exponent
        const int sh = __clz(man) - 8;
        man = (man << sh) & 0x7fffffu;
        ex = 1 - sh;
    }
    // rebias 127 -> 1023; zero stays zero, the all-ones exponent (inf / NaN) stays all ones
    const uint32_t dex = ex == 0xff ? 0x7ffu : (zero ? 0u : uint32_t(ex + 896));
    const uint32_t hi = sgn | (dex << 20) | (man >> 3);
    const uint32_t lo = man << 29;
    return __hiloint2double(int(hi), int(lo));
}

__device__ __forceinline__ float d2f_ieee(double x) {
    const uint32_t hi = uint32_t(__double2hiint(x)), lo = uint32_t(__double2loint(x));
    const uint32_t sgn = hi & 0x80000000u;
    const int e = int((hi >> 20) & 0x7ffu);  // biased binary64 exponent
    const uint32_t mhi = hi & 0xfffffu;      // top 20 of the 52 significand bits
    uint32_t bits;
    if (e >= 897 && e <= 1150) {
        // binary32 normal range before rounding: keep 23 significand bits, round the other 29
        bits = (uint32_t(e - 896) << 23) | (mhi << 3) | (lo >> 29);
        const uint32_t rem = lo & 0x1fffffffu;
        const uint32_t up = (rem > 0x10000000u) || (rem == 0x10000000u && (bits & 1u)) ? 1u : 0u;
        bits += up;  // a carry out of the significand increments the exponent (to inf at the top)
    } else if (e == 0x7ff) {
        const bool nan = (mhi | lo) != 0;
        bits = 0x7f800000u | (nan ? (0x400000u | (mhi << 3) | (lo >> 29)) : 0u);
    } else if (e > 1150) {
        bits = 0x7f800000u;  // beyond the largest binary32 after rounding: infinity
    } else {
        // binary32 subnormal or zero: the value in units of 2^-149 is m * 2^(e - 926) with the
        // full significand m (implicit bit included when e > 0); round the shifted-out part
        const uint64_t m = (uint64_t(mhi | (e > 0 ? 0x100000u : 0u)) << 32) | lo;
        const int sh = e > 0 ? 926 - e : 925;  // >= 30
        if (sh >= 64) {
            bits = 0u;  // below half the smallest subnormal
        } else {
            const uint64_t q = m >> sh;
            const uint64_t rem = m & ((uint64_t(1) << sh) - 1);
            const uint64_t half = uint64_t(1) << (sh - 1);
            bits = uint32_t(q) + ((rem > half || (rem == half && (q & 1))) ? 1u : 0u);
        }
    }
    return __uint_as_float(sgn | bits);
}

// cvt<D>(x): x as type D (float or double), through the functions above when the types differ.
template <class D>
__device__ __forceinline__ D cvt(float x) {
    if constexpr (sizeof(D) == 8) return f2d_ieee(x);
    else return x;
}
template <class D>
__device__ __forceinline__ D cvt(double x) {
    if constexpr (sizeof(D) == 4) return d2f_ieee(x);
    else return x;
}

}  // namespace emfuse
