// Conversions between IEEE 754 binary32 and binary64 on the integer units.
//
// On this part the FP64 pipe also executes the FP32 <-> FP64 conversion
// instructions, at the FP64 rate (about 1.7 operations per SM cycle, against
// 64 or more for integer operations).  The kernels whose time is their FP64
// operation count (the FP64 residual, the fold of the correction, the output)
// therefore convert by rearranging the bits instead: the binary64 and binary32
// layouts (sign, biased exponent, fraction; biases 1023 and 127) give both
// directions directly.
//
//   f32_to_f64     exact for every input (zeros, subnormals, infinities; a
//                  NaN keeps its sign and payload, quiet bit included)
//   f64_to_f32_rn  rounded to nearest, ties to even, as IEEE 754 defines
//                  it: overflow to infinity, gradual underflow to binary32
//                  subnormals, a NaN becomes the default quiet NaN
//
// Both are checked bit for bit against the hardware conversions
// (osmodi_probe_convert).
#pragma once
#include <cstdint>

namespace osm {

__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t sign = b & 0x80000000u;
    int e = (int)((b >> 23) & 0xFFu);
    uint32_t m = b & 0x7FFFFFu;
    if (e == 0xFF) {  // infinity, NaN: all-ones exponent, the fraction moved up
        return __hiloint2double((int)(sign | 0x7FF00000u | (m >> 3)), (int)(m << 29));
    }
    if (e == 0) {
        if (m == 0) return __hiloint2double((int)sign, 0);
        // subnormal: m x 2^-149; shift the leading one to the hidden bit
        const int sh = __clz(m) - 8;
        m = (m << sh) & 0x7FFFFFu;
        e = 1 - sh;
    }
    // value 1.m x 2^(e - 127) = 1.m x 2^((e + 896) - 1023)
    return __hiloint2double((int)(sign | ((uint32_t)(e + 896) << 20) | (m >> 3)), (int)(m << 29));
}

__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e == 0x7FF) return __uint_as_float(sign | (((hi & 0xFFFFFu) | lo) ? 0x7FC00000u : 0x7F800000u));
    const int ef = e - 896;  // binary32 biased exponent
    if (ef >= 0xFF) return __uint_as_float(sign | 0x7F800000u);
    if (ef > 0) {
        // keep 23 fraction bits (20 from hi, 3 from lo); 29 bits go
        const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1FFFFFFFu;
        uint32_t mag = ((uint32_t)ef << 23) | mant;
        // a carry out of the fraction raises the exponent (to infinity at the top)
        mag += (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;
        return __uint_as_float(sign | mag);
    }
    // binary32 subnormal or zero: k = round(|x| x 2^149) with the full
    // 53-bit significand M, |x| = M x 2^(e - 1075), so k = M / 2^(926 - e)
    const int s = 926 - e;  // >= 30 here
    if (s > 63) return __uint_as_float(sign);
    const uint64_t M = ((uint64_t)(hi & 0xFFFFFu) << 32 | lo) | (e ? (1ull << 52) : 0ull);
    const uint64_t q = M >> s, r = M & ((1ull << s) - 1ull), half = 1ull << (s - 1);
    const uint64_t k = q + ((r > half || (r == half && (q & 1ull))) ? 1ull : 0ull);
    return __uint_as_float(sign | (uint32_t)k);  // k = 2^23 is the smallest normal: right bits
}

}  // namespace osm
