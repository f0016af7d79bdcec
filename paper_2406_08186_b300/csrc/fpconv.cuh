// IEEE 754 conversions between binary64 and binary32 done with integer
// operations on the encodings.  On this GPU the FP64 unit, which also
// performs the hardware conversions, runs at a small fraction of the integer
// and FP32 rate, so kernels that convert many values (packing a double
// accumulator into complex64, widening fp32 terms before a double add) use
// these instead.  Both follow the standard's definitions directly:
//   f64_to_f32_rn: roundTiesToEven of the binary64 significand to the binary32
//                  precision at the result's exponent (gradual underflow to
//                  subnormals, overflow to infinity, NaN stays NaN);
//   f32_to_f64:    exact widening (binary32 subnormals are normalised).
// The header compiles as plain C++ too, so the host can check it against the
// host CPU's own conversions.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define HW_HD __host__ __device__ __forceinline__
#else
#define HW_HD inline
#endif

namespace fpconv {

HW_HD uint64_t bits64(double x)
{
#if defined(__CUDA_ARCH__)
    return static_cast<uint64_t>(__double_as_longlong(x));
#else
    uint64_t b;
    std::memcpy(&b, &x, 8);
    return b;
#endif
}

HW_HD double from_bits64(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(static_cast<long long>(b));
#else
    double x;
    std::memcpy(&x, &b, 8);
    return x;
#endif
}

HW_HD uint32_t bits32(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t b;
    std::memcpy(&b, &x, 4);
    return b;
#endif
}

HW_HD float from_bits32(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float x;
    std::memcpy(&x, &b, 4);
    return x;
#endif
}

HW_HD int clz32(uint32_t v)
{
#if defined(__CUDA_ARCH__)
    return __clz(static_cast<int>(v));
#else
    return v ? __builtin_clz(v) : 32;
#endif
}

HW_HD float f64_to_f32_rn_general(double x)
{
    const uint64_t b = bits64(x);
    const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
    const int e = static_cast<int>((b >> 52) & 0x7ff);
    const uint64_t m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7ff)   // infinity, or a quiet NaN keeping the top payload bits
        return from_bits32(sign | 0x7f800000u | (m ? 0x00400000u | static_cast<uint32_t>(m >> 29) : 0u));
    if (e == 0) return from_bits32(sign);   // binary64 subnormals lie far below half the least binary32 one
    const int fe = e - 1023 + 127;          // biased binary32 exponent of the unrounded value
    if (fe >= 255) return from_bits32(sign | 0x7f800000u);
    const uint64_t sig = m | (1ull << 52);  // 53-bit significand, value = sig * 2^(e - 1075)
    // bits of sig dropped: 29 for a normal result; for a subnormal one, as many
    // as put the unit in the last place at 2^-149
    const int shift = (fe >= 1) ? 29 : 30 - fe;
    if (shift > 54) return from_bits32(sign);   // below half of 2^-149
    uint64_t kept = sig >> shift;
    const uint64_t rem = sig & ((1ull << shift) - 1);
    const uint64_t half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (kept & 1))) ++kept;
    // normal: kept carries the implicit bit at 2^23, so adding (fe - 1) << 23
    // gives exponent and fraction, and a carry out of the fraction bumps the
    // exponent (up to infinity); subnormal: kept is the fraction itself, and
    // a carry to 2^23 is the least normal number
    const uint32_t mag = (fe >= 1) ? (static_cast<uint32_t>(fe - 1) << 23) + static_cast<uint32_t>(kept)
                                   : static_cast<uint32_t>(kept);
    return from_bits32(sign | mag);
}

// rounding x to binary32 when the result is a normal number of exponent at
// most 2^126 (so that a carry out of the fraction cannot overflow): add just
// under half a unit of the kept part, plus one when the kept part is odd, and
// truncate; otherwise the general path
HW_HD float f64_to_f32_rn(double x)
{
    const uint64_t b = bits64(x);
    const uint32_t e = static_cast<uint32_t>(b >> 52) & 0x7ffu;
    if (e - 897u < 253u) {
        const uint64_t r = b + 0x0FFFFFFFull + ((b >> 29) & 1u);
        const uint32_t mag = static_cast<uint32_t>(((r >> 29) & 0x3FFFFFFFFull) - (896ull << 23));
        return from_bits32((static_cast<uint32_t>(b >> 32) & 0x80000000u) | mag);
    }
    return f64_to_f32_rn_general(x);
}

HW_HD double f32_to_f64_general(float f)
{
    const uint32_t b = bits32(f);
    const uint64_t sign = static_cast<uint64_t>(b & 0x80000000u) << 32;
    const int e = static_cast<int>((b >> 23) & 0xff);
    const uint32_t m = b & 0x7fffffu;
    if (e == 0xff) return from_bits64(sign | 0x7ff0000000000000ull | (static_cast<uint64_t>(m) << 29));
    if (e == 0) {
        if (m == 0) return from_bits64(sign);
        // subnormal m * 2^-149 with its leading one at bit p
        const int p = 31 - clz32(m);
        const uint64_t frac = (static_cast<uint64_t>(m) << (52 - p)) & 0xFFFFFFFFFFFFFull;
        return from_bits64(sign | (static_cast<uint64_t>(p - 149 + 1023) << 52) | frac);
    }
    return from_bits64(sign | (static_cast<uint64_t>(e - 127 + 1023) << 52) | (static_cast<uint64_t>(m) << 29));
}

// normal binary32 values: move the exponent and fraction fields over and
// rebias; zero, subnormals, infinities and NaN take the general path
HW_HD double f32_to_f64(float f)
{
    const uint32_t b = bits32(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e - 1u < 254u) {
        const uint32_t hi = (b & 0x80000000u) | (((b >> 3) & 0x0FFFFFFFu) + (896u << 20));
        return from_bits64((static_cast<uint64_t>(hi) << 32) | (static_cast<uint64_t>(b) << 29 & 0xFFFFFFFFull));
    }
    return f32_to_f64_general(f);
}

}  // namespace fpconv
