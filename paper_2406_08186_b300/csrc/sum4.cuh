// The sum of four doubles rounded once (round to nearest, ties to even),
// computed with integer operations on the encodings when that is exact: the
// complex128 Grover coin sums each vertex's four amplitudes, and on this GPU
// the FP64 unit (about 2 operations per clock per SM) bounds that kernel, so
// the three additions move to the integer units.
//
// Method (IEEE 754 binary64): with E the largest exponent field among the
// nonzero addends, every addend x_i = (-1)^s_i M_i 2^(e_i - 1075) (M_i the
// 53-bit significand) is placed as a signed 64-bit integer M_i 2^(8 - (E -
// e_i)), i.e. on a grid of 2^(E - 1083); when no addend sits more than 8
// binades below the largest, none loses a bit, the integer sum is the exact
// sum, and rounding it to 53 significant bits gives the correctly rounded
// result.  Other cases (an addend more than 8 binades smaller, subnormal,
// infinite or NaN addends, a result outside the normal range) take the
// sequential double additions ((x0 + x1) + x2) + x3 instead.  The choice
// depends on the inputs only, so every path that uses this sum agrees bit for
// bit.
//
// The 64-bit values are handled as two 32-bit halves with funnel shifts and
// 32-bit leading-zero counts: measured on this GPU, variable 64-bit shifts and
// 64-bit leading-zero counts issue on the FP64 pipe, which would defeat the
// purpose.  The header compiles as plain C++ for the host check.
#pragma once

#include <cstdint>

#include "fpconv.cuh"

namespace sum4 {

// (hi:lo) << k and (hi:lo) >> k for 0 <= k <= 31, halves only
HW_HD void shl64(uint32_t &hi, uint32_t &lo, int k)
{
#if defined(__CUDA_ARCH__)
    hi = __funnelshift_l(lo, hi, k);
#else
    hi = k ? (hi << k) | (lo >> (32 - k)) : hi;
#endif
    lo = lo << k;
}

HW_HD void shr64(uint32_t &hi, uint32_t &lo, int k)
{
#if defined(__CUDA_ARCH__)
    lo = __funnelshift_r(lo, hi, k);
#else
    lo = k ? (lo >> k) | (hi << (32 - k)) : lo;
#endif
    hi = hi >> k;
}

// (hi:lo) << k for 0 <= k <= 63
HW_HD void shl64_wide(uint32_t &hi, uint32_t &lo, int k)
{
    if (k >= 32) {
        hi = lo << (k - 32);
        lo = 0;
    } else {
        shl64(hi, lo, k);
    }
}

HW_HD int clz32(uint32_t v)
{
#if defined(__CUDA_ARCH__)
    return __clz(static_cast<int>(v));
#else
    return v ? __builtin_clz(v) : 32;
#endif
}

HW_HD uint64_t join(uint32_t hi, uint32_t lo) { return (static_cast<uint64_t>(hi) << 32) | lo; }

// the sequential sum, kept out of line so that the compiler does not compute
// it (on the FP64 unit) alongside the integer path on every call
#if defined(__CUDACC__)
static __device__ __noinline__ double sum4_seq_dev(double x0, double x1, double x2, double x3)
{
    return ((x0 + x1) + x2) + x3;
}
#endif
HW_HD double sum4_seq(double x0, double x1, double x2, double x3)
{
#if defined(__CUDA_ARCH__)
    return sum4_seq_dev(x0, x1, x2, x3);
#else
    return ((x0 + x1) + x2) + x3;
#endif
}

HW_HD double sum4_rn(double x0, double x1, double x2, double x3)
{
    const double xs[4] = {x0, x1, x2, x3};
    uint32_t hi[4], lo[4];
    int e[4];
    int E = 0;
    bool special = false, allzero = true, allneg = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t u = fpconv::bits64(xs[i]);
        hi[i] = static_cast<uint32_t>(u >> 32);
        lo[i] = static_cast<uint32_t>(u);
        e[i] = static_cast<int>((hi[i] >> 20) & 0x7ff);
        const bool zero = ((hi[i] & 0x7FFFFFFFu) | lo[i]) == 0;
        special = special || e[i] == 0x7ff || (e[i] == 0 && !zero);   // inf / NaN / subnormal
        allzero = allzero && zero;
        allneg = allneg && (hi[i] >> 31);
        E = (e[i] > E) ? e[i] : E;
    }
    if (allzero) return fpconv::from_bits64(allneg ? 0x8000000000000000ull : 0ull);   // IEEE sum of zeros
    // signed 64-bit accumulator as two halves
    uint32_t th = 0, tl = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (e[i] == 0) continue;   // a zero adds nothing
        const int s = E - e[i];
        special = special || s > 8;
        uint32_t mh = (hi[i] & 0xFFFFFu) | 0x100000u, ml = lo[i];   // 53-bit significand
        shl64(mh, ml, (8 - s) & 31);
        if (hi[i] >> 31) {   // two's complement of the addend
            ml = ~ml;
            mh = ~mh;
            const uint32_t c = (++ml == 0) ? 1u : 0u;
            mh += c;
        }
        const uint32_t nl = tl + ml;
        th = th + mh + ((nl < tl) ? 1u : 0u);
        tl = nl;
    }
    if (!special) {
        if ((th | tl) == 0) return 0.0;   // exact cancellation: +0 when rounding to nearest
        const bool neg = (th >> 31) != 0;
        uint64_t sign = 0;
        if (neg) {   // magnitude
            tl = ~tl;
            th = ~th;
            const uint32_t c = (++tl == 0) ? 1u : 0u;
            th += c;
            sign = 0x8000000000000000ull;
        }
        // value = (th:tl) 2^(E - 1083); keep 53 significant bits
        const int lz = th ? clz32(th) : 32 + clz32(tl);
        const int shift = 11 - lz;   // bits below the 53 kept ones (negative: room to spare)
        int B = E - 8 + shift;       // biased exponent of the kept significand
        uint32_t rh = th, rl = tl;
        if (shift > 0) {
            // remainder below the kept bits, and half a unit of the last kept bit
            const uint32_t rem = tl & ((1u << shift) - 1u), half = 1u << (shift - 1);
            shr64(rh, rl, shift);
            if (rem > half || (rem == half && (rl & 1u))) {
                const uint32_t c = (++rl == 0) ? 1u : 0u;
                rh += c;
            }
            if (rh >> 21) {   // the rounding carried into a new bit
                shr64(rh, rl, 1);
                ++B;
            }
        } else {
            shl64_wide(rh, rl, -shift);
        }
        if (B >= 1 && B <= 0x7fe)
            return fpconv::from_bits64(sign | (static_cast<uint64_t>(B) << 52) | (join(rh, rl) & 0xFFFFFFFFFFFFFull));
    }
    return sum4_seq(x0, x1, x2, x3);
}

// componentwise sums of the complex terms t(0) .. t(count-1), count >= 1
// (t returns a type with double .x, .y, and is called once per term, in
// order): groups of four consecutive terms summed by sum4_rn (a short last
// group padded with -0, which leaves any sum unchanged), the group sums
// added in order in double.  The next group's terms are fetched before the
// current group is summed, so its loads overlap the integer work; the first
// group's sum starts the total (no addition to 0.0 on the FP64 unit).
template <typename F>
HW_HD void load_group(int j0, int count, F &t, double (&x)[4], double (&y)[4])
{
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        if (j0 + u < count) {
            const auto p = t(j0 + u);
            x[u] = p.x;
            y[u] = p.y;
        } else {
            x[u] = -0.0;
            y[u] = -0.0;
        }
    }
}

template <typename F>
HW_HD void grouped_sum2(int count, F t, double &sx, double &sy)
{
    double cx[4], cy[4], nx[4], ny[4];
    load_group(0, count, t, cx, cy);
    load_group(4, count, t, nx, ny);
    sx = sum4_rn(cx[0], cx[1], cx[2], cx[3]);
    sy = sum4_rn(cy[0], cy[1], cy[2], cy[3]);
    for (int j0 = 4; j0 < count; j0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            cx[u] = nx[u];
            cy[u] = ny[u];
        }
        load_group(j0 + 4, count, t, nx, ny);
        sx += sum4_rn(cx[0], cx[1], cx[2], cx[3]);
        sy += sum4_rn(cy[0], cy[1], cy[2], cy[3]);
    }
}

// group sums of a block of up to four groups: the one group itself, else
// their sum rounded once more by sum4_rn (missing groups are -0)
HW_HD double fold_groups(const double (&g)[4], int ng)
{
    return ng == 1 ? g[0] : sum4_rn(g[0], g[1], g[2], g[3]);
}

// componentwise sums of K terms held in an array (K known at compile time,
// so every index is constant): groups of four summed by sum4_rn as in
// grouped_sum2, then every block of four consecutive group sums (16 terms)
// rounded once more by fold_groups, the block sums added in order in double.
// Up to 16 terms this is one double rounding fewer per group than
// grouped_sum2 and no double addition at all (three fewer FP64 operations
// per component for 16 terms); the kernels that use it are compared with
// each other bit for bit, not with grouped_sum2's.
template <int K, typename V>
HW_HD void grouped_sum2_fixed(const V (&p)[K], double &sx, double &sy)
{
#pragma unroll
    for (int b0 = 0; b0 < K; b0 += 16) {
        double gx[4], gy[4];
        int ng = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j0 = b0 + 4 * q;
            gx[q] = -0.0;
            gy[q] = -0.0;
            if (j0 < K) {
                double x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    x[u] = (j0 + u < K) ? double(p[j0 + u < K ? j0 + u : 0].x) : -0.0;
                    y[u] = (j0 + u < K) ? double(p[j0 + u < K ? j0 + u : 0].y) : -0.0;
                }
                gx[q] = sum4_rn(x[0], x[1], x[2], x[3]);
                gy[q] = sum4_rn(y[0], y[1], y[2], y[3]);
                ng = q + 1;
            }
        }
        const double bx = fold_groups(gx, ng), by = fold_groups(gy, ng);
        sx = (b0 == 0) ? bx : sx + bx;
        sy = (b0 == 0) ? by : sy + by;
    }
}

}  // namespace sum4
