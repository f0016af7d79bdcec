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
//
// Three forms compute the same function and return the same bits for every
// input: sum4_rn_cases (one branch per case), sum4_rn (an early return for
// four zeros, a select-only path for the common case, short branches for the
// rest) and sum4_rn_flat (selects throughout).  Which is fastest depends on
// the kernel: measured, the four-arc kernels take sum4_rn and the loops over
// groups of a long vertex take sum4_rn_flat.
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

// The method with one branch per case, the plainest statement of it (host
// checks compare the other two forms with it and with rational arithmetic).
HW_HD double sum4_rn_cases(double x0, double x1, double x2, double x3)
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

// the per-case form out of line (the rare inputs of sum4_rn_flat)
#if defined(__CUDACC__)
static __device__ __noinline__ double sum4_cases_dev(double x0, double x1, double x2, double x3)
{
    return sum4_rn_cases(x0, x1, x2, x3);
}
#endif
HW_HD double sum4_cases_call(double x0, double x1, double x2, double x3)
{
#if defined(__CUDA_ARCH__)
    return sum4_cases_dev(x0, x1, x2, x3);
#else
    return sum4_rn_cases(x0, x1, x2, x3);
#endif
}

HW_HD uint32_t lo32(uint64_t v) { return static_cast<uint32_t>(v); }
HW_HD uint32_t hi32(uint64_t v) { return static_cast<uint32_t>(v >> 32); }

// The same function with a fast path: all four addends zero returns at once
// (a state with real amplitudes has all-zero imaginary sums); otherwise the
// four addends are aligned independently, summed as a tree (the negative ones
// as one's complements plus their count) and rounded with selects only, so a
// warp whose lanes see different signs and rounding cases runs one stream.
// The other cases branch off without recomputing anything: infinite, NaN or
// subnormal addends, a spread of more than 8 binades and a result outside the
// normal range take the sequential sum (out of line); an exact cancellation
// returns +0; a sum that cancelled down to fewer than 54 bits is exact and is
// shifted up instead of rounded.
HW_HD double sum4_rn(double x0, double x1, double x2, double x3)
{
    const double xs[4] = {x0, x1, x2, x3};
    uint32_t hi[4], lo[4];
    int e[4];
    bool nz[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t u = fpconv::bits64(xs[i]);
        hi[i] = hi32(u);
        lo[i] = lo32(u);
        e[i] = static_cast<int>((hi[i] >> 20) & 0x7ff);
        nz[i] = ((hi[i] << 1) | lo[i]) != 0;
    }
    if (!(nz[0] || nz[1] || nz[2] || nz[3])) {
        // a sum of zeros is -0 only when every addend is -0
        const uint32_t allneg = (hi[0] & hi[1] & hi[2] & hi[3]) >> 31;
        return fpconv::from_bits64(static_cast<uint64_t>(allneg) << 63);
    }
    const int E01 = e[0] > e[1] ? e[0] : e[1], E23 = e[2] > e[3] ? e[2] : e[3];
    const int E = E01 > E23 ? E01 : E23;
    // the smallest exponent field among the nonzero addends: infinity or NaN
    // (E = 0x7ff), a subnormal (0) or a spread of more than 8 binades is special
    int em[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) em[i] = nz[i] ? e[i] : 0x7ff;
    const int Em01 = em[0] < em[1] ? em[0] : em[1], Em23 = em[2] < em[3] ? em[2] : em[3];
    const int Em = Em01 < Em23 ? Em01 : Em23;
    const bool special = E == 0x7ff || Em == 0 || E - Em > 8;
    uint32_t nneg = 0;
    uint64_t a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int sft = E - e[i];
        // 53-bit significand (zero for a zero addend) placed at 2^(8 - sft)
        uint32_t mh = (hi[i] & 0xFFFFFu) | (nz[i] ? 0x100000u : 0u), ml = lo[i];
        shl64(mh, ml, (8 - sft) & 31);
        const uint32_t neg = hi[i] >> 31, m = 0u - neg;   // all ones for a negative addend
        nneg += neg;
        a[i] = join(mh ^ m, ml ^ m);                      // -x = ~x + 1: the +1s are nneg
    }
    // signed 64-bit sum on the grid 2^(E - 1083), |sum| < 2^63 (integer adds)
    const uint64_t t = (a[0] + a[1]) + (a[2] + a[3]) + nneg;
    const uint32_t sgn = hi32(t) >> 31;
    const uint64_t mag = (t ^ (0ull - sgn)) + sgn;
    const uint32_t th = hi32(mag), tl = lo32(mag);
    const int lz = th ? clz32(th) : 32 + clz32(tl);
    const int sh = 11 - lz;                           // bits below the kept 53
    // round to nearest even: add half a unit of the last kept bit less one,
    // plus that bit, then drop the sh low bits
    const uint32_t inc = ((1u << ((sh - 1) & 31)) - 1u) + ((tl >> (sh & 31)) & 1u);
    const uint64_t r = mag + inc;
    uint32_t kh = hi32(r), kl = lo32(r);
    shr64(kh, kl, sh & 31);
    uint32_t carry = kh >> 21;                        // the rounding carried to 2^53
    if (special || sh <= 0) {
        if (special) return sum4_seq(x0, x1, x2, x3);
        if (mag == 0) return 0.0;                     // exact cancellation: +0 when rounding to nearest
        // at most 53 significant bits: exact, shifted up to the leading bit
        kh = th;
        kl = tl;
        shl64_wide(kh, kl, -sh);
        carry = 0;
    }
    const int B = E - 8 + sh + static_cast<int>(carry);
    if (B < 1 || B > 0x7fe) return sum4_seq(x0, x1, x2, x3);
    // (B - 1 - carry) 2^52 + kept: the implicit bit (2^52, or 2^53 after a
    // carry) lands in the exponent field
    return fpconv::from_bits64((static_cast<uint64_t>(sgn) << 63) +
                               (static_cast<uint64_t>(static_cast<uint32_t>(B - 1 - static_cast<int>(carry))) << 52) +
                               join(kh, kl));
}

// The same function with every step as a select (no early return for zeros
// either) up to one branch to the per-case form (special inputs, a sum that
// cancelled below 54 bits, a result outside the normal range): used where the terms are
// general complex amplitudes, summed in a loop of groups, so that the code a
// group inlines stays short.
HW_HD double sum4_rn_flat(double x0, double x1, double x2, double x3)
{
    const double xs[4] = {x0, x1, x2, x3};
    uint32_t hi[4], lo[4];
    int e[4];
    bool nz[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint64_t u = fpconv::bits64(xs[i]);
        hi[i] = hi32(u);
        lo[i] = lo32(u);
        e[i] = static_cast<int>((hi[i] >> 20) & 0x7ff);
        nz[i] = ((hi[i] << 1) | lo[i]) != 0;
    }
    const int E01 = e[0] > e[1] ? e[0] : e[1], E23 = e[2] > e[3] ? e[2] : e[3];
    const int E = E01 > E23 ? E01 : E23;
    int em[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) em[i] = nz[i] ? e[i] : 0x7ff;
    const int Em01 = em[0] < em[1] ? em[0] : em[1], Em23 = em[2] < em[3] ? em[2] : em[3];
    const int Em = Em01 < Em23 ? Em01 : Em23;
    const bool special = E == 0x7ff || Em == 0 || E - Em > 8;
    uint32_t nneg = 0;
    uint64_t a[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int sft = E - e[i];
        uint32_t mh = (hi[i] & 0xFFFFFu) | (nz[i] ? 0x100000u : 0u), ml = lo[i];
        shl64(mh, ml, (8 - sft) & 31);
        const uint32_t neg = hi[i] >> 31, m = 0u - neg;
        nneg += neg;
        a[i] = join(mh ^ m, ml ^ m);
    }
    const uint64_t t = (a[0] + a[1]) + (a[2] + a[3]) + nneg;
    const uint32_t sgn = hi32(t) >> 31;
    const uint64_t mag = (t ^ (0ull - sgn)) + sgn;
    const uint32_t th = hi32(mag), tl = lo32(mag);
    const int lz = th ? clz32(th) : 32 + clz32(tl);
    const int sh = 11 - lz;
    // round to nearest even (sh > 0; a sum that cancelled below 54 bits,
    // sh <= 0, is exact and goes to the per-case form)
    const uint32_t inc = ((1u << ((sh - 1) & 31)) - 1u) + ((tl >> (sh & 31)) & 1u);
    const uint64_t r = mag + inc;
    uint32_t kh = hi32(r), kl = lo32(r);
    shr64(kh, kl, sh & 31);
    const uint32_t carry = kh >> 21;
    const int B = E - 8 + sh + static_cast<int>(carry);
    const uint64_t bits = (static_cast<uint64_t>(sgn) << 63) +
                          (static_cast<uint64_t>(static_cast<uint32_t>(B - 1 - static_cast<int>(carry))) << 52) +
                          join(kh, kl);
    const bool allzero = !(nz[0] || nz[1] || nz[2] || nz[3]);
    const bool cancel = mag == 0;
    const bool ok = allzero || (!special && (cancel || (sh > 0 && B >= 1 && B <= 0x7fe)));
    if (!ok) return sum4_cases_call(x0, x1, x2, x3);
    const uint32_t allneg = (hi[0] & hi[1] & hi[2] & hi[3]) >> 31;
    return fpconv::from_bits64(allzero ? (static_cast<uint64_t>(allneg) << 63) : cancel ? 0ull : bits);
}

// componentwise sums of the complex terms t(0) .. t(count-1), count >= 1
// (t returns a type with double .x, .y, and is called once per term, in
// order): groups of four consecutive terms summed by sum4_rn (a short last
// group padded with -0, which leaves any sum unchanged), the group sums
// added in order in double.  The next group's terms are fetched before the
// current group is summed, so its loads overlap the integer work; the first
// group's sum starts the total (no addition to 0.0 on the FP64 unit).  The
// groups take sum4_rn_flat (same results as sum4_rn).
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
    sx = sum4_rn_flat(cx[0], cx[1], cx[2], cx[3]);
    sy = sum4_rn_flat(cy[0], cy[1], cy[2], cy[3]);
    for (int j0 = 4; j0 < count; j0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            cx[u] = nx[u];
            cy[u] = ny[u];
        }
        load_group(j0 + 4, count, t, nx, ny);
        sx += sum4_rn_flat(cx[0], cx[1], cx[2], cx[3]);
        sy += sum4_rn_flat(cy[0], cy[1], cy[2], cy[3]);
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
