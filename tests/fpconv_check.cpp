// Checks the integer-only binary64 <-> binary32 conversions of the CUDA
// kernels against the host CPU's IEEE conversions (round to nearest even):
// random encodings over the whole range, values at and around every rounding
// boundary (ties, the subnormal range, the overflow threshold) and specials.
// Prints "ok <count>" or the first mismatch; exits non-zero on a mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>

#include "fpconv.cuh"

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next()
{
    // splitmix64
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static long checked = 0;

static bool same32(float a, float b)
{
    if (std::isnan(a) && std::isnan(b)) return true;
    uint32_t x, y;
    std::memcpy(&x, &a, 4);
    std::memcpy(&y, &b, 4);
    return x == y;
}

static bool same64(double a, double b)
{
    if (std::isnan(a) && std::isnan(b)) return true;
    uint64_t x, y;
    std::memcpy(&x, &a, 8);
    std::memcpy(&y, &b, 8);
    return x == y;
}

static bool check_d(double d)
{
    ++checked;
    const float want = static_cast<float>(d);
    const float got = fpconv::f64_to_f32_rn(d);
    if (!same32(want, got)) {
        std::printf("f64_to_f32_rn(%a): got %a want %a\n", d, double(got), double(want));
        return false;
    }
    return true;
}

static bool check_f(float f)
{
    ++checked;
    const double want = static_cast<double>(f);
    const double got = fpconv::f32_to_f64(f);
    if (!same64(want, got)) {
        std::printf("f32_to_f64(%a): got %a want %a\n", double(f), got, want);
        return false;
    }
    return true;
}

int main()
{
    // random binary64 encodings (all exponents) and random binary32 encodings
    for (int i = 0; i < 4000000; ++i) {
        uint64_t b = next();
        double d;
        std::memcpy(&d, &b, 8);
        if (!check_d(d)) return 1;
        uint32_t c = static_cast<uint32_t>(next());
        float f;
        std::memcpy(&f, &c, 4);
        if (!check_f(f)) return 1;
    }
    // doubles whose exponent lands in or near the binary32 range, with low
    // bits that sit exactly on, just below and just above a rounding tie
    for (int e = -160; e <= 130; ++e) {
        for (int i = 0; i < 4000; ++i) {
            const uint64_t frac = next() & 0xFFFFFFFFFFFFFull;
            const uint64_t tie_bits[4] = {frac, (frac & ~0x1FFFFFFFull) | 0x10000000ull,
                                          (frac & ~0x1FFFFFFFull) | 0x0FFFFFFFull,
                                          (frac & ~0x1FFFFFFFull) | 0x10000001ull};
            for (uint64_t fb : tie_bits) {
                const uint64_t b = (uint64_t(e + 1023) << 52) | fb | ((next() & 1) << 63);
                double d;
                std::memcpy(&d, &b, 8);
                if (!check_d(d)) return 1;
                // subnormal-range ties: the tie bit moves up as the exponent falls
                if (e < -126) {
                    const int drop = 29 + (-126 - e);
                    if (drop < 53) {
                        const uint64_t low = (1ull << drop) - 1;
                        const uint64_t t = (b & ~low) | (1ull << (drop - 1));
                        std::memcpy(&d, &t, 8);
                        if (!check_d(d)) return 1;
                    }
                }
            }
        }
    }
    // specials and edges
    const double specials[] = {0.0, -0.0, std::numeric_limits<double>::infinity(),
                               -std::numeric_limits<double>::infinity(), std::nan(""),
                               std::numeric_limits<double>::denorm_min(), std::numeric_limits<double>::max(),
                               double(std::numeric_limits<float>::max()),
                               std::nextafter(double(std::numeric_limits<float>::max()), 1e300),
                               3.4028235677973366e38, 3.4028235677973362e38,
                               double(std::numeric_limits<float>::denorm_min()),
                               double(std::numeric_limits<float>::denorm_min()) / 2,
                               std::nextafter(double(std::numeric_limits<float>::denorm_min()) / 2, 1.0),
                               double(std::numeric_limits<float>::min()),
                               std::nextafter(double(std::numeric_limits<float>::min()), 0.0), 1.0, -1.0, 0.1};
    for (double d : specials)
        if (!check_d(d) || !check_d(-d)) return 1;
    const float fspecials[] = {0.0f, -0.0f, std::numeric_limits<float>::infinity(), std::nanf(""),
                               std::numeric_limits<float>::denorm_min(), std::numeric_limits<float>::min(),
                               std::numeric_limits<float>::max(), 1.0f, 0.1f};
    for (float f : fspecials)
        if (!check_f(f) || !check_f(-f)) return 1;
    std::printf("ok %ld\n", checked);
    return 0;
}
