// Reads lines "a b c d" of 16-digit hex encodings of doubles from stdin and
// prints, per line, the hex encodings of the three forms of the four-term sum
// (sum4_rn, sum4_rn_flat, sum4_rn_cases) of a, b, c, d (host build of the
// device header, for the correctly rounded reference in test_sum4.py).
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "sum4.cuh"

int main()
{
    unsigned long long h[4];
    while (std::scanf("%llx %llx %llx %llx", &h[0], &h[1], &h[2], &h[3]) == 4) {
        double x[4];
        for (int i = 0; i < 4; ++i) std::memcpy(&x[i], &h[i], 8);
        const double r[3] = {sum4::sum4_rn(x[0], x[1], x[2], x[3]), sum4::sum4_rn_flat(x[0], x[1], x[2], x[3]),
                             sum4::sum4_rn_cases(x[0], x[1], x[2], x[3])};
        unsigned long long o[3];
        std::memcpy(o, r, 24);
        std::printf("%016llx %016llx %016llx\n", o[0], o[1], o[2]);
    }
    return 0;
}
