// Reads lines "a b c d" of 16-digit hex encodings of doubles from stdin and
// prints the hex encoding of sum4::sum4_rn(a, b, c, d) per line (host build of
// the device header, for the correctly rounded reference in test_sum4.py).
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
        const double r = sum4::sum4_rn(x[0], x[1], x[2], x[3]);
        unsigned long long o;
        std::memcpy(&o, &r, 8);
        std::printf("%016llx\n", o);
    }
    return 0;
}
