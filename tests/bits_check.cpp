// Host harness for the integer FP64 -> FP32 round-to-odd and FP32 -> FP64
// conversions of the kernels (gadi_bits.cuh): reads "o <hex double bits>" or
// "f <hex float bits>" lines and prints the FP32 bits of the round-to-odd
// value or the FP64 bits of the float, one per line.
#include <cstdio>

#include "gadi_bits.cuh"

int main()
{
    char kind;
    unsigned long long xb;
    while (std::scanf(" %c %llx", &kind, &xb) == 2) {
        if (kind == 'o') {
            std::printf("%08x\n", (unsigned)gadi::float_bits_round_odd(gadi::double_of(xb)));
        } else {
            float f;
            const unsigned u = (unsigned)xb;
            std::memcpy(&f, &u, sizeof f);
            std::printf("%016llx\n", (unsigned long long)gadi::bits_of(gadi::double_of_float(f)));
        }
    }
    return 0;
}
