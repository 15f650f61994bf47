// Division through a precomputed reciprocal (csrc/fastdiv.h) against the
// integer division, on the host: every n below 2^22 and every n in the top
// 2^22 of [0, 2^31) for a set of divisors (mode counts, row lengths, half
// rows), and the multiples of d and their neighbours for every d < 70,000.
// Prints "ok <cases>" or the first failing (n, d).
#include <cstdio>
#include <cstdint>

#include "fastdiv.h"

static bool check(unsigned n, unsigned d, unsigned r, unsigned long long &cases) {
    ++cases;
    if (pp::fdiv(n, d, r) != n / d) {
        std::printf("FAIL %u %u\n", n, d);
        return false;
    }
    return true;
}

int main() {
    const unsigned top = 0x80000000u;
    unsigned long long cases = 0;
    const unsigned ds[] = {1, 2, 3, 7, 9, 17, 33, 65, 129, 200, 256, 257, 400, 512, 1000, 4096, 65535, 1u << 20};
    for (unsigned d : ds) {
        const unsigned r = pp::fdiv_rcp(d);
        for (unsigned n = 0; n < (1u << 22); ++n)
            if (!check(n, d, r, cases)) return 1;
        for (unsigned n = top - (1u << 22); n < top; ++n)
            if (!check(n, d, r, cases)) return 1;
    }
    for (unsigned d = 1; d < 70000; ++d) {
        const unsigned r = pp::fdiv_rcp(d);
        const unsigned step = d < 4096 ? 997u * d : d;   // about 2,000 multiples per d, spread over the range
        for (unsigned long long q = 0; q * d < top; q += (step / d) ? (step / d) : 1) {
            const unsigned m = (unsigned)(q * d);
            if (!check(m, d, r, cases)) return 1;
            if (m > 0 && !check(m - 1, d, r, cases)) return 1;
            if (m + 1 < top && !check(m + 1, d, r, cases)) return 1;
            if (q > 4096 && d >= 4096) q += 2 * 4096;   // thin out the large divisors
        }
        if (!check(top - 1, d, r, cases)) return 1;
    }
    std::printf("ok %llu\n", cases);
    return 0;
}
