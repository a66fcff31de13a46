// Host check of pw::dadd_int (csrc/pw_dadd.cuh): wherever it accepts a pair
// of operands, its result must equal the host's IEEE 754 binary64 addition
// (round to nearest even) bit for bit. Operand pairs come from a seeded
// 64-bit generator (splitmix64) in families that reach every branch: random
// normal bit patterns, nearby magnitudes of either sign (cancellation),
// exponent gaps around the alignment limits (31..33, 52..56, 62..66), exact
// ties, sums that carry into a new binade, and operands near the ends of the
// normal range. Prints "cases N accepted A bad B".
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pw_dadd.cuh"

static uint64_t state = 0x2107135000000001ull;

static uint64_t next_u64() {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double from_bits(uint64_t b) {
    double x;
    memcpy(&x, &b, 8);
    return x;
}

static uint64_t bits(double x) {
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

// sign s, biased exponent e, fraction f (52 bits)
static double make(uint64_t s, uint64_t e, uint64_t f) {
    return from_bits((s << 63) | ((e & 0x7FFull) << 52) | (f & 0xFFFFFFFFFFFFFull));
}

static long long cases = 0, accepted = 0, bad = 0;

static void check(double x, double y) {
    ++cases;
    double r;
    if (!pw::dadd_int(x, y, &r)) return;
    ++accepted;
    volatile double want = x + y;
    if (bits(r) != bits(want)) {
        if (bad < 10)
            printf("mismatch: %a + %a: got %a want %a\n", x, y, r, (double)want);
        ++bad;
    }
}

int main() {
    const int n = 400000;
    for (int q = 0; q < n; ++q) {
        const uint64_t a = next_u64(), b = next_u64(), c = next_u64();
        // 1: random normal operands, exponents anywhere
        check(make(a >> 63, 1 + (a >> 40) % 2046, b), make(b >> 63, 1 + (b >> 40) % 2046, c));
        // 2: magnitudes within a few binades, either sign
        const uint64_t e = 900 + (a >> 20) % 200;
        check(make(a >> 63, e, b), make(c >> 63, e - 3 + (c >> 20) % 7, a));
        // 3: near-cancellation: same exponent, fractions sharing high bits
        const uint64_t keep = 1 + (c >> 10) % 52;
        const uint64_t fb = (b & ~((1ull << keep) - 1)) | (c & ((1ull << keep) - 1));
        check(make(0, e, b), make(1, e, fb));
        check(make(0, e, b), make(1, e - 1, fb));
        // 4: exponent gaps at the alignment limits
        static const int gaps[] = {31, 32, 33, 52, 53, 54, 55, 56, 62, 63, 64, 65, 66};
        const int g = gaps[(a >> 5) % 13];
        check(make(b >> 63, e, a), make(c >> 63, e - g, b));
        // 5: ties: y holds only the bit just below x's last place, or that
        // bit plus a far lower one
        const double x = make(0, e, a);
        check(x, make(b >> 63, e - 53, 0));
        check(x, make(b >> 63, e - 53, c & 0xFull));
        check(x, make(0, e - 53, 1ull << 51));
        // 6: sums that carry into the next binade (fractions near all ones)
        check(make(0, e, 0xFFFFFFFFFFFFFull - (a & 0xFF)), make(0, e - (b % 4), c));
        // 7: near the ends of the normal range (results there fall back)
        check(make(a >> 63, 2046 - (b % 3), c), make(a >> 63, 2046 - (c % 3), b));
        check(make(0, 1 + (b % 3), c), make(1, 1 + (c % 3), b));
        // 8: operands the fast path refuses (zeros, subnormals, infinities, NaN)
        check(make(0, 0, a), make(0, e, b));
        check(0.0, make(1, e, b));
        check(make(0, 0x7FF, 0), make(0, e, b));
        check(make(0, 0x7FF, 1), make(0, e, b));
    }
    printf("cases %lld accepted %lld bad %lld\n", cases, accepted, bad);
    return bad == 0 ? 0 : 1;
}
