// Host check of the library's exact 128-by-64-bit floor division (Knuth's
// Algorithm D with 32-bit digits), which the peel uses for every integer
// threshold: random and edge-case dividends and divisors against the
// compiler's unsigned __int128 division.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include "dupin_common.cuh"
static unsigned long long sm = 88172645463325252ull;
static unsigned long long rnd() { sm ^= sm << 13; sm ^= sm >> 7; sm ^= sm << 17; return sm; }
static long long ref(u128 X, unsigned long long Y) {
    if (X >= ((u128)Y << 63)) return 0x7fffffffffffffffLL;
    return (long long)(X / Y);
}
int main(int argc, char **argv) {
    const long long iters = argc > 1 ? atoll(argv[1]) : 2000000;
    long long bad = 0, n = 0;
    for (long long it = 0; it < iters; it++) {
        unsigned long long y = rnd() >> (rnd() % 64);
        if (y == 0) y = 1;
        u128 x = ((u128)rnd() << 64) | rnd();
        int sh = rnd() % 128;
        x >>= sh;
        if (rnd() % 4 == 0) { u128 q = rnd() >> (rnd() % 64); x = q * (u128)y + (rnd() % 3 == 0 ? 0 : (u128)(rnd() % y)); }
        long long a = floor_div_sat(x, y), b = ref(x, y);
        n++;
        if (a != b) { if (bad < 5) printf("mismatch x_hi=%llx x_lo=%llx y=%llx got %lld want %lld\n", (unsigned long long)(x>>64), (unsigned long long)x, y, a, b); bad++; }
    }
    // edges
    unsigned long long ys[] = {1, 2, 3, 0xffffffffull, 0x100000000ull, 0xffffffffffffffffull, 0x8000000000000000ull, 0x7fffffffffffffffull};
    for (unsigned long long y : ys) for (int k = 0; k < 200; k++) {
        u128 x = ((u128)y << 63) - 1 - (u128)(rnd() % 1000);
        if (floor_div_sat(x, y) != ref(x, y)) bad++;
        x = (u128)rnd() * y; if (floor_div_sat(x, y) != ref(x, y)) bad++;
        n += 2;
    }
    printf("%lld cases, %lld mismatches\n", n, bad);
    return bad != 0;
}
