// Host check of the library's modular arithmetic against 128-bit integer
// arithmetic and trial division: the Barrett reciprocal and 62-bit Barrett
// products (ci_device.cuh), and the 32-bit Montgomery products, windowed
// powers and Miller-Rabin test (ci_modarith.cuh).  The same functions run on
// the device; here they are called from host code.  Prints one line per part
// and "ok" when nothing differs; exits 1 otherwise.
#include <cstdint>
#include <cstdio>
#include <random>

#include "ci_device.cuh"
#include "ci_modarith.cuh"

using namespace ci::dev;
typedef unsigned __int128 u128;

static uint64_t ref_mu(uint64_t M) {
    const uint32_t n = 64u - (uint32_t)__builtin_clzll(M);
    const u128 q = ((u128)1 << (2 * n + 1)) / M;
    return n <= 61 ? (uint64_t)(q << (61 - n)) : (uint64_t)q;
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
    u128 r = 1 % m, b = a % m;
    for (; e; e >>= 1) {
        if (e & 1) r = r * b % m;
        b = b * b % m;
    }
    return (uint64_t)r;
}

static bool prime_td(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t d = 2; d * d <= n; ++d)
        if (n % d == 0) return false;
    return true;
}

int main() {
    std::mt19937_64 g(20121123);
    long bad = 0, n = 0;

    // barrett_mu and Barrett62 products: every bit length 2..62, edges and random moduli
    for (uint32_t bits = 2; bits <= 62; ++bits) {
        const uint64_t lo = 1ull << (bits - 1), hi = (1ull << bits) - 1;
        for (int k = 0; k < 4000; ++k) {
            uint64_t M = k == 0 ? lo : k == 1 ? hi : k == 2 ? lo + 1 : lo + g() % (hi - lo + 1);
            if (M < 3) M = 3;
            const uint64_t mu = barrett_mu(M);
            bad += mu != ref_mu(M), ++n;
            if (!(M & 1)) continue;  // the Barrett products serve odd moduli
            Barrett62 B;
            B.set(M, mu);
            for (int j = 0; j < 4; ++j) {
                const uint64_t a = j == 0 ? M - 1 : g() % M, b = j == 1 ? M - 1 : g() % M;
                bad += B.mul(a, b) != (uint64_t)((u128)a * b % M), ++n;
            }
        }
    }
    printf("barrett: %ld of %ld differ\n", bad, n);
    long bad_b = bad;

    // Mont32: products, conversions, windowed powers and powers of 2
    bad = n = 0;
    const uint32_t edge[] = {3u, 5u, 7u, 61u, 63u, 65535u, 2147483647u, 2147483649u, 4294967291u, 4294967295u};
    for (int t = 0; t < 40000; ++t) {
        uint32_t m = t < 10 ? edge[t] : ((uint32_t)g() | 1u);
        if (m < 3) m = 3;
        const Mont32 M(m);
        for (int k = 0; k < 4; ++k) {
            const uint32_t a = (uint32_t)(g() % m), b = (uint32_t)(g() % m);
            const uint32_t am = M.to(a);
            bad += M.from(M.mul(am, M.to(b))) != (uint32_t)((uint64_t)a * b % m), ++n;
            const uint32_t x = (uint32_t)g();
            bad += M.from(M.to_any(x)) != x % m, ++n;
            const uint64_t w = g() % ((uint64_t)m << 32);
            bad += M.from(M.to_wide(w)) != w % m, ++n;
            const uint64_t e = g() >> (g() % 64);
            bad += M.from(M.pow_m(am, e)) != powmod(a, e, m), ++n;
            bad += M.from(M.pow_m(am, k)) != powmod(a, k, m), ++n;
            const uint32_t e32 = (uint32_t)(g() >> (g() % 64));
            bad += M.from(M.pow2_m(e32)) != powmod(2, e32, m), ++n;
        }
        const Barrett32 B(m - 1 > 1 ? m - 1 : 2);
        const uint64_t a = g() % B.m, e = g() >> (g() % 64);
        bad += B.pow(a, e) != powmod(a, e, B.m), ++n;
    }
    printf("montgomery: %ld of %ld differ\n", bad, n);
    long bad_m = bad;

    // Miller-Rabin against trial division
    bad = n = 0;
    for (uint64_t v = 0; v < 100000; ++v) bad += is_prime_u32(v) != prime_td(v), ++n;
    for (int k = 0; k < 3000; ++k) {
        const uint64_t v = (g() & 0xFFFFFFFFull) | 1u;
        bad += is_prime_u32(v) != prime_td(v), ++n;
    }
    // strong pseudoprimes to bases 2 (2047), 2 and 3 (1373653), 2, 3 and 5 (25326001),
    // 2, 3, 5 and 7 (3215031751), and the largest 32-bit prime
    const uint64_t special[] = {2047ull, 1373653ull, 25326001ull, 3215031751ull, 4294967291ull, 4294967295ull};
    for (uint64_t v : special) bad += is_prime_u32(v) != prime_td(v), ++n;
    printf("miller-rabin: %ld of %ld differ\n", bad, n);

    const bool ok = bad_b == 0 && bad_m == 0 && bad == 0;
    printf("%s\n", ok ? "ok" : "FAILED");
    return ok ? 0 : 1;
}
