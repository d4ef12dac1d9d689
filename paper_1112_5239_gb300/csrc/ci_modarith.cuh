// ci_modarith.cuh -- modular arithmetic for moduli below 2^32 on the device:
// Barrett reduction (Barrett, CRYPTO 1986) with a per-modulus reciprocal, and
// the Miller-Rabin primality test on top of it.
#pragma once

#include <cstdint>

namespace ci {
namespace dev {

// x mod m for x < 2^64 and 2 <= m < 2^32, with mu = floor((2^64 - 1) / m).
// The quotient estimate q = floor(x mu / 2^64) satisfies
// x/m - 2 < q <= x/m, so x - q m lies in [0, 3m): two conditional
// subtractions give the residue.
struct Barrett32 {
    uint64_t m, mu;
    __device__ __forceinline__ explicit Barrett32(uint64_t mod) : m(mod), mu(~0ull / mod) {}
    __device__ __forceinline__ uint64_t reduce(uint64_t x) const {
        uint64_t r = x - __umul64hi(x, mu) * m;
        if (r >= m) r -= m;
        if (r >= m) r -= m;
        return r;
    }
    __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) const { return reduce(a * b); }  // a, b < 2^32
    // a^e mod m by square-and-multiply (a < 2^32).
    __device__ __forceinline__ uint64_t pow(uint64_t a, uint64_t e) const {
        uint64_t r = reduce(1);
        a = reduce(a);
        while (e) {
            if (e & 1ull) r = mul(r, a);
            a = mul(a, a);
            e >>= 1;
        }
        return r;
    }
};

// Miller-Rabin with bases 2, 7, 61: exact for odd n < 4,759,123,141
// (Jaeschke 1993), so for every odd n in [3, 2^32).  A base that is a multiple
// of n (n = 7, 61) proves nothing and is skipped.
__device__ __forceinline__ bool is_prime_u32(uint64_t n) {
    if (n < 3 || n >= (1ull << 32) || (n & 1ull) == 0) return n == 2;
    const Barrett32 B(n);
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1ull) == 0) {
        d >>= 1;
        ++s;
    }
    const uint32_t bases[3] = {2u, 7u, 61u};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (bases[i] % n == 0) continue;
        uint64_t x = B.pow(bases[i], d);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int r = 1; r < s; ++r) {
            x = B.mul(x, x);
            if (x == n - 1) {
                composite = false;
                break;
            }
        }
        if (composite) return false;
    }
    return true;
}

}  // namespace dev
}  // namespace ci
