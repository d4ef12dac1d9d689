// ci_modarith.cuh -- modular arithmetic for moduli below 2^32 on the device:
// Barrett reduction (Barrett, CRYPTO 1986) with a per-modulus reciprocal for
// any modulus, Montgomery multiplication (Montgomery, Math. Comp. 1985) for
// odd moduli, and the Miller-Rabin primality test.
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

// Montgomery arithmetic for an odd modulus 3 <= m < 2^32 with R = 2^32:
// values in Montgomery form a R mod m, REDC(t) = t R^-1 mod m for t < m^2.
// REDC: u = (t mod R) m' mod R with m' = -m^-1 mod R; (t + u m) / R < 2m,
// computed without the 65-bit sum: the low halves of t and u m cancel, with a
// carry exactly when t mod R != 0.
struct Mont32 {
    uint64_t m;
    uint32_t np;   // -m^-1 mod 2^32
    uint64_t r2;   // R^2 mod m
    uint64_t one;  // R mod m, the Montgomery form of 1
    __device__ __forceinline__ explicit Mont32(uint64_t mod) : m(mod) {
        uint32_t inv = (uint32_t)mod;  // Newton: each step doubles the correct low bits (3 to start)
#pragma unroll
        for (int i = 0; i < 4; ++i) inv *= 2u - (uint32_t)mod * inv;
        np = 0u - inv;
        one = (1ull << 32) % mod;
        r2 = one * one % mod;
    }
    __device__ __forceinline__ uint64_t redc(uint64_t t) const {
        const uint32_t u = (uint32_t)t * np;
        uint64_t r = (t >> 32) + (((uint64_t)u * m) >> 32) + ((uint32_t)t != 0u ? 1u : 0u);
        return r >= m ? r - m : r;
    }
    __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) const { return redc(a * b); }  // a, b < m
    __device__ __forceinline__ uint64_t to(uint64_t a) const { return mul(a % m, r2); }
    __device__ __forceinline__ uint64_t from(uint64_t a) const { return redc(a); }
    // (a^e in Montgomery form) for a in Montgomery form.
    __device__ __forceinline__ uint64_t pow_m(uint64_t a, uint64_t e) const {
        uint64_t r = one;
        while (e) {
            if (e & 1ull) r = mul(r, a);
            a = mul(a, a);
            e >>= 1;
        }
        return r;
    }
    __device__ __forceinline__ uint64_t pow(uint64_t a, uint64_t e) const { return from(pow_m(to(a), e)); }
};

// Miller-Rabin with bases 2, 7, 61: exact for odd n < 4,759,123,141
// (Jaeschke 1993), so for every odd n in [3, 2^32).  A base that is a multiple
// of n (n = 7, 61) proves nothing and is skipped.
__device__ __forceinline__ bool is_prime_u32(uint64_t n) {
    if (n < 3 || n >= (1ull << 32) || (n & 1ull) == 0) return n == 2;
    const Mont32 M(n);
    const uint64_t one = M.one, minus_one = n - M.one;  // Montgomery forms of 1 and n - 1
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
        uint64_t x = M.pow_m(M.to(bases[i]), d);
        if (x == one || x == minus_one) continue;
        bool composite = true;
        for (int r = 1; r < s; ++r) {
            x = M.mul(x, x);
            if (x == minus_one) {
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
