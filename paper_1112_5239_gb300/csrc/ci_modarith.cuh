// ci_modarith.cuh -- modular arithmetic for moduli below 2^32 on the device:
// Barrett reduction (Barrett, CRYPTO 1986) with a per-modulus reciprocal for
// any modulus, Montgomery multiplication (Montgomery, Math. Comp. 1985) for
// odd moduli, and the Miller-Rabin primality test.  Host-callable as well
// (the device intrinsics have host equivalents), so that the host test of
// tests/native checks these exact functions against 128-bit arithmetic.
#pragma once

#include <cstdint>

namespace ci {
namespace dev {

__host__ __device__ __forceinline__ uint32_t umulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint64_t umulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Leading zeros of a nonzero word.
__host__ __device__ __forceinline__ int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return __builtin_clz(x);
#endif
}

__host__ __device__ __forceinline__ int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

// x mod m for x < 2^64 and 2 <= m < 2^32, with mu = floor((2^64 - 1) / m).
// The quotient estimate q = floor(x mu / 2^64) satisfies
// x/m - 2 < q <= x/m, so x - q m lies in [0, 3m): two conditional
// subtractions give the residue.
struct Barrett32 {
    uint64_t m, mu;
    __host__ __device__ __forceinline__ explicit Barrett32(uint64_t mod) : m(mod), mu(~0ull / mod) {}
    __host__ __device__ __forceinline__ uint64_t reduce(uint64_t x) const {
        uint64_t r = x - umulhi64(x, mu) * m;
        if (r >= m) r -= m;
        if (r >= m) r -= m;
        return r;
    }
    __host__ __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) const { return reduce(a * b); }  // a, b < 2^32
    // a^e mod m by square-and-multiply (a < 2^32).
    __host__ __device__ __forceinline__ uint64_t pow(uint64_t a, uint64_t e) const {
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
// values in Montgomery form a R mod m, REDC(t) = t R^-1 mod m for t < m R.
// REDC: u = (t mod R) m' mod R with m' = -m^-1 mod R; (t + u m) / R < 2m,
// computed without the 65-bit sum: the low halves of t and u m cancel, with a
// carry exactly when t mod R != 0.  Operands are 32-bit words, so a product
// is one 32 x 32 -> 64-bit multiply and REDC one low and one high product.
struct Mont32 {
    uint32_t m;
    uint32_t np;   // -m^-1 mod 2^32
    uint32_t one;  // R mod m, the Montgomery form of 1
    uint32_t r2;   // R^2 mod m
    __host__ __device__ __forceinline__ explicit Mont32(uint32_t mod) : m(mod) {
        uint32_t inv = mod;  // Newton: each step doubles the correct low bits (3 to start)
#pragma unroll
        for (int i = 0; i < 4; ++i) inv *= 2u - mod * inv;
        np = 0u - inv;
        one = (0u - mod) % mod;  // (2^32 - m) mod m = R mod m
        r2 = (uint32_t)((uint64_t)one * one % mod);
    }
    __host__ __device__ __forceinline__ uint32_t redc(uint64_t t) const {  // t < m R
        const uint32_t u = (uint32_t)t * np;
        const uint64_t r = (t >> 32) + umulhi32(u, m) + ((uint32_t)t != 0u ? 1u : 0u);
        return (uint32_t)(r >= m ? r - m : r);
    }
    __host__ __device__ __forceinline__ uint32_t mul(uint32_t a, uint32_t b) const {  // a, b < m
        return redc((uint64_t)a * b);
    }
    // Montgomery form of a < m; of any a, through one 32-bit remainder.
    __host__ __device__ __forceinline__ uint32_t to(uint32_t a) const { return mul(a, r2); }
    __host__ __device__ __forceinline__ uint32_t to_any(uint32_t a) const { return to(a < m ? a : a % m); }
    // Montgomery form of t < m R without a 64-bit remainder: REDC(t) = t R^-1,
    // and two products by R^2 give t R.
    __host__ __device__ __forceinline__ uint32_t to_wide(uint64_t t) const { return mul(mul(redc(t), r2), r2); }
    __host__ __device__ __forceinline__ uint32_t from(uint32_t a) const { return redc(a); }
    // (a^e in Montgomery form) for a in Montgomery form, left to right over
    // 2-bit windows of e: two squarings and one product by a^w (w = 0 takes
    // the form of 1) per window, the same work in every lane whatever its
    // exponent bits, so a warp never runs both sides of a branch.
    __host__ __device__ __forceinline__ uint32_t pow_m(uint32_t a, uint64_t e) const {
        if (e == 0) return one;
        const uint32_t a2 = mul(a, a), a3 = mul(a2, a);
        int i = (63 - clz64(e)) & ~1;  // the window that holds the top bit
        uint32_t w = (uint32_t)(e >> i) & 3u;
        uint32_t r = w == 1u ? a : w == 2u ? a2 : a3;
        for (i -= 2; i >= 0; i -= 2) {
            r = mul(r, r);
            r = mul(r, r);
            w = (uint32_t)(e >> i) & 3u;
            r = mul(r, w == 0u ? one : w == 1u ? a : w == 2u ? a2 : a3);
        }
        return r;
    }
    // (2^e in Montgomery form), left to right: a squaring per bit and, for a
    // set bit, a doubling (the Montgomery form is linear, so 2 x R mod m is
    // the doubled form), taken by a select.
    __host__ __device__ __forceinline__ uint32_t pow2_m(uint32_t e) const {
        uint32_t r = one;
        for (int i = 31 - clz32(e | 1u); i >= 0; --i) {
            r = mul(r, r);
            const uint64_t d = 2ull * r;
            const uint32_t rd = (uint32_t)(d >= m ? d - m : d);
            r = (e >> i) & 1u ? rd : r;
        }
        return r;
    }
};

// Miller-Rabin with bases 2, 7, 61: exact for odd n < 4,759,123,141
// (Jaeschke 1993), so for every odd n in [3, 2^32).  A base that is a multiple
// of n (n = 7, 61) proves nothing and is skipped.
__host__ __device__ __forceinline__ bool is_prime_u32(uint64_t n64) {
    if (n64 < 3 || n64 >= (1ull << 32) || (n64 & 1ull) == 0) return n64 == 2;
    const uint32_t n = (uint32_t)n64;
    const Mont32 M(n);
    const uint32_t one = M.one, minus_one = n - M.one;  // Montgomery forms of 1 and n - 1
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1u) == 0) {
        d >>= 1;
        ++s;
    }
    const uint32_t bases[3] = {2u, 7u, 61u};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const uint32_t b = bases[i] < n ? bases[i] : bases[i] % n;
        if (b == 0) continue;
        uint32_t x = b == 2u ? M.pow2_m(d) : M.pow_m(M.to(b), d);
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
