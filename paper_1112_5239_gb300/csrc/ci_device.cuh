// ci_device.cuh -- device building blocks of the chaotic-iterations PRNG for
// sm_103a: seeding, strategy sources (Algorithm 2 XORshift, 32-bit xor128,
// BBS with Barrett reduction), and the per-warp generation loop that runs
// Algorithm 4/5's mixing and the Eq. (Oplus) update with the lanes' state in
// registers.
//
// Mapping of the paper's thread model onto a warp: one lane per stream; a group
// of C <= 32 consecutive lanes mixes within itself, so a warp holds 32 / C
// whole groups and the exchange of last strategies ("shmem[o1]",
// "shmem[o2]") is two register shuffles.  All lanes of the warp execute each
// shuffle before any lane updates its slot, which is the synchronous reading
// of Algorithm 4's unsynchronised shared-memory read/write: iteration i reads
// the partners' strategies of iteration i - 1.
#pragma once

#include <cuda.h>  // CUtensorMap (TMA descriptor type only)

#include <cstdint>

#include "ci_internal.h"

namespace ci {
namespace dev {

constexpr uint32_t kFull = 0xffffffffu;

// A bounds check of the CI_CHECKED build, written where every lane of the warp
// is converged: if `cond` fails in any lane, lane 0 records (id, index) in the
// state's status word (the first failure wins) and the whole warp returns from
// the enclosing function, so no lane leaves a warp-collective step early and
// the guarded access is never made.  Compiled out otherwise.
#ifdef CI_CHECKED
#define CI_WARP_CHECK(st, cond, id, index)                                                             \
    do {                                                                                              \
        if (__any_sync(0xffffffffu, !(cond))) {                                                       \
            if ((threadIdx.x & 31) == 0 && (st).check)                                                \
                atomicCAS((st).check, 0ull,                                                           \
                          ((unsigned long long)(id) << 56) | ((unsigned long long)(index) & ((1ull << 56) - 1))); \
            return;                                                                                   \
        }                                                                                             \
    } while (0)
#else
#define CI_WARP_CHECK(st, cond, id, index) ((void)0)
#endif

// ------------------------------------------------------------------ seeding
// splitmix64 (Steele, Lea & Flood 2014) used counter-based: draw k of lane l
// is the (l * 2^32 + k + 1)-th output of the generator started at `seed`.
__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t lane_draw(uint64_t seed, uint64_t lane, uint64_t k) {
    return sm64_mix(seed + ((lane << 32) + k + 1ull) * 0x9E3779B97F4A7C15ull);
}

// ------------------------------------------------------- strategy sources
// Each source: load/store of its words for lane l, the pair of combination
// arrays the lane uses, and next() returning the lane's own strategy word.

// 32-bit xor128 (Marsaglia), the xor-like the paper uses for Algorithm 4.
struct SrcXor128 {
    static constexpr bool kHeavy = false;
    uint32_t a, b, c, d;
    __device__ __forceinline__ void load(const DevState &s, uint64_t l) {
        a = s.u32[F_A * s.P + l];
        b = s.u32[F_B * s.P + l];
        c = s.u32[F_C * s.P + l];
        d = s.u32[F_D * s.P + l];
    }
    __device__ __forceinline__ void store(const DevState &s, uint64_t l) const {
        s.u32[F_A * s.P + l] = a;
        s.u32[F_B * s.P + l] = b;
        s.u32[F_C * s.P + l] = c;
        s.u32[F_D * s.P + l] = d;
    }
    __device__ __forceinline__ void arrays(const DevState &, uint64_t, int &a1, int &a2) const {
        a1 = 0;
        a2 = 1;
    }
    __device__ __forceinline__ uint32_t next() {
        const uint32_t s = a ^ (a << 11);
        a = b;
        b = c;
        c = d;
        d = d ^ (d >> 19) ^ (s ^ (s >> 8));
        return d;
    }
};

// Algorithm 2: z ^= z << 13; z ^= z >> 17; z ^= z << 5.
struct SrcXorshift32 {
    static constexpr bool kHeavy = false;
    uint32_t z;
    __device__ __forceinline__ void load(const DevState &s, uint64_t l) { z = s.u32[F_A * s.P + l]; }
    __device__ __forceinline__ void store(const DevState &s, uint64_t l) const { s.u32[F_A * s.P + l] = z; }
    __device__ __forceinline__ void arrays(const DevState &, uint64_t, int &a1, int &a2) const {
        a1 = 0;
        a2 = 1;
    }
    __device__ __forceinline__ uint32_t next() {
        z ^= z << 13;
        z ^= z >> 17;
        z ^= z << 5;
        return z;
    }
};

// xor64, the 64-bit xorshift of the paper's Sec. 7 measurements; the lane's
// strategy word is the low 32 bits of each step.
struct SrcXor64 {
    static constexpr bool kHeavy = false;
    uint64_t z;
    __device__ __forceinline__ void load(const DevState &s, uint64_t l) {
        z = (uint64_t)s.u32[F_A * s.P + l] | ((uint64_t)s.u32[F_B * s.P + l] << 32);
    }
    __device__ __forceinline__ void store(const DevState &s, uint64_t l) const {
        s.u32[F_A * s.P + l] = (uint32_t)z;
        s.u32[F_B * s.P + l] = (uint32_t)(z >> 32);
    }
    __device__ __forceinline__ void arrays(const DevState &, uint64_t, int &a1, int &a2) const {
        a1 = 0;
        a2 = 1;
    }
    __device__ __forceinline__ uint32_t next() {
        z ^= z << 13;
        z ^= z >> 7;
        z ^= z << 17;
        return (uint32_t)z;
    }
};

// ------------------------------------------------ Barrett arithmetic
// a b mod M for M of bit length n, 2 <= n <= 62, and canonical a, b < M, by
// Barrett reduction (Barrett 1986; base-2 form of Menezes et al., Handbook of
// Applied Cryptography, Alg. 14.42) with one bit more precision on both sides
// of the quotient estimate: X = a b, q1 = floor(X / 2^(n-2)),
// mu = floor(2^(2n+1) / M), q = floor(q1 mu / 2^(n+3)).  Each floor then
// costs less than 1/2 (X < 2^(2n), M >= 2^(n-1)), so q >= floor(X / M) - 1
// and r = X - q M lies in [0, 2M): one subtraction gives the canonical
// residue (the textbook estimate needs two).  q1 < 2^(n+2) and
// mu < 2^(n+2) fit 64 bits; the state stores mu << (61 - n) for n <= 61 and
// mu itself for n = 62, where one shift of the product's high half follows.
// Canonical at every step, so the BBS low bits need no conversion (a
// Montgomery square plus the reduction to canonical form measured 22 % slower
// at full occupancy on sm_103a).
__host__ __device__ __forceinline__ uint64_t mul_hi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ uint32_t bit_length64(uint64_t M) {
#ifdef __CUDA_ARCH__
    return 64u - (uint32_t)__clzll((long long)M);
#else
    return 64u - (uint32_t)__builtin_clzll(M);
#endif
}

// The stored reciprocal floor(2^(2n+1) / M), shifted as described above.
// Scaled by 2^(64-n), it is the quotient of the 128-bit 2^(n+65) = hi 2^64 by
// the normalised divisor d = M 2^(64-n) (top bit set, d > hi), found as two
// 32-bit quotient digits, each estimated from the divisor's top half and
// corrected at most twice (Knuth, TAOCP 2, Alg. 4.3.1D, in the two-digit form
// of Warren's Hacker's Delight).  The only other case, M = 2^61 (d = hi),
// and M < 2 take restoring long division.
__host__ __device__ __forceinline__ uint64_t barrett_mu(uint64_t M) {
    const uint32_t n = bit_length64(M);
    uint64_t q;
    const uint64_t d = n >= 2 ? M << (64 - n) : 0, hi = 1ull << (n + 1);
    if (n >= 2 && hi < d) {
        const uint64_t d1 = d >> 32, d0 = d & 0xFFFFFFFFull;
        uint64_t q1 = hi / d1, r = hi - q1 * d1;  // digit 1 of (hi 2^32) / d
        while ((q1 >> 32) || q1 * d0 > (r << 32)) {
            --q1;
            r += d1;
            if (r >> 32) break;
        }
        const uint64_t u = (hi << 32) - q1 * d;  // partial remainder, below d
        uint64_t q0 = u / d1;                    // digit 0 of (u 2^32) / d
        r = u - q0 * d1;
        while ((q0 >> 32) || q0 * d0 > (r << 32)) {
            --q0;
            r += d1;
            if (r >> 32) break;
        }
        q = (q1 << 32) | q0;
    } else {
        uint64_t rem = 1;
        q = 0;
        for (uint32_t i = 0; i < 2 * n + 1; ++i) {
            rem <<= 1;
            q <<= 1;
            if (rem >= M) {
                rem -= M;
                q |= 1;
            }
        }
    }
    return n <= 61 ? q << (61 - n) : q;
}

// 32 x 32 -> 64-bit product, one mul.wide (a single wide multiply-add on the
// FMA-heavy pipe).
__device__ __forceinline__ uint64_t mul_wide32(uint32_t a, uint32_t b) {
    uint64_t r;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(r) : "r"(a), "r"(b));
    return r;
}

struct Barrett62 {
    uint64_t M, mu;      // mu: barrett_mu(M)
    uint32_t s1, s2, t;  // n - 2; 66 - n (at most 63: below n = 4, X < 2^64 and the high half is 0); n == 62
    uint32_t sl;         // n - 34 (limb form, n >= 34)
    uint64_t nM;         // 2^64 - M
    __host__ __device__ __forceinline__ void set(uint64_t mod, uint64_t mu_stored) {
        M = mod;
        mu = mu_stored;
        const uint32_t n = bit_length64(mod);
        s1 = n - 2;
        s2 = 66 - n < 63 ? 66 - n : 63;
        t = n == 62 ? 1u : 0u;
        sl = n >= 34 ? n - 34 : 0u;
        nM = 0ull - mod;
    }
    __host__ __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) const {
        const uint64_t lo = a * b, hi = mul_hi64(a, b);
        const uint64_t q = mul_hi64((hi << s2) | (lo >> s1), mu) >> t;
        const uint64_t r = lo - q * M;
        return r >= M ? r - M : r;
    }
    __host__ __device__ __forceinline__ uint64_t sqr(uint64_t x) const { return mul(x, x); }

    // The same Barrett square on 32-bit limbs, for 34 <= n <= 62 (so the
    // quotient input floor(X / 2^(n-2)) starts in limb 1 or above).
    // Schoolbook products (Knuth, TAOCP 2, Alg. 4.3.1M), each one mul.wide;
    // every carry is an explicit add-with-carry, so the products are the only
    // work on the FMA-heavy pipe, the kernel's limiting pipe.
    //   X = x^2 = x0^2 + 2 x0 x1 2^32 + x1^2 2^64 (x1 < 2^30, so 2 x1 fits);
    //   q1 = X >> (n - 2): two funnel shifts by n - 34 of limbs 1..3;
    //   q = floor(q1 mu / 2^64) >> t: all four partial products, exactly;
    //   r = X - q M mod 2^64 (r < 2M < 2^63), then one conditional
    //   subtraction, decided by the sign of r - M.
    // Equal to mul(x, x) for every canonical x (checked on the host against
    // 128-bit remainders for every n from 34 to 62, and on the GPU).
    __device__ __forceinline__ uint64_t sqr_limb(uint64_t x) const {
        const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
        const uint64_t p00 = mul_wide32(x0, x0), d = mul_wide32(x0, x1 + x1), p11 = mul_wide32(x1, x1);
        uint32_t X1, X2, X3;
        asm("add.cc.u32 %0, %3, %4;\n\t"
            "addc.cc.u32 %1, %5, %6;\n\t"
            "addc.u32 %2, %7, 0;"
            : "=r"(X1), "=r"(X2), "=r"(X3)
            : "r"((uint32_t)(p00 >> 32)), "r"((uint32_t)d), "r"((uint32_t)p11), "r"((uint32_t)(d >> 32)),
              "r"((uint32_t)(p11 >> 32)));
        const uint32_t q0 = __funnelshift_r(X1, X2, sl), q1 = __funnelshift_r(X2, X3, sl);
        const uint32_t m0 = (uint32_t)mu, m1 = (uint32_t)(mu >> 32);
        const uint32_t c00 = __umulhi(q0, m0);
        const uint64_t c01 = mul_wide32(q0, m1), c10 = mul_wide32(q1, m0), c11 = mul_wide32(q1, m1);
        uint32_t w2, w3;  // bits 64..127 of q1 mu
        asm("{\n\t.reg .u32 a, b, c, a2;\n\t"
            "add.cc.u32 a, %2, %3;\n\t"
            "addc.cc.u32 b, %4, %5;\n\t"
            "addc.u32 c, %6, 0;\n\t"
            "add.cc.u32 a2, a, %7;\n\t"
            "addc.cc.u32 %0, b, %8;\n\t"
            "addc.u32 %1, c, 0;\n\t}"
            : "=r"(w2), "=r"(w3)
            : "r"(c00), "r"((uint32_t)c01), "r"((uint32_t)(c01 >> 32)), "r"((uint32_t)c11),
              "r"((uint32_t)(c11 >> 32)), "r"((uint32_t)c10), "r"((uint32_t)(c10 >> 32)));
        const uint32_t qa = __funnelshift_r(w2, w3, t), qb = w3 >> t;
        const uint32_t n0 = (uint32_t)nM, n1 = (uint32_t)(nM >> 32);
        uint64_t r = mul_wide32(qa, n0) + (((uint64_t)X1 << 32) | (uint32_t)p00);
        const uint32_t rh = (uint32_t)(r >> 32) + qa * n1 + qb * n0;
        r = ((uint64_t)rh << 32) | (uint32_t)r;
        const uint64_t dm = r - M;
        return (int32_t)(dm >> 32) < 0 ? r : dm;
    }
};

// Blum Blum Shub strategy source (Algorithm 5 generalised to w = 5 bits per
// squaring for 62-bit moduli): 7 chunks of 5 bits, then two shift steps.
struct SrcBbs {
    static constexpr bool kHeavy = true;
    Barrett62 B;
    uint64_t y;  // BBS state, canonical in [0, M)
    uint32_t sel;
    bool limb;  // every modulus of the warp has 34..62 bits (all seeded ones): the limb-form square;
                // otherwise (33-bit imported moduli) the generic one
    __device__ __forceinline__ void load(const DevState &s, uint64_t l) {
        y = s.u64[G_Y * s.P + l];
        B.set(s.u64[G_M * s.P + l], s.u64[G_MU * s.P + l]);
        sel = s.u32[F_SEL * s.P + l];
        limb = __all_sync(kFull, bit_length64(B.M) >= 34u);
    }
    __device__ __forceinline__ void store(const DevState &s, uint64_t l) const { s.u64[G_Y * s.P + l] = y; }
    __device__ __forceinline__ void arrays(const DevState &, uint64_t, int &a1, int &a2) const {
        a1 = (int)(sel & 7u);
        a2 = 8 + (int)((sel >> 8) & 7u);
    }
    // One BBS output: x <- x^2 mod M (its low bits are the secure ones).
    template <bool kLimb>
    __device__ __forceinline__ uint32_t bbs() {
        y = kLimb ? B.sqr_limb(y) : B.sqr(y);
        return (uint32_t)y;
    }
    template <bool kLimb>
    __device__ __forceinline__ uint32_t assemble() {
        uint32_t t = 0;
#pragma unroll
        for (int c = 0; c < 7; ++c) t = (t << 5) | (bbs<kLimb>() & 31u);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const uint32_t shift = bbs<kLimb>() & 3u;
            t <<= shift;
            t |= bbs<kLimb>() & ((1u << shift) - 1u);  // array_shift = {0, 1, 3, 7}
        }
        return t;
    }
    // `limb` is the same in every lane of the warp, so the branch never diverges.
    __device__ __forceinline__ uint32_t next() { return limb ? assemble<true>() : assemble<false>(); }
};

// Algorithm 5 as printed: eight BBS generators per lane with moduli below
// 2^16, so x^2 fits 32 bits.  x^2 mod M by Barrett reduction with
// mu = floor(2^32 / M): q = mulhi(x^2, mu) is floor(x^2 / M) or one less, so a
// single conditional subtraction gives the canonical residue, taken as the
// unsigned minimum of r and r - M (r - M wraps above r when r < M).  The
// arrays are read from BBS1 and BBS2 when the call starts; at the end of the
// call generator k (state and modulus) is stored in place k + 1.
struct SrcBbs16 {
    static constexpr bool kHeavy = true;
    uint32_t y[8], M[8], mu[8];
    uint32_t sel1, sel2;
    __device__ __forceinline__ void load(const DevState &s, uint64_t l) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            y[k] = s.u32[(F_Y16 + k) * s.P + l];
            M[k] = s.u32[(F_M16 + k) * s.P + l];
            mu[k] = (uint32_t)((1ull << 32) / M[k]);
        }
        sel1 = y[0] & 7u;
        sel2 = y[1] & 7u;
    }
    __device__ __forceinline__ void store(const DevState &s, uint64_t l) const {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            s.u32[(F_Y16 + (k + 1) % 8) * s.P + l] = y[k];
            s.u32[(F_M16 + (k + 1) % 8) * s.P + l] = M[k];
        }
    }
    __device__ __forceinline__ void arrays(const DevState &, uint64_t, int &a1, int &a2) const {
        a1 = (int)sel1;
        a2 = 8 + (int)sel2;
    }
    template <int K>
    __device__ __forceinline__ uint32_t bbs() {  // BBS(K+1)
        const uint32_t a = y[K] * y[K];
        const uint32_t r = a - __umulhi(a, mu[K]) * M[K];
        y[K] = min(r, r - M[K]);
        return y[K];
    }
    __device__ __forceinline__ uint32_t next() {
        // Four low bits of BBS1 .. BBS8 into bits 31-28 .. 3-0: each funnel
        // shift moves t down four bits and brings the next generator's low
        // nibble in at the top, so BBS8 enters first and BBS1 last (the eight
        // generators are independent, so the order of their steps is free).
        uint32_t t = bbs<7>() << 28;
        t = __funnelshift_r(t, bbs<6>(), 4);
        t = __funnelshift_r(t, bbs<5>(), 4);
        t = __funnelshift_r(t, bbs<4>(), 4);
        t = __funnelshift_r(t, bbs<3>(), 4);
        t = __funnelshift_r(t, bbs<2>(), 4);
        t = __funnelshift_r(t, bbs<1>(), 4);
        t = __funnelshift_r(t, bbs<0>(), 4);
        uint32_t shift = bbs<2>() & 3u;
        t <<= shift;
        t |= bbs<0>() & ((1u << shift) - 1u);  // array_shift = {0, 1, 3, 7}
        shift = bbs<6>() & 3u;
        t <<= shift;
        t |= bbs<1>() & ((1u << shift) - 1u);
        return t;
    }
};

// ----------------------------------------------------- generation loop
enum Sink { SINK_V4 = 0, SINK_SCALAR = 1, SINK_QC = 2, SINK_DIGEST = 3 };

// Multiplier of the per-stream output digest D <- D * K + x (mod 2^64),
// an odd 64-bit constant.
constexpr uint64_t kDigestMul = 0xD1342543DE82EF95ull;

// Algorithm 4/5 inner step for one lane: t = own ^ slot[o1] ^ slot[o2];
// slot = t; x ^= t (Eq. Oplus); returns the output x.
template <class Src>
__device__ __forceinline__ uint32_t ci_step(Src &src, uint32_t &x, uint32_t &slot, int p1, int p2) {
    const uint32_t own = src.next();
    const uint32_t s1 = __shfl_sync(kFull, slot, p1);
    const uint32_t s2 = __shfl_sync(kFull, slot, p2);
    const uint32_t t = own ^ s1 ^ s2;
    slot = t;
    x ^= t;
    return x;
}

// Quarter-circle test of one output pair in 24-bit fixed point, as a miss:
// a = o0 >> 8, b = o1 >> 8, and the pair misses iff a^2 + b^2 >= 2^48, i.e.
// iff bit 16 of the high word of the (at most 49-bit) sum is set.  The two
// shifts and the bit test are written as high halves of products by 2^24 and
// 2^16, which keep them on the FMA pipe: the fused loop is otherwise bound by
// the integer ALU pipe (xor-like shifts, mixing XORs).  The multipliers sit in
// constant memory so that they stay multiplies.
static __constant__ uint32_t c_qc_mul[2] = {1u << 24, 1u << 16};
__device__ __forceinline__ uint32_t qc_miss(uint32_t o0, uint32_t o1) {
    const uint32_t a = __umulhi(o0, c_qc_mul[0]), b = __umulhi(o1, c_qc_mul[0]);
    const uint64_t s = (uint64_t)a * a + (uint64_t)b * b;
    return __umulhi((uint32_t)(s >> 32), c_qc_mul[1]);
}

// Launch-shape choices of the written sinks, picked by the autotuner:
// KT = outputs per stream staged per flush (tile depth: 32 or 64, i.e. 128- or
// 256-byte row segments), CACHE = store policy (0: streaming st.global.cs,
// evict-first; 1: default write-back st.global).
template <int KT_, int CACHE_>
struct TileCfg {
    static constexpr int KT = KT_;
    static constexpr int CH = KT_ / 4;  // 16-byte chunks per tile row
    static constexpr int CACHE = CACHE_;
};
using TileDefault = TileCfg<32, 0>;

// Index of word `col` of row `row` in a warp's 32 x KT staging tile: 16-byte
// chunks XOR-swizzled by row so that both the per-lane 16-byte row writes and
// the per-row reads are free of bank conflicts.
template <int KT>
__device__ __forceinline__ int tile_word(int row, int col) {
    return row * KT + ((((col >> 2) ^ (row & 7))) << 2) + (col & 3);
}

template <int CACHE>
__device__ __forceinline__ void store16(uint32_t *p, const uint4 &v) {
    if (CACHE == 0)
        __stcs(reinterpret_cast<uint4 *>(p), v);
    else
        *reinterpret_cast<uint4 *>(p) = v;
}

template <int CACHE>
__device__ __forceinline__ void store4(uint32_t *p, uint32_t v) {
    if (CACHE == 0)
        __stcs(p, v);
    else
        *p = v;
}

// Runs n iterations of warp group g (lanes 32g .. 32g+31) of state `st`.
// Written sinks store stream r's outputs at out[r * ld + col0 + i]
// (r = 32g + lane < st.S only); SINK_QC adds the lane's quarter-circle hits
// to counts[r]; SINK_DIGEST stores the Horner digest of the call's outputs,
// D = sum_i x_i K^(n-1-i) mod 2^64, to counts[r].  `tile` is this warp's
// 32 x TC::KT words of shared memory (written sinks).  SINK_V4 needs out, ld
// and col0 aligned to 4 words.
template <class Src, int SINK, class TC = TileDefault>
__device__ __forceinline__ void warp_task(const DevState &st, uint64_t g, uint64_t n, uint32_t *out,
                                          uint64_t ld, uint64_t col0, uint64_t *counts,
                                          uint4 *tile) {
    constexpr int KT = (SINK == SINK_V4 || SINK == SINK_SCALAR) ? TC::KT : 32;
    constexpr int CH = KT / 4;
    CI_WARP_CHECK(st, g < st.P / 32, CHK_GROUP, g);
    if (SINK == SINK_V4 || SINK == SINK_SCALAR) CI_WARP_CHECK(st, col0 + n <= ld, CHK_COLS, col0 + n);
    if (SINK == SINK_V4) CI_WARP_CHECK(st, (col0 | ld) % 4 == 0, CHK_V4_ALIGN, col0);
    const int lane = threadIdx.x & 31;
    const uint64_t l = g * 32 + lane;
    Src src;
    src.load(st, l);
    uint32_t x = st.u32[F_X * st.P + l];
    uint32_t slot = st.u32[F_SLOT * st.P + l];
    int a1, a2;
    src.arrays(st, l, a1, a2);
    const int p1 = st.table[a1 * 32 + lane];
    const int p2 = st.table[a2 * 32 + lane];
    const uint64_t row0 = g * 32;
    const uint64_t nfull = n - n % KT;
    uint32_t *tw = reinterpret_cast<uint32_t *>(tile);
    uint64_t hits = 0;

    for (uint64_t i0 = 0; i0 < nfull; i0 += KT) {
        if (SINK == SINK_DIGEST) {
#pragma unroll(Src::kHeavy ? 1 : 32)
            for (int k = 0; k < 32; ++k) hits = hits * kDigestMul + ci_step(src, x, slot, p1, p2);
        } else if (SINK == SINK_QC) {
            uint32_t m = 0;
#pragma unroll(Src::kHeavy ? 1 : 16)
            for (int k = 0; k < 16; ++k) {
                const uint32_t o0 = ci_step(src, x, slot, p1, p2);
                const uint32_t o1 = ci_step(src, x, slot, p1, p2);
                m += qc_miss(o0, o1);
            }
            hits += 16u - m;
        } else {
#pragma unroll(Src::kHeavy ? 1 : CH)
            for (int q = 0; q < CH; ++q) {
                uint4 v;
                v.x = ci_step(src, x, slot, p1, p2);
                v.y = ci_step(src, x, slot, p1, p2);
                v.z = ci_step(src, x, slot, p1, p2);
                v.w = ci_step(src, x, slot, p1, p2);
                tile[lane * CH + (q ^ (lane & 7))] = v;
            }
            __syncwarp();
            if (SINK == SINK_V4) {
                constexpr int RPI = 32 / CH;  // tile rows per warp-wide store
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const int r = RPI * k + lane / CH, c = lane % CH;
                    const uint4 v = tile[r * CH + (c ^ (r & 7))];
                    if (row0 + r < st.S) store16<TC::CACHE>(out + (row0 + r) * ld + col0 + i0 + 4 * c, v);
                }
            } else {
#pragma unroll 4
                for (int r = 0; r < 32; ++r) {
#pragma unroll
                    for (int h = 0; h < KT / 32; ++h) {
                        const int c = 32 * h + lane;
                        const uint32_t v = tw[tile_word<KT>(r, c)];
                        if (row0 + r < st.S) store4<TC::CACHE>(out + (row0 + r) * ld + col0 + i0 + c, v);
                    }
                }
            }
            __syncwarp();
        }
    }

    const int rem = (int)(n - nfull);
    if (rem) {
        if (SINK == SINK_DIGEST) {
            for (int k = 0; k < rem; ++k) hits = hits * kDigestMul + ci_step(src, x, slot, p1, p2);
        } else if (SINK == SINK_QC) {
            uint32_t m = 0;
            for (int k = 0; k < rem / 2; ++k) {
                const uint32_t o0 = ci_step(src, x, slot, p1, p2);
                const uint32_t o1 = ci_step(src, x, slot, p1, p2);
                m += qc_miss(o0, o1);
            }
            hits += (uint32_t)(rem / 2) - m;
        } else {
            for (int k = 0; k < rem; ++k) tw[tile_word<KT>(lane, k)] = ci_step(src, x, slot, p1, p2);
            __syncwarp();
            for (int r = 0; r < 32; ++r) {
                for (int c = lane; c < rem; c += 32)
                    if (row0 + r < st.S) out[(row0 + r) * ld + col0 + nfull + c] = tw[tile_word<KT>(r, c)];
            }
            __syncwarp();
        }
    }

    src.store(st, l);
    st.u32[F_X * st.P + l] = x;
    st.u32[F_SLOT * st.P + l] = slot;
    if (SINK == SINK_QC && l < st.S) counts[l] += hits;
    if (SINK == SINK_DIGEST && l < st.S) counts[l] = hits;
}

// ------------------------------------------------ TMA bulk tensor stores
// A warp's 32 x 32 staging tile leaves as ONE cp.async.bulk.tensor store: the
// tile's layout (16-byte chunk c of row r at chunk position c ^ (r % 8), tile
// base 1024-byte aligned) is the TMA 128-byte swizzle, so the tensor map uses
// CU_TENSOR_MAP_SWIZZLE_128B over the output [rows][cols] with a 32 x 32 box.
// The store carries an L2 evict-first policy (outputs are streamed out, as the
// 16-byte path's st.global.cs does).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tma_store_tile(const CUtensorMap *map, const void *smem, int x, int y,
                                               uint64_t policy) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;"
                 :
                 : "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(s), "l"(policy)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until at most one committed store still reads its shared-memory source.
__device__ __forceinline__ void tma_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_read_0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Wait until every committed store has completed.
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Make this thread's ordinary shared-memory writes visible to the TMA unit.
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Written sink through TMA: per 32-iteration tile, the lanes fill one of two
// 4 KB tiles (double buffering: a tile is refilled only after the store issued
// from it two tiles earlier has read it), then lane 0 issues the tile's bulk
// tensor store at (column col0 + i0, row 32 g); rows past the tensor's row
// count (streams >= S) are clipped by the TMA unit.  A ragged tail of fewer
// than 32 iterations leaves through ordinary stores.  `tiles` is 2 x 4 KB,
// 1024-byte aligned.  Requires out 16-byte aligned, ld % 4 == 0, col0 % 4 == 0
// (checked by the host when it builds the tensor map).
template <class Src>
__device__ __forceinline__ void warp_task_tma(const DevState &st, uint64_t g, uint64_t n, const CUtensorMap *map,
                                              uint32_t *out, uint64_t ld, uint64_t col0, uint4 *tiles) {
    CI_WARP_CHECK(st, g < st.P / 32, CHK_GROUP, g);
    CI_WARP_CHECK(st, col0 + n <= ld, CHK_COLS, col0 + n);
    CI_WARP_CHECK(st, col0 % 4 == 0, CHK_TMA_ALIGN, col0);
    const int lane = threadIdx.x & 31;
    const uint64_t l = g * 32 + lane;
    Src src;
    src.load(st, l);
    uint32_t x = st.u32[F_X * st.P + l];
    uint32_t slot = st.u32[F_SLOT * st.P + l];
    int a1, a2;
    src.arrays(st, l, a1, a2);
    const int p1 = st.table[a1 * 32 + lane];
    const int p2 = st.table[a2 * 32 + lane];
    const uint64_t row0 = g * 32;
    const uint64_t nfull = n & ~31ull;
    if (lane == 0) tma_wait_read_0();  // tiles free (stores of the previous task have read them)
    __syncwarp();
    const uint64_t policy = l2_evict_first_policy();
    int k = 0;
    for (uint64_t i0 = 0; i0 < nfull; i0 += 32, ++k) {
        uint4 *tile = tiles + (k & 1) * 256;
        if (k >= 2) {
            if (lane == 0) tma_wait_read_1();
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint4 v;
            v.x = ci_step(src, x, slot, p1, p2);
            v.y = ci_step(src, x, slot, p1, p2);
            v.z = ci_step(src, x, slot, p1, p2);
            v.w = ci_step(src, x, slot, p1, p2);
            tile[lane * 8 + (q ^ (lane & 7))] = v;
        }
        fence_smem_to_async();
        __syncwarp();
        if (lane == 0) tma_store_tile(map, tile, (int)(col0 + i0), (int)row0, policy);
    }
    const int rem = (int)(n - nfull);
    if (rem) {
        if (lane == 0) tma_wait_read_0();
        __syncwarp();
        uint32_t *tw = reinterpret_cast<uint32_t *>(tiles);
        for (int kk = 0; kk < rem; ++kk) tw[tile_word<32>(lane, kk)] = ci_step(src, x, slot, p1, p2);
        __syncwarp();
        for (int r = 0; r < 32; ++r)
            if (lane < rem && row0 + r < st.S) out[(row0 + r) * ld + col0 + nfull + lane] = tw[tile_word<32>(r, lane)];
        __syncwarp();
    }
    src.store(st, l);
    st.u32[F_X * st.P + l] = x;
    st.u32[F_SLOT * st.P + l] = slot;
}

}  // namespace dev
}  // namespace ci
