// ci_split.cu -- time-parallel generation of long streams by jump-ahead
// (include/ci_prng.h: ci_generate_split).  Not a construct of the paper: it
// cuts one call of n iterations into K segments of `len` iterations that run
// at the same time, with results identical to the sequential call.
//
// Why it is exact.  Per warp, the own words o(i) of the strategy sources do
// not depend on the mixing state, and the mixing is GF(2)-linear on the
// lanes: with s the vector of the 32 lanes' slots and P the 32 x 32 matrix
// whose row l has ones at the partners o1(l), o2(l) (Algorithm 4/5),
//   s(i) = o(i) ^ P s(i-1),   x(i) = x(i-1) ^ s(i)   (Eq. Oplus),
// so a segment started from (s, x) = (0, 0) gives a particular solution, and
// the true one adds P^j s_a to s and x_a ^ (P + ... + P^j) s_a to x.
//
// Steps of one call (all on the caller's stream):
//   1. k_split_setup: segment states k = 0 .. K-1 are copies of the state
//      with the own generator jumped ahead by k len iterations (GF(2) matrix
//      powers for the xor-likes, x <- x^(2^(11 k len) mod lambda(M)) for BBS,
//      each of the eight 16-bit generators by its own squaring count for
//      Algorithm 5 as printed) and (s, x) = (0, 0) for k >= 1;
//   2. written outputs of the BBS sources (62-bit and Algorithm 5 as
//      printed), where generation is the cost, with many warp groups:
//      k_split_run_fix runs every segment from there into its output
//      columns, and as soon as a segment and its predecessor's true end are
//      done, XORs the segment's homogeneous part into its outputs (the
//      mixing step with zero own words: two shuffles per output), which also
//      gives the segment's true end; the fix-ups overlap the other segments'
//      generation;
//   3. the same with few warp groups, where one serial chain of fix-ups per
//      group would outlast the generation: pass 1 (k_split_run) into the
//      output columns, the carry scan of step 4 (true starts only), then
//      k_split_fixup runs all fix-ups at once;
//   4. otherwise (xor-like outputs are cheaper to generate again than to
//      read back, and consumer sinks have no outputs to fix): pass 1
//      (k_split_run) runs segments 0 .. K-2 into a digest sink (only their
//      end states are needed); k_split_carry, one block per warp group,
//      scans the segments: the true start of segment k is its predecessor's
//      particular end plus (Q s_a, x_a ^ S s_a) with Q = P^len,
//      S = P + ... + P^len (a chunked parallel scan over up to 16 warps);
//      pass 2 (k_split_run) runs every segment from its true start, with the
//      own words k_split_setup jumped to, into the sink;
//   5. the last segment's end state becomes the caller's state, and the
//      per-segment quarter-circle counts or digests are combined.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "ci_split.h"
#include "ci_device.cuh"
#include "ci_trace.h"

namespace ci {
namespace {

using namespace dev;

// ------------------------------------------------ xor-like jump tables
// Column form of the GF(2)-linear step A of a xor-like with W 32-bit words:
// T[i][j] = A^(2^i) e_j, so v <- A^(2^i) v is the XOR of the columns j at the
// set bits of v.  Built on the device from the sources' own next().
constexpr int kJumpLevels = 64;
__device__ uint32_t g_jump_xor128[kJumpLevels][128][4];
__device__ uint32_t g_jump_xor64[kJumpLevels][64][2];
__device__ uint32_t g_jump_xs32[kJumpLevels][32][1];

template <int W>
__device__ __forceinline__ void step_words(uint32_t (&v)[W]) {
    if (W == 4) {
        SrcXor128 s;
        s.a = v[0];
        s.b = v[1 % W];
        s.c = v[2 % W];
        s.d = v[3 % W];
        s.next();
        v[0] = s.a;
        v[1 % W] = s.b;
        v[2 % W] = s.c;
        v[3 % W] = s.d;
    } else if (W == 2) {
        SrcXor64 s;
        s.z = (uint64_t)v[0] | ((uint64_t)v[1 % W] << 32);
        s.next();
        v[0] = (uint32_t)s.z;
        v[1 % W] = (uint32_t)(s.z >> 32);
    } else {
        SrcXorshift32 s;
        s.z = v[0];
        s.next();
        v[0] = s.z;
    }
}

// One block of 32 W threads; thread j owns column j at every level.
template <int W>
__global__ void k_build_jump(uint32_t (*T)[32 * W][W]) {
    const int j = threadIdx.x;
    uint32_t v[W];
#pragma unroll
    for (int w = 0; w < W; ++w) v[w] = (w == j / 32) ? (1u << (j % 32)) : 0u;
    step_words<W>(v);
#pragma unroll
    for (int w = 0; w < W; ++w) T[0][j][w] = v[w];
    for (int i = 1; i < kJumpLevels; ++i) {
        __syncthreads();
        uint32_t r[W] = {};
        for (int b = 0; b < 32 * W; ++b)
            if ((T[i - 1][j][b / 32] >> (b % 32)) & 1u)
#pragma unroll
                for (int w = 0; w < W; ++w) r[w] ^= T[i - 1][b][w];
#pragma unroll
        for (int w = 0; w < W; ++w) T[i][j][w] = r[w];
    }
}

template <int W>
__device__ __forceinline__ void jump_words(uint32_t (&v)[W], uint64_t dist, const uint32_t (*T)[32 * W][W]) {
    for (int i = 0; dist; ++i, dist >>= 1) {
        if (!(dist & 1ull)) continue;
        uint32_t r[W] = {};
        for (int b = 0; b < 32 * W; ++b)
            if ((v[b / 32] >> (b % 32)) & 1u)
#pragma unroll
                for (int w = 0; w < W; ++w) r[w] ^= T[i][b][w];
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = r[w];
    }
}

std::mutex g_tables_mu;
std::vector<int> g_tables_ready;  // per device ordinal

cudaError_t ensure_jump_tables(cudaStream_t stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if ((int)g_tables_ready.size() <= dev) g_tables_ready.resize(dev + 1, 0);
    if (g_tables_ready[dev]) return cudaSuccess;
    void *p128 = nullptr, *p64 = nullptr, *p32 = nullptr;
    if ((e = cudaGetSymbolAddress(&p128, g_jump_xor128)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress(&p64, g_jump_xor64)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress(&p32, g_jump_xs32)) != cudaSuccess) return e;
    k_build_jump<4><<<1, 128, 0, stream>>>(static_cast<uint32_t(*)[128][4]>(p128));
    k_build_jump<2><<<1, 64, 0, stream>>>(static_cast<uint32_t(*)[64][2]>(p64));
    k_build_jump<1><<<1, 32, 0, stream>>>(static_cast<uint32_t(*)[32][1]>(p32));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Wait once, so that calls on any stream of this device find finished tables.
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return e;
    g_tables_ready[dev] = 1;
    return cudaSuccess;
}

// ------------------------------------------------ BBS jump
// x <- x^(2^E) mod M with E = 11 * dist squarings, through the exponent
// 2^E mod lambda(M), lambda = lcm(p - 1, q - 1) (x is a unit mod M);
// lambda and its Barrett reciprocal come from k_split_lambda.
__device__ __forceinline__ uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// a^e mod M for a < M, left to right over 2-bit windows of e: two squarings
// and one product by a^w (by 1 for w = 0) per window, the same work in every
// lane whatever its exponent bits.
__device__ __forceinline__ uint64_t pow_mod(const Barrett62 &B, uint64_t a, uint64_t e) {
    if (e == 0) return 1 % B.M;
    const uint64_t a2 = B.mul(a, a), a3 = B.mul(a2, a), one = 1 % B.M;
    int i = (63 - __clzll((long long)e)) & ~1;  // the window that holds the top bit
    uint32_t w = (uint32_t)(e >> i) & 3u;
    uint64_t r = w == 1u ? a : w == 2u ? a2 : a3;
    for (i -= 2; i >= 0; i -= 2) {
        r = B.mul(r, r);
        r = B.mul(r, r);
        w = (uint32_t)(e >> i) & 3u;
        r = B.mul(r, w == 0u ? one : w == 1u ? a : w == 2u ? a2 : a3);
    }
    return r;
}

__device__ __forceinline__ uint64_t bbs_jump(uint64_t y, uint64_t M, uint64_t mu, uint64_t lam, uint64_t lam_mu,
                                             uint64_t squarings) {
    Barrett62 L;
    L.set(lam, lam_mu);
    // 2^squarings mod lam by square-and-multiply on the exponent's bits
    const uint64_t e = pow_mod(L, 2 % lam, squarings);
    Barrett62 B;
    B.set(M, mu);
    return pow_mod(B, y, e);
}

// ------------------------------------------------ segment states
struct SegSpace {
    DevState v0;        // view of segment 0 (pointers into the workspace)
    uint64_t stride;    // bytes between segment states
    __device__ __forceinline__ DevState at(uint64_t k) const {
        DevState s = v0;
        const uint64_t off = k * stride;
        s.table = v0.table + off;
        s.u32 = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(v0.u32) + off);
        if (v0.u64) s.u64 = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(v0.u64) + off);
        return s;
    }
};

constexpr int kOwnWords = 4;  // F_A .. F_D (CI_VAR_BBS16: the eight states F_Y16 ..)

// Own words of every segment's start (k >= 1), saved by k_split_setup for the
// regenerate form: field f of segment k, lane l at u32[(f * K + k) * P + l].
struct OwnSave {
    uint32_t *u32;  // `count` fields from `first` (nullptr: not saved)
    uint64_t *u64;  // the BBS state (CI_VAR_BBS)
    int first, count;
};

// Algorithm 5 as printed, run as a segment of one call: the arrays are the
// ones the call chose when it started (stored in the sel field by
// k_split_setup, as sel1 | sel2 << 8), and the generators are not rotated at
// the segment's end (the call rotates them once, when its last segment
// becomes the caller's state).
struct SrcBbs16Seg : SrcBbs16 {
    __device__ __forceinline__ void load(const DevState &s, uint64_t l) {
        SrcBbs16::load(s, l);
        const uint32_t sel = s.u32[F_SEL * s.P + l];
        sel1 = sel & 7u;
        sel2 = (sel >> 8) & 7u;
    }
    __device__ __forceinline__ void store(const DevState &s, uint64_t l) const {
#pragma unroll
        for (int k = 0; k < 8; ++k) s.u32[(F_Y16 + k) * s.P + l] = y[k];
    }
};

// Squarings of generator k (BBS1 .. BBS8) per output of Algorithm 5 as printed:
// one chunk each, then BBS3 and BBS1, BBS7 and BBS2 for the two shift steps.
__constant__ uint32_t c_bbs16_squarings[8] = {2, 2, 2, 1, 1, 1, 2, 1};

// lambda(M) = lcm(p - 1, q - 1) of each lane's BBS modulus and its Barrett
// reciprocal, once per lane (every segment's jump uses them):
// lam[l] = lambda, lam[P + l] = barrett_mu(lambda).
__global__ void __launch_bounds__(256) k_split_lambda(DevState src, uint64_t *lam) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < src.P; l += stride) {
        const uint64_t p = src.u32[F_P * src.P + l], q = src.u32[F_Q * src.P + l];
        const uint64_t v = (p - 1) / gcd64(p - 1, q - 1) * (q - 1);
        lam[l] = v;
        lam[src.P + l] = barrett_mu(v);
    }
}

// lambda(M) = lcm(p - 1, q - 1) of each 16-bit modulus M = p q (p != q primes,
// as seeded), by trial division; lam[k * P + l] for generator k of lane l.
__global__ void __launch_bounds__(256) k_split_lambda16(DevState src, uint32_t *lam) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < src.P; l += stride)
        for (int k = 0; k < 8; ++k) {
            const uint32_t M = src.u32[(F_M16 + k) * src.P + l];
            uint32_t p = M;  // a prime M (not seeded) gets lambda = M - 1
            for (uint32_t d = 3; d * d <= M; d += 2)
                if (M % d == 0) {
                    p = d;
                    break;
                }
            const uint32_t q = p == M ? 2u : M / p;
            uint32_t a = p - 1, b = q - 1;
            while (b) {
                const uint32_t t = a % b;
                a = b;
                b = t;
            }
            lam[(uint64_t)k * src.P + l] = (p - 1) / a * (q - 1);
        }
}

__device__ __forceinline__ uint32_t pow_mod32(uint32_t a, uint64_t e, uint32_t m) {
    uint64_t r = 1 % m, b = a % m;
    while (e) {
        if (e & 1ull) r = r * b % m;
        b = b * b % m;
        e >>= 1;
    }
    return (uint32_t)r;
}

// Thread (k, l): segment k's lane l.  Copies the caller's lane (and the
// partner table), jumps the own generator by k * len iterations and, for
// k >= 1, clears slot and x.
__global__ void __launch_bounds__(256) k_split_setup(DevState src, SegSpace seg, uint32_t K, uint64_t len,
                                                     int variant, int xl, OwnSave own, const uint32_t *lam16,
                                                     const uint64_t *lam64) {
    const int nf = variant == CI_VAR_BBS16 ? kU32FieldsBbs16 : kU32Fields;
    const uint64_t total = (uint64_t)(K + (variant == CI_VAR_BBS16 ? 1 : 0)) * src.P;  // BBS16: slot K, a copy of the start
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t k = t / src.P, l = t % src.P;
        const DevState d = seg.at(k);
        for (uint64_t w = l; w < kTableBytes / 4; w += src.P)
            reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(d.table))[w] =
                reinterpret_cast<const uint32_t *>(src.table)[w];
        for (int f = 0; f < nf; ++f) d.u32[f * src.P + l] = src.u32[f * src.P + l];
        if (variant == CI_VAR_BBS)
            for (int f = 0; f < kU64Fields; ++f) d.u64[f * src.P + l] = src.u64[f * src.P + l];
        if (variant == CI_VAR_BBS16)  // the arrays the call chose at its start, for every segment
            d.u32[F_SEL * src.P + l] = (src.u32[F_Y16 * src.P + l] & 7u) | ((src.u32[(F_Y16 + 1) * src.P + l] & 7u) << 8);
        if (k == 0 || k == K) continue;
        d.u32[F_X * src.P + l] = 0;
        d.u32[F_SLOT * src.P + l] = 0;
        const uint64_t dist = k * len;
        if (variant == CI_VAR_BBS16) {
            for (int g = 0; g < 8; ++g) {  // x <- x^(2^(c_g dist) mod lambda(M)) mod M
                const uint32_t M = src.u32[(F_M16 + g) * src.P + l], lam = lam16[(uint64_t)g * src.P + l];
                const uint32_t e = pow_mod32(2, c_bbs16_squarings[g] * dist, lam);
                d.u32[(F_Y16 + g) * src.P + l] = pow_mod32(src.u32[(F_Y16 + g) * src.P + l], e, M);
            }
        } else if (variant == CI_VAR_BBS) {
            d.u64[G_Y * src.P + l] = bbs_jump(src.u64[G_Y * src.P + l], src.u64[G_M * src.P + l],
                                              src.u64[G_MU * src.P + l], lam64[l], lam64[src.P + l], 11ull * dist);
        } else if (xl == CI_XL_XOR128) {
            uint32_t v[4];
            for (int w = 0; w < 4; ++w) v[w] = src.u32[(F_A + w) * src.P + l];
            jump_words<4>(v, dist, g_jump_xor128);
            for (int w = 0; w < 4; ++w) d.u32[(F_A + w) * src.P + l] = v[w];
        } else if (xl == CI_XL_XOR64) {
            uint32_t v[2] = {src.u32[F_A * src.P + l], src.u32[F_B * src.P + l]};
            jump_words<2>(v, dist, g_jump_xor64);
            d.u32[F_A * src.P + l] = v[0];
            d.u32[F_B * src.P + l] = v[1];
        } else {
            uint32_t v[1] = {src.u32[F_A * src.P + l]};
            jump_words<1>(v, dist, g_jump_xs32);
            d.u32[F_A * src.P + l] = v[0];
        }
        if (own.u32) {
            for (int f = 0; f < own.count; ++f)
                own.u32[((uint64_t)f * K + k) * src.P + l] = d.u32[(own.first + f) * src.P + l];
            if (own.u64) own.u64[k * src.P + l] = d.u64[G_Y * src.P + l];
        }
    }
}

// 32 x 32 GF(2) matrices over a warp's lanes, lane l holding row l (bit m of
// row l = entry (l, m)).  C = A B: row_l(C) = XOR of row_m(B) over the set
// bits m of row_l(A).  M v for a vector of words v (one per lane): lane l
// takes the XOR of v_m over the set bits m of row_l(M).
__device__ __forceinline__ uint32_t mat_mul(uint32_t a_row, uint32_t b_row) {
    uint32_t c = 0;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const uint32_t b = __shfl_sync(kFull, b_row, m);
        c ^= ((a_row >> m) & 1u) ? b : 0u;
    }
    return c;
}

__device__ __forceinline__ uint32_t mat_vec(uint32_t m_row, uint32_t v) {
    uint32_t r = 0;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const uint32_t b = __shfl_sync(kFull, v, m);
        r ^= ((m_row >> m) & 1u) ? b : 0u;
    }
    return r;
}

// The carry scan over the segments of one warp group, with one block of NW
// (up to 16) warps per group.  c_j, the true (slot, x) at the start of segment j, obeys
// c_j = e_{j-1} ^ H(c_{j-1}), c_0 = 0 (segment 0 ran from the true state),
// with e_{j-1} the particular end of segment j-1 and H(s, x) = (Q s, x ^ S s).
// Warp w owns steps j in [j0, j1) (m = ceil((K-1) / NW) each):
//   1. local scan from zero: d_j = e_{j-1} ^ H(d_{j-1}), d_{j0-1} = 0, kept in
//      starts[j]; its end goes to shared memory;
//   2. carry-in c_{j0-1}: fold the earlier warps' local ends through H^m,
//      whose pair (Q_m, T_m) follows from (Q, S) by the binary method on m
//      (H^(a+b) = (Q_a Q_b, T_b ^ T_a Q_b));
//   3. c_j = d_j ^ H^(j - j0 + 1)(c_{j0-1}).
// Fix-up form (`own` == nullptr): c_j goes to starts[j].  Regenerate form:
// c_j and the saved own words of segment j's start go into its state.
template <class Src>
__global__ void __launch_bounds__(512) k_split_carry(SegSpace seg, uint32_t K, uint64_t len, uint2 *starts,
                                                      OwnSave own) {
    __shared__ uint32_t end_s[16][32], end_x[16][32];
    const uint64_t g = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, NW = blockDim.x >> 5;
    const DevState s0 = seg.at(0);
    const uint64_t P = s0.P, l = g * 32 + lane;
    CI_WARP_CHECK(s0, g < P / 32, CHK_GROUP, g);  // g = blockIdx.x: every warp of the block returns together
    Src src;
    src.load(s0, l);
    int a1, a2;
    src.arrays(s0, l, a1, a2);
    const uint32_t prow = (1u << s0.table[a1 * 32 + lane]) ^ (1u << s0.table[a2 * 32 + lane]);
    // Q = P^len, S = P + ... + P^len, by the bits of len from the top:
    // (Q, S) for k -> 2k: S <- S ^ Q S, Q <- Q Q; k -> k + 1: Q <- Q P, S <- S ^ Q.
    uint32_t Q = 1u << lane, S = 0;
    for (int b = 63; b >= 0; --b) {
        S ^= mat_mul(Q, S);
        Q = mat_mul(Q, Q);
        if ((len >> b) & 1ull) {
            Q = mat_mul(Q, prow);
            S ^= Q;
        }
    }
    const uint32_t m = (K - 1 + NW - 1) / NW;
    const uint32_t j0 = 1 + w * m, j1 = min(K, j0 + m);
    // 1. local scan; segment ends loaded one step ahead
    uint32_t ds = 0, dx = 0;
    if (j0 < j1) {
        DevState d = seg.at(j0 - 1);
        uint32_t es = d.u32[F_SLOT * P + l], ex = d.u32[F_X * P + l];
        for (uint32_t j = j0; j < j1; ++j) {
            uint32_t ns_e = 0, nx_e = 0;
            if (j + 1 < j1) {
                d = seg.at(j);
                ns_e = d.u32[F_SLOT * P + l];
                nx_e = d.u32[F_X * P + l];
            }
            const uint32_t ns = es ^ mat_vec(Q, ds);
            dx = ex ^ dx ^ mat_vec(S, ds);
            ds = ns;
            starts[(uint64_t)j * P + l] = make_uint2(ds, dx);
            es = ns_e;
            ex = nx_e;
        }
    }
    end_s[w][lane] = ds;
    end_x[w][lane] = dx;
    __syncthreads();
    // 2. H^m and this warp's carry-in
    uint32_t Qm = 1u << lane, Tm = 0;
    for (int b = 31; b >= 0; --b) {
        Tm ^= mat_mul(Tm, Qm);
        Qm = mat_mul(Qm, Qm);
        if ((m >> b) & 1u) {
            Qm = mat_mul(Qm, Q);
            Tm = S ^ mat_mul(Tm, Q);
        }
    }
    uint32_t cs = 0, cx = 0;
    for (int v = 0; v < w; ++v) {
        const uint32_t ns = end_s[v][lane] ^ mat_vec(Qm, cs);
        cx = end_x[v][lane] ^ cx ^ mat_vec(Tm, cs);
        cs = ns;
    }
    // 3. true starts of this warp's segments
    for (uint32_t j = j0; j < j1; ++j) {
        const uint32_t ns = mat_vec(Q, cs);
        cx ^= mat_vec(S, cs);
        cs = ns;
        const uint2 dj = starts[(uint64_t)j * P + l];
        const uint32_t ts = dj.x ^ cs, tx = dj.y ^ cx;
        if (!own.u32) {
            starts[(uint64_t)j * P + l] = make_uint2(ts, tx);
        } else {
            const DevState d = seg.at(j);
            d.u32[F_SLOT * P + l] = ts;
            d.u32[F_X * P + l] = tx;
            for (int f = 0; f < own.count; ++f) d.u32[(own.first + f) * P + l] = own.u32[((uint64_t)f * K + j) * P + l];
            if (own.u64) d.u64[G_Y * P + l] = own.u64[(uint64_t)j * P + l];
        }
    }
}

// Written sink: segment k >= 1 wrote its particular outputs (zero start).
// From its true start c = (s_a, x_a), the homogeneous part is h <- P h,
// acc <- acc ^ h per iteration (two shuffles, as in the mixing step with a
// zero own word); output i of the segment gets acc XORed in.  The warp stages
// 32 iterations of its 32 rows in the swizzled tile and updates the outputs
// as 16-byte row segments (V4) or words.  Another warp wrote those outputs,
// so they are read through L2 (ld.global.cg).  Returns H(c) = (h, acc) at the
// segment's end.
template <bool V4>
__device__ __forceinline__ uint2 fix_segment(uint2 c, int p1, int p2, uint64_t n, uint32_t *base, uint64_t row0,
                                             uint64_t S, uint64_t ld, uint4 *tile) {
    const int lane = threadIdx.x & 31;
    uint32_t *tw = reinterpret_cast<uint32_t *>(tile);
    uint32_t h = c.x, acc = c.y;
    auto step = [&]() {
        h = __shfl_sync(kFull, h, p1) ^ __shfl_sync(kFull, h, p2);
        acc ^= h;
        return acc;
    };
    const uint64_t nfull = n - n % 32;
    for (uint64_t i0 = 0; i0 < nfull; i0 += 32) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint4 f;
            f.x = step();
            f.y = step();
            f.z = step();
            f.w = step();
            tile[lane * 8 + (q ^ (lane & 7))] = f;
        }
        __syncwarp();
        if (V4) {
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                const int r = 4 * kk + lane / 8, cc = lane % 8;
                if (row0 + r < S) {
                    uint4 *p = reinterpret_cast<uint4 *>(base + (row0 + r) * ld + i0 + 4 * cc);
                    const uint4 v = tile[r * 8 + (cc ^ (r & 7))];
                    uint4 o = __ldcg(p);
                    o.x ^= v.x;
                    o.y ^= v.y;
                    o.z ^= v.z;
                    o.w ^= v.w;
                    store16<0>(reinterpret_cast<uint32_t *>(p), o);
                }
            }
        } else {
            for (int r = 0; r < 32; ++r)
                if (row0 + r < S) {
                    uint32_t *p = base + (row0 + r) * ld + i0 + lane;
                    *p = __ldcg(p) ^ tw[tile_word<32>(r, lane)];
                }
        }
        __syncwarp();
    }
    const int rem = (int)(n - nfull);
    if (rem) {
        for (int kk = 0; kk < rem; ++kk) tw[tile_word<32>(lane, kk)] = step();
        __syncwarp();
        for (int r = 0; r < 32; ++r)
            if (lane < rem && row0 + r < S) {
                uint32_t *p = base + (row0 + r) * ld + nfull + lane;
                *p = __ldcg(p) ^ tw[tile_word<32>(r, lane)];
            }
        __syncwarp();
    }
    return make_uint2(h, acc);
}

// The fix-ups as a kernel of their own, after pass 1 and the carry scan:
// work unit = (segment k >= 1, warp group g), all independent; the last
// segment also corrects its end state.
template <class Src, bool V4>
__global__ void __launch_bounds__(256) k_split_fixup(SegSpace seg, const uint2 *starts, uint32_t K, uint64_t len,
                                                     uint64_t len_last, uint64_t groups, uint32_t *out, uint64_t ld,
                                                     uint64_t col0) {
    __shared__ uint4 tiles[8][256];
    const int lane = threadIdx.x & 31;
    uint4 *tile = tiles[threadIdx.x >> 5];
    const DevState s0 = seg.at(0);
    const uint64_t P = s0.P;
    const uint64_t units = (uint64_t)(K - 1) * groups;
    for (uint64_t u = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5); u < units; u += (uint64_t)gridDim.x * 8) {
        const uint64_t k = 1 + u / groups, g = u % groups, l = g * 32 + lane;
        CI_WARP_CHECK(s0, k < K && g < P / 32, CHK_SEGMENT, k);
        CI_WARP_CHECK(s0, col0 + k * len + (k + 1 == K ? len_last : len) <= ld, CHK_SEG_COLS, k);
        if (V4) CI_WARP_CHECK(s0, ((col0 + k * len) | ld) % 4 == 0, CHK_V4_ALIGN, k);
        Src src;
        src.load(s0, l);
        int a1, a2;
        src.arrays(s0, l, a1, a2);
        const uint2 hk = fix_segment<V4>(starts[k * P + l], s0.table[a1 * 32 + lane], s0.table[a2 * 32 + lane],
                                         k + 1 == K ? len_last : len, out + col0 + k * len, g * 32, s0.S, ld, tile);
        if (k + 1 == K) {
            const DevState d = seg.at(K - 1);
            d.u32[F_SLOT * P + l] ^= hk.x;
            d.u32[F_X * P + l] ^= hk.y;
        }
    }
}

// The last segment's state becomes the caller's state (the sel field, which
// generation never changes, stays the caller's).  CI_VAR_BBS16: generator k
// (state and modulus) moves to place k + 1, the call's one rotation.
__global__ void __launch_bounds__(256) k_split_copy_back(DevState dst, DevState last, int variant) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < dst.P; l += stride) {
        for (int f = 0; f < kU32Fields; ++f)
            if (f != F_SEL) dst.u32[f * dst.P + l] = last.u32[f * dst.P + l];
        if (variant == CI_VAR_BBS16)
            for (int k = 0; k < 8; ++k) {
                dst.u32[(F_Y16 + (k + 1) % 8) * dst.P + l] = last.u32[(F_Y16 + k) * dst.P + l];
                dst.u32[(F_M16 + (k + 1) % 8) * dst.P + l] = last.u32[(F_M16 + k) * dst.P + l];
            }
        if (dst.u64)
            for (int f = 0; f < kU64Fields; ++f) dst.u64[f * dst.P + l] = last.u64[f * dst.P + l];
    }
}

// Combines per-segment consumer results r[k * P + l] for stream l < S:
// quarter-circle counts are added to out[l]; digests are joined by Horner,
// D = sum_k D_k K^(n - end of segment k), the last segment ending at n.
__global__ void __launch_bounds__(256) k_split_combine(const uint64_t *r, uint64_t *out, uint64_t P, uint64_t S,
                                                       uint32_t K, uint64_t len, uint64_t len_last, int digest) {
    const uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= S) return;
    if (!digest) {
        uint64_t c = 0;
        for (uint32_t k = 0; k < K; ++k) c += r[(uint64_t)k * P + l];
        out[l] += c;
        return;
    }
    auto kpow = [](uint64_t e) {
        uint64_t b = kDigestMul, p = 1;
        while (e) {
            if (e & 1ull) p *= b;
            b *= b;
            e >>= 1;
        }
        return p;
    };
    const uint64_t step = kpow(len);
    uint64_t d = 0, mult = 1;
    for (uint32_t k = K; k-- > 0;) {
        d += r[(uint64_t)k * P + l] * mult;
        mult *= (k == K - 1) ? kpow(len_last) : step;
    }
    out[l] = d;
}

// Consumer results from written rows: the scratch form of a BBS-source
// consumer call, whose outputs were written (and fixed up) into `rows`, row r
// (stride n) holding stream r's n outputs.  Work unit = (row r, chunk
// [b, e) of clen outputs), one warp.  Quarter-circle sink: the chunk's hits
// among its pairs (o_2k, o_2k+1) are added to out[r] (clen and n even).
// Digest sink: the chunk contributes K^(n-e) sum_{b<=i<e} o_i K^(e-1-i), so
// the contributions of all chunks sum to D = sum_i o_i K^(n-1-i); lane j
// takes outputs e-1-j, e-1-j-32, ... with the running power K^j, K^(j+32), ...,
// and out[r] (cleared before) receives the warp's sum.
__device__ __forceinline__ uint64_t digest_pow(uint64_t e) {
    uint64_t b = kDigestMul, p = 1;
    while (e) {
        if (e & 1ull) p *= b;
        b *= b;
        e >>= 1;
    }
    return p;
}

template <bool kDigest>
__global__ void __launch_bounds__(256) k_consume_rows(const uint32_t *rows, uint64_t S, uint64_t n, uint64_t clen,
                                                      uint64_t chunks, uint64_t *out) {
    const int lane = threadIdx.x & 31;
    const uint64_t units = S * chunks;
    for (uint64_t u = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; u < units; u += (uint64_t)gridDim.x * 8) {
        const uint64_t r = u / chunks, c = u % chunks;
        const uint64_t b = c * clen, e = b + clen < n ? b + clen : n;
        const uint32_t *row = rows + r * n;
        uint64_t v = 0;
        if (kDigest) {
            uint64_t pw = digest_pow((uint64_t)lane);
            const uint64_t step = digest_pow(32);
            for (uint64_t t = (uint64_t)lane; t < e - b; t += 32) {
                v += (uint64_t)row[e - 1 - t] * pw;
                pw *= step;
            }
        } else {
            const uint2 *pairs = reinterpret_cast<const uint2 *>(row + b);
            for (uint64_t k = (uint64_t)lane; k < (e - b) / 2; k += 32) {
                const uint2 o = pairs[k];
                v += 1u - qc_miss(o.x, o.y);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(out + r), kDigest ? v * digest_pow(n - e) : v);
    }
}

// ------------------------------------------------ host side
constexpr uint32_t kMaxSegments = kSplitMaxSegments;
constexpr uint64_t kMinSegment = 256;       // iterations per segment (auto choice, BBS)
constexpr uint64_t kMinAutoSegment = 1024;  // ... xor-likes, and when a single call splits on its own
constexpr uint64_t kScratchWords = 1ull << 29;  // scratch outputs of a BBS-source consumer call (2 GiB)
// Written BBS-source outputs take the one-launch fix-up form from this many
// warp groups per SM on: its fix-ups run as one serial chain per group among
// the squaring warps, which keeps pace only with enough groups; below it,
// pass 1, the carry scan and the fix-ups run as three launches.
#ifndef CI_ONE_LAUNCH_GROUPS_PER_SM
#define CI_ONE_LAUNCH_GROUPS_PER_SM 12
#endif
constexpr uint64_t kOneLaunchGroupsPerSm = CI_ONE_LAUNCH_GROUPS_PER_SM;

// One pass over segments [k_begin, k_end): work unit u is segment
// k_begin + u / groups, warp group u % groups, run for its length (len, the
// last segment len_last) by the generator's warp loop into SINK: written
// outputs at column col0 + k len of rows of stride ld; consumer results into
// aux + k P.  Segment 0 is the caller's own state when `zero` < 0, else the
// segment state with that index.
// Instantiated per source and sink, with at most 64 registers (4 blocks of 8
// warps per SM): the all-source batched kernel needs 128, which held the
// BBS segments to 16 resident warps per SM.  BBS segments (one serial
// squaring chain per lane) ask for 5 blocks, i.e. 48 registers; segments of
// Algorithm 5 as printed (eight generators per lane, 118 registers in the
// single-call kernel) for 2 blocks, 128 registers, so that their loop does
// not spill.
template <class Src>
constexpr int split_min_blocks() {
    return std::is_same<Src, SrcBbs>::value ? 5 : std::is_same<Src, SrcBbs16Seg>::value ? 2 : 4;
}

template <class Src, int SINK>
__global__ void __launch_bounds__(256, split_min_blocks<Src>()) k_split_run(SegSpace seg, DevState caller, int zero, uint32_t k_begin,
                                                   uint32_t k_end, uint32_t K, uint64_t len, uint64_t len_last,
                                                   uint64_t groups, uint32_t *out, uint64_t ld, uint64_t col0,
                                                   uint64_t *aux) {
    __shared__ uint4 tiles[8][256];
    uint4 *tile = tiles[threadIdx.x >> 5];
    const uint64_t units = (uint64_t)(k_end - k_begin) * groups;
    // warp w of block b starts at unit w * gridDim.x + b: a partial last
    // round of warps is spread over every block (and SM)
    for (uint64_t u = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; u < units; u += (uint64_t)gridDim.x * 8) {
        const uint64_t k = k_begin + u / groups, g = u % groups;
        CI_WARP_CHECK(caller, k < K, CHK_SEGMENT, k);
        const DevState st = k != 0 ? seg.at(k) : zero < 0 ? caller : seg.at((uint64_t)zero);
        const uint64_t n = k + 1 == K ? len_last : len;
        if (SINK == SINK_V4 || SINK == SINK_SCALAR)
            warp_task<Src, SINK>(st, g, n, out, ld, col0 + k * len, nullptr, tile);
        else
            warp_task<Src, SINK>(st, g, n, nullptr, 0, 0, aux + k * caller.P, tile);
    }
}

template <class Src, int SINK>
cudaError_t launch_split_run(const SegSpace &sp, const DevState &caller, int zero, uint32_t kb, uint32_t ke,
                             uint32_t K, uint64_t len, uint64_t len_last, uint32_t *out, uint64_t ld, uint64_t col0,
                             uint64_t *aux, cudaStream_t stream) {
    static int per_sm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_split_run<Src, SINK>, 256, 0);
        if (per_sm <= 0) per_sm = 1;
    });
    const uint64_t groups = caller.P / 32, units = (uint64_t)(ke - kb) * groups;
    if (units == 0) return cudaSuccess;
    const int blocks = (int)std::min<uint64_t>(units, (uint64_t)sm_count() * per_sm);  // a block per unit at most
    k_split_run<Src, SINK><<<blocks, 256, 0, stream>>>(sp, caller, zero, kb, ke, K, len, len_last, groups, out, ld,
                                                       col0, aux);
    return cudaGetLastError();
}

// Written BBS-source outputs, fix-up form, in one launch.  Work units are the
// pass-1 units (segment k, warp group g), taken from a device counter in
// segment-major order.  Fix-up (g, k), k >= 1, needs two events: pass 1 of
// (g, k) has written its particular outputs and end e_k, and the true start
// c_k of segment k is known.  c_1 is the end of segment 0 (which ran from the
// true state), and c_(k+1) = e_k ^ H(c_k), which fix-up (g, k) produces
// itself by running the homogeneous recurrence through the segment, so the
// carry needs no matrix powers.  Each event adds one to events[k groups + g];
// the warp whose addition makes it two runs the fix-up at once, then goes on
// to the group's next segment while that one's pass 1 is already done.  No
// warp waits for another, and the fix-ups' memory traffic overlaps the other
// warps' squarings.  The last segment's fix-up corrects the call's end state.

// Adds one to the event count *ev once the earlier writes of every lane are
// visible device-wide (the release half of the pattern); true in every lane
// when this addition made the count two, the other event's writes then being
// visible to the warp's L2 reads (the acquire half).
__device__ __forceinline__ bool second_event(uint32_t *ev) {
    __threadfence();
    __syncwarp();
    uint32_t old = 0;
    if ((threadIdx.x & 31) == 0) old = atomicAdd(ev, 1u);
    old = __shfl_sync(kFull, old, 0);
    __threadfence();
    return old == 1u;
}

template <class Src, int SINK>
__global__ void __launch_bounds__(256, split_min_blocks<Src>()) k_split_run_fix(SegSpace seg, uint32_t K, uint64_t len,
                                                       uint64_t len_last, uint64_t groups, uint32_t *out, uint64_t ld,
                                                       uint64_t col0, uint2 *starts, uint32_t *events,
                                                       unsigned long long *next_unit) {
    __shared__ uint4 tiles[8][256];
    uint4 *tile = tiles[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const DevState s0 = seg.at(0);
    const uint64_t P = s0.P, units = (uint64_t)K * groups;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(next_unit, 1ull);
        u = __shfl_sync(kFull, u, 0);
        if (u >= units) return;
        uint64_t k = u / groups;
        const uint64_t g = u % groups, l = g * 32 + lane;
        const DevState st = seg.at(k);
        warp_task<Src, SINK>(st, g, k + 1 == K ? len_last : len, out, ld, col0 + k * len, nullptr, tile);
        if (k == 0) {  // the same threads stored segment 0's end: c_1
            starts[P + l] = make_uint2(st.u32[F_SLOT * P + l], st.u32[F_X * P + l]);
            k = 1;
        }
        int p1 = -1, p2 = -1;
        while (second_event(events + k * groups + g)) {
            CI_WARP_CHECK(s0, k < K && g < P / 32, CHK_SEGMENT, k);
            CI_WARP_CHECK(s0, col0 + k * len + (k + 1 == K ? len_last : len) <= ld, CHK_SEG_COLS, k);
            if (SINK == SINK_V4) CI_WARP_CHECK(s0, ((col0 + k * len) | ld) % 4 == 0, CHK_V4_ALIGN, k);
            if (p1 < 0) {
                Src src;
                src.load(s0, l);
                int a1, a2;
                src.arrays(s0, l, a1, a2);
                p1 = s0.table[a1 * 32 + lane];
                p2 = s0.table[a2 * 32 + lane];
            }
            const uint2 hk = fix_segment<SINK == SINK_V4>(__ldcg(starts + k * P + l), p1, p2,
                                                          k + 1 == K ? len_last : len, out + col0 + k * len, g * 32,
                                                          s0.S, ld, tile);
            const DevState d = seg.at(k);
            const uint32_t ts = __ldcg(d.u32 + F_SLOT * P + l) ^ hk.x, tx = __ldcg(d.u32 + F_X * P + l) ^ hk.y;
            if (k + 1 == K) {
                d.u32[F_SLOT * P + l] = ts;
                d.u32[F_X * P + l] = tx;
                break;
            }
            starts[(k + 1) * P + l] = make_uint2(ts, tx);
            ++k;
        }
    }
}

template <class Src, int SINK>
cudaError_t launch_split_run_fix(const SegSpace &sp, uint32_t K, uint64_t len, uint64_t len_last, uint64_t groups,
                                 uint32_t *out, uint64_t ld, uint64_t col0, uint2 *starts, uint32_t *events,
                                 unsigned long long *next_unit, cudaStream_t stream) {
    static int per_sm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_split_run_fix<Src, SINK>, 256, 0);
        if (per_sm <= 0) per_sm = 1;
    });
    const uint64_t units = (uint64_t)K * groups;
    const int blocks = (int)std::min<uint64_t>((units + 7) / 8, (uint64_t)sm_count() * per_sm);
    k_split_run_fix<Src, SINK><<<blocks, 256, 0, stream>>>(sp, K, len, len_last, groups, out, ld, col0, starts, events,
                                                           next_unit);
    return cudaGetLastError();
}

template <int SINK>
cudaError_t split_run_sink(int variant, int xl, const SegSpace &sp, const DevState &caller, int caller0, uint32_t kb,
                           uint32_t ke, uint32_t K, uint64_t len, uint64_t len_last, uint32_t *out, uint64_t ld,
                           uint64_t col0, uint64_t *aux, cudaStream_t stream) {
    if (variant == CI_VAR_BBS)
        return launch_split_run<SrcBbs, SINK>(sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0, aux, stream);
    if (variant == CI_VAR_BBS16)
        return launch_split_run<SrcBbs16Seg, SINK>(sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0, aux,
                                                   stream);
    if (xl == CI_XL_XORSHIFT32)
        return launch_split_run<SrcXorshift32, SINK>(sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0, aux,
                                                     stream);
    if (xl == CI_XL_XOR64)
        return launch_split_run<SrcXor64, SINK>(sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0, aux,
                                                stream);
    return launch_split_run<SrcXor128, SINK>(sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0, aux,
                                             stream);
}

// Runs segments [kb, ke) into the caller's sink (CI_SINK_*); written outputs
// take 16-byte stores when out, ld and col0 allow it.  Segment 0: the caller's
// state (zero < 0) or segment state `zero`.
cudaError_t split_run(const ci_states_s &h, int sink, const SegSpace &sp, int caller0, uint32_t kb, uint32_t ke,
                      uint32_t K, uint64_t len, uint64_t len_last, uint32_t *out, uint64_t ld, uint64_t col0,
                      uint64_t *aux, cudaStream_t stream) {
    const DevState caller = h.view();
    if (sink == CI_SINK_QC)
        return split_run_sink<SINK_QC>(h.variant, h.xl, sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0,
                                       aux, stream);
    if (sink == CI_SINK_DIGEST)
        return split_run_sink<SINK_DIGEST>(h.variant, h.xl, sp, caller, caller0, kb, ke, K, len, len_last, out, ld,
                                           col0, aux, stream);
    const bool v4 = (reinterpret_cast<uintptr_t>(out) & 15u) == 0 && ld % 4 == 0 && col0 % 4 == 0 && len % 4 == 0;
    if (v4)
        return split_run_sink<SINK_V4>(h.variant, h.xl, sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0,
                                       aux, stream);
    return split_run_sink<SINK_SCALAR>(h.variant, h.xl, sp, caller, caller0, kb, ke, K, len, len_last, out, ld, col0,
                                       aux, stream);
}

int split_block_count(uint64_t items) {
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((items + 255) / 256, (uint64_t)sm_count() * 8));
}

}  // namespace
}  // namespace ci

namespace ci {

cudaError_t split_prepare(cudaStream_t stream) { return ensure_jump_tables(stream); }

uint64_t split_segments(const ci_states_s &h, uint64_t n, uint64_t requested) {
    const uint64_t groups = h.P / 32;
    uint64_t K = requested;
    if (K == 0) {  // fill about four waves of resident warps
        const uint64_t target = (uint64_t)sm_count() * 64;
        // cheap xor-like segments: fewer, longer ones (the setup's GF(2) jumps
        // cost more than their generation)
        const uint64_t min_len = h.variant == CI_VAR_XOR ? kMinAutoSegment : kMinSegment;
        K = std::max<uint64_t>(1, target / groups);
        K = std::min<uint64_t>(K, std::max<uint64_t>(1, n / min_len));
    }
    K = std::min<uint64_t>(K, kMaxSegments);
    const uint64_t len = ((n + K - 1) / K + 31) / 32 * 32;  // whole staging tiles, 16-byte column offsets
    return (n + len - 1) / len;
}

uint64_t split_auto_bbs(const ci_states_s &h, uint64_t n, int sink) {
    if (h.variant != CI_VAR_BBS) return 1;
    const uint64_t groups = h.P / 32, sms = (uint64_t)sm_count();
    uint64_t K;
    // consumer sinks whose outputs fit the scratch are written, fixed up and
    // reduced (split_launch), so they take the written rule
    if (sink == CI_SINK_WRITTEN || h.S <= kScratchWords / n) {
        // Measured on 2^9 .. 2^13 warp groups of 2^12 .. 2^15 iterations:
        // about ten waves of resident warps (40 per SM) in the one-launch
        // form, four in the three-launch form; segments of at least 256.
        K = groups >= kOneLaunchGroupsPerSm * sms ? (400 * sms + groups / 2) / groups : 160 * sms / groups;
        K = std::min<uint64_t>(K, n / kMinSegment);
    } else {
        // Larger consumer calls generate twice (pass 1, then pass 2 from the
        // true starts): only states that fill less than about two waves.
        const uint64_t target = sms * 128;
        if (groups * 2 > target) return 1;
        K = std::min<uint64_t>(target / groups, std::max<uint64_t>(1, n / kMinAutoSegment));
    }
    K = std::min<uint64_t>(K, kMaxSegments);
    if (K <= 1) return 1;
    const uint64_t len = ((n + K - 1) / K + 31) / 32 * 32;
    return (n + len - 1) / len;
}

uint64_t split_auto(const ci_states_s &h, uint64_t n, int sink) {
    if (h.variant == CI_VAR_BBS) return split_auto_bbs(h, n, sink);
    const uint64_t groups = h.P / 32, sms = (uint64_t)sm_count();
    if (h.variant == CI_VAR_BBS16) {
        // Algorithm 5 as printed: each warp is bound by its own eight chains,
        // so only states of at most one warp group per SM gain from more
        // warps (measured, written: 1 group 39x, 32 groups 7x, 128 groups
        // 2.8x faster; 512 groups slower), with about two waves of the split
        // kernels' 16 resident warps per SM and segments of at least 256.
        if (groups > sms) return 1;
        uint64_t K = std::min<uint64_t>(sms * 32 / groups, n / kMinSegment);
        K = std::min<uint64_t>(K, kMaxSegments);
        if (K <= 1) return 1;
        const uint64_t len = ((n + K - 1) / K + 31) / 32 * 32;
        return (n + len - 1) / len;
    }
    // xor-likes: only states with no more warp groups than SMs (measured:
    // 4-11x faster up to 128 groups, slower from 512 groups on, where the
    // setup's GF(2) jumps outweigh the parallelism)
    if (h.variant != CI_VAR_XOR || groups > sms) return 1;
    uint64_t K = std::min<uint64_t>(sms * 64 / groups, std::max<uint64_t>(1, n / kMinAutoSegment));
    K = std::min<uint64_t>(K, kMaxSegments);
    if (K <= 1) return 1;
    const uint64_t len = ((n + K - 1) / K + 31) / 32 * 32;
    return (n + len - 1) / len;
}

ci_status split_launch(const ci_states_s &hs, uint64_t n, int sink, uint32_t *out, uint64_t ld, uint64_t col0,
                       uint64_t *aux, uint64_t K, cudaStream_t stream) {
    TraceRange trace("split");
    const ci_states_s *h = &hs;
    const bool b16 = h->variant == CI_VAR_BBS16, bbs = h->variant == CI_VAR_BBS;
    cudaError_t e;
    if (K <= 1) {  // one segment: the caller's state, straight into the sink
        if (b16) {  // one whole call, with its array choice and rotation
            if (sink == CI_SINK_QC) e = launch_fused_qc(*h, n, aux, stream);
            else if (sink == CI_SINK_DIGEST) e = launch_digest(*h, n, aux, stream);
            else if (ld == n && col0 == 0) e = launch_generate(*h, n, out, stream);
            else return fail(CI_E_INVAL, "unsplit CI_VAR_BBS16 output needs ld == n and col0 == 0");
        } else {
            SegSpace none{};
            e = split_run(*h, sink, none, -1, 0, 1, 1, n, n, out, ld, col0, aux, stream);
        }
        return e == cudaSuccess ? CI_OK : cuda_fail(e, "split run");
    }
    // BBS-source consumer sinks: generation is the cost, so the outputs are
    // written (and fixed up) once into a scratch of at most kScratchWords
    // words and reduced into the sink, instead of generating the segments
    // twice; larger calls take the regenerate form below.
    if (sink != CI_SINK_WRITTEN && (bbs || b16) && h->S <= kScratchWords / n) {
        uint32_t *rows = nullptr;
        if ((e = cudaMallocAsync(reinterpret_cast<void **>(&rows), 4 * h->S * n, stream)) != cudaSuccess)
            return cuda_fail(e, "scratch outputs");
        ci_status st = CI_OK;
        if (sink == CI_SINK_DIGEST && (e = cudaMemsetAsync(aux, 0, 8 * h->S, stream)) != cudaSuccess)
            st = cuda_fail(e, "clearing digests");
        if (st == CI_OK) st = split_launch(*h, n, CI_SINK_WRITTEN, rows, n, 0, nullptr, K, stream);
        if (st == CI_OK) {
            // about four waves of 8-warp blocks; chunks of whole 64-output steps
            const uint64_t target = (uint64_t)sm_count() * 8 * 16;
            uint64_t chunks = std::max<uint64_t>(1, std::min<uint64_t>((target + h->S - 1) / h->S, n / 1024));
            const uint64_t clen = ((n + chunks - 1) / chunks + 63) / 64 * 64;
            chunks = (n + clen - 1) / clen;
            const int blocks = (int)std::min<uint64_t>(h->S * chunks, (uint64_t)sm_count() * 16);
            if (sink == CI_SINK_DIGEST)
                k_consume_rows<true><<<blocks, 256, 0, stream>>>(rows, h->S, n, clen, chunks, aux);
            else
                k_consume_rows<false><<<blocks, 256, 0, stream>>>(rows, h->S, n, clen, chunks, aux);
            if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "consuming scratch outputs");
        }
        cudaFreeAsync(rows, stream);
        return st;
    }
    if ((e = ensure_jump_tables(stream)) != cudaSuccess) return cuda_fail(e, "jump tables");
    const uint64_t groups = h->P / 32;
    const uint64_t len = ((n + K - 1) / K + 31) / 32 * 32;
    const uint64_t len_last = n - (K - 1) * len;

    const uint64_t stride = (h->bytes + 255) / 256 * 256;
    const uint64_t slots = K + (b16 ? 1 : 0);  // BBS16: slot K keeps the call's start (for pass 2)
    // Written BBS outputs are fixed up in place (generation is the cost);
    // xor-like outputs are cheaper to generate again than to read back.
    const bool written = sink == CI_SINK_WRITTEN;
    const bool fixup = written && (bbs || b16);
    const int own_first = b16 ? (int)F_Y16 : (int)F_A, own_count = b16 ? 8 : kOwnWords;
    const uint64_t res_bytes = 8ull * K * h->P;  // per-segment consumer results
    const uint64_t own_bytes = fixup ? 0 : (4ull * own_count + (bbs ? 8ull : 0ull)) * K * h->P;
    const uint64_t lam_bytes = b16 ? 4ull * 8 * h->P : bbs ? 16ull * h->P : 0;
    uint8_t *ws = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void **>(&ws), stride * slots + 2 * res_bytes + own_bytes + lam_bytes,
                             stream)) != cudaSuccess)
        return cuda_fail(e, "workspace");
    uint64_t *res1 = reinterpret_cast<uint64_t *>(ws + stride * slots);
    uint64_t *res3 = res1 + K * h->P;
    uint8_t *after = reinterpret_cast<uint8_t *>(res3 + K * h->P);
    OwnSave own{nullptr, nullptr, own_first, own_count};
    if (!fixup) {
        own.u32 = reinterpret_cast<uint32_t *>(after);
        own.u64 = bbs ? reinterpret_cast<uint64_t *>(own.u32 + (uint64_t)own_count * K * h->P) : nullptr;
    }
    uint32_t *lam16 = b16 ? reinterpret_cast<uint32_t *>(after + own_bytes) : nullptr;
    uint64_t *lam64 = bbs ? reinterpret_cast<uint64_t *>(after + own_bytes) : nullptr;

    // Handles over the segment states (host copies of the caller's, moved).
    std::vector<ci_states_s> segs(slots, *h);
    for (uint64_t k = 0; k < slots; ++k) {
        segs[k].dev = ws + k * stride;
        segs[k].owns = false;
    }
    SegSpace sp;
    sp.v0 = segs[0].view();
    sp.stride = stride;
    const DevState src = h->view();

    ci_status st = CI_OK;
    if (b16) k_split_lambda16<<<split_block_count(h->P), 256, 0, stream>>>(src, lam16);
    if (bbs) k_split_lambda<<<split_block_count(h->P), 256, 0, stream>>>(src, lam64);
    k_split_setup<<<split_block_count(slots * h->P), 256, 0, stream>>>(src, sp, (uint32_t)K, len, h->variant, h->xl,
                                                                       own, lam16, lam64);
    if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "split setup");

    if (st == CI_OK && fixup && groups >= kOneLaunchGroupsPerSm * (uint64_t)sm_count()) {
        // one launch: pass 1 with the fix-ups folded in; then the final state
        uint2 *starts = reinterpret_cast<uint2 *>(res1);  // true starts (slot, x) of segments 1 .. K-1
        unsigned long long *next_unit = reinterpret_cast<unsigned long long *>(res3);
        uint32_t *events = reinterpret_cast<uint32_t *>(next_unit + 1);  // K * groups counts
        const bool v4 = (reinterpret_cast<uintptr_t>(out) & 15u) == 0 && ld % 4 == 0 && col0 % 4 == 0;
        const uint32_t k32 = (uint32_t)K;
        if ((e = cudaMemsetAsync(res3, 0, 8 + 4 * K * groups, stream)) == cudaSuccess) {
            if (bbs)
                e = v4 ? launch_split_run_fix<SrcBbs, SINK_V4>(sp, k32, len, len_last, groups, out, ld, col0, starts,
                                                               events, next_unit, stream)
                       : launch_split_run_fix<SrcBbs, SINK_SCALAR>(sp, k32, len, len_last, groups, out, ld, col0,
                                                                   starts, events, next_unit, stream);
            else
                e = v4 ? launch_split_run_fix<SrcBbs16Seg, SINK_V4>(sp, k32, len, len_last, groups, out, ld, col0,
                                                                    starts, events, next_unit, stream)
                       : launch_split_run_fix<SrcBbs16Seg, SINK_SCALAR>(sp, k32, len, len_last, groups, out, ld, col0,
                                                                        starts, events, next_unit, stream);
        }
        if (e == cudaSuccess) {
            k_split_copy_back<<<split_block_count(h->P), 256, 0, stream>>>(src, segs[K - 1].view(), h->variant);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) st = cuda_fail(e, "split pass 1 with fix-ups");
        cudaFreeAsync(ws, stream);
        return st;
    }
    // pass 1: particular solutions (fix-up: all segments, into their columns;
    // otherwise segments 0 .. K-2, of which only the end states are needed)
    if (st == CI_OK) {
        e = fixup ? split_run(*h, sink, sp, 0, 0, (uint32_t)K, (uint32_t)K, len, len_last, out, ld, col0, nullptr,
                              stream)
                  : split_run(*h, CI_SINK_DIGEST, sp, 0, 0, (uint32_t)K - 1, (uint32_t)K, len, len_last, nullptr, 0,
                              0, res1, stream);
        if (e != cudaSuccess) st = cuda_fail(e, "split pass 1");
    }
    uint2 *starts = reinterpret_cast<uint2 *>(res1);  // K * P (slot, x) pairs, after pass 1
    if (st == CI_OK) {
        const unsigned threads = 32u * (unsigned)std::min<uint64_t>(16, K - 1);
        if (bbs)
            k_split_carry<SrcBbs><<<(unsigned)groups, threads, 0, stream>>>(sp, (uint32_t)K, len, starts, own);
        else if (b16)
            k_split_carry<SrcBbs16Seg><<<(unsigned)groups, threads, 0, stream>>>(sp, (uint32_t)K, len, starts, own);
        else
            k_split_carry<SrcXor128><<<(unsigned)groups, threads, 0, stream>>>(sp, (uint32_t)K, len, starts, own);
        if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "split carry");
    }
    if (st == CI_OK && fixup) {  // homogeneous parts into segments 1 .. K-1, then the final state
        const bool v4 = (reinterpret_cast<uintptr_t>(out) & 15u) == 0 && ld % 4 == 0 && col0 % 4 == 0;
        const int blocks = split_block_count((K - 1) * groups * 32);
        if (bbs)
            v4 ? k_split_fixup<SrcBbs, true><<<blocks, 256, 0, stream>>>(sp, starts, (uint32_t)K, len, len_last,
                                                                          groups, out, ld, col0)
               : k_split_fixup<SrcBbs, false><<<blocks, 256, 0, stream>>>(sp, starts, (uint32_t)K, len, len_last,
                                                                           groups, out, ld, col0);
        else
            v4 ? k_split_fixup<SrcBbs16Seg, true><<<blocks, 256, 0, stream>>>(sp, starts, (uint32_t)K, len, len_last,
                                                                               groups, out, ld, col0)
               : k_split_fixup<SrcBbs16Seg, false><<<blocks, 256, 0, stream>>>(sp, starts, (uint32_t)K, len,
                                                                                len_last, groups, out, ld, col0);
        if ((e = cudaGetLastError()) == cudaSuccess)
            k_split_copy_back<<<split_block_count(h->P), 256, 0, stream>>>(src, segs[K - 1].view(), h->variant);
        if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "split fix-up");
        cudaFreeAsync(ws, stream);
        return st;
    }
    if (st == CI_OK && sink == CI_SINK_QC && (e = cudaMemsetAsync(res3, 0, res_bytes, stream)) != cudaSuccess)
        st = cuda_fail(e, "clearing counts");
    if (st == CI_OK) {  // pass 2: every segment from its true start into the sink
        e = split_run(*h, sink, sp, b16 ? (int)K : -1, 0, (uint32_t)K, (uint32_t)K, len, len_last, out, ld, col0,
                      res3, stream);
        if (e != cudaSuccess) st = cuda_fail(e, "split pass 2");
    }
    if (st == CI_OK) {
        k_split_copy_back<<<split_block_count(h->P), 256, 0, stream>>>(src, segs[K - 1].view(), h->variant);
        if (!written)
            k_split_combine<<<(unsigned)((h->S + 255) / 256), 256, 0, stream>>>(res3, aux, h->P, h->S, (uint32_t)K,
                                                                                len, len_last, sink == CI_SINK_DIGEST);
        if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "split finish");
    }
    cudaFreeAsync(ws, stream);
    return st;
}

}  // namespace ci

extern "C" ci_status ci_generate_split(ci_states h, uint64_t n, int32_t sink, void *out_dev,
                                       uint64_t out_capacity, uint32_t n_segments, void *cuda_stream) {
    using namespace ci;
    if (!valid_handle(h)) return fail(CI_E_STATE, "invalid states handle");
    if (sink != CI_SINK_WRITTEN && sink != CI_SINK_QC && sink != CI_SINK_DIGEST)
        return fail(CI_E_INVAL, "unknown sink");
    if (n == 0) return CI_OK;
    if (!out_dev) return fail(CI_E_INVAL, "output is NULL");
    if (sink == CI_SINK_WRITTEN && (n > ~0ull / h->S || out_capacity < h->S * n))
        return fail(CI_E_INVAL, "out_capacity is smaller than n_streams * n");
    if (sink == CI_SINK_QC && (n & 1ull)) return fail(CI_E_INVAL, "quarter-circle sink needs an even length");
    const uint64_t K = split_segments(*h, n, n_segments);
    const cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    if (K <= 1) {  // unsplit: one launch of the tuned single-call kernel
        const cudaError_t e = sink == CI_SINK_QC       ? launch_fused_qc(*h, n, static_cast<uint64_t *>(out_dev), cs)
                              : sink == CI_SINK_DIGEST ? launch_digest(*h, n, static_cast<uint64_t *>(out_dev), cs)
                                                       : launch_generate(*h, n, static_cast<uint32_t *>(out_dev), cs);
        return check_epilogue(cs, e == cudaSuccess ? CI_OK : cuda_fail(e, "unsplit generation kernel launch"));
    }
    if (sink == CI_SINK_WRITTEN)
        return check_epilogue(cs, split_launch(*h, n, sink, static_cast<uint32_t *>(out_dev), n, 0, nullptr, K, cs));
    return check_epilogue(cs, split_launch(*h, n, sink, nullptr, n, 0, static_cast<uint64_t *>(out_dev), K, cs));
}
