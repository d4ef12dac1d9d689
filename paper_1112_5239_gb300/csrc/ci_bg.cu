// ci_bg.cu -- the chaotic Blum-Goldwasser cryptosystem of Sec. 9.2 on the
// device (include/ci_prng.h: ci_bg_encrypt, ci_bg_decrypt).
//
// Per message: x_0 = r^2 mod N, b_i = the w low bits of x_i
// (w = floor(log2 floor(log2 N))), x_{i+1} = x_i^2 mod N.  The keystream is
// Eq. (Oplus) run on the b_i from S^0: k_i = S^0 ^ b_0 ^ ... ^ b_i, and
// chunk i of the ciphertext is c_i = m_i ^ k_i; the ciphertext carries
// y = x_L.  Decryption recovers x_0 from y with the factors p, q = 3 mod 4
// (square roots by the exponent ((p + 1) / 4)^L, joined by Garner's CRT) and
// regenerates the same keystream.
//
// One lane owns one message; a warp owns 32 consecutive messages.  When the
// chunk count is a multiple of 32 and both buffers are 16-byte aligned, each
// lane moves its own 32 chunks per step with two 16-byte loads and stores.
// Otherwise the warp moves its messages' chunks (one byte each,
// message-major) through a warp-private 32 x 32 byte tile in shared memory,
// so global loads and stores are 32-byte rows while each lane walks its own
// row.  The squarings use the Barrett reduction of the BBS strategy source
// (modulus odd, below 2^62), which keeps x_i canonical so its low bits are
// read directly; a warp whose moduli all have at least 34 bits takes its
// limb form.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ci_device.cuh"
#include "ci_internal.h"
#include "ci_trace.h"
#include "ci_modarith.cuh"

namespace ci {
namespace {

using namespace dev;

#ifndef CI_BG_MIN_BLOCKS
#define CI_BG_MIN_BLOCKS 6  // resident blocks per SM asked of the register allocator: 40 registers,
                            // no spills (measured: 6 and 8 equal, 4 slower for decryption)
#endif

constexpr int kBgWarps = 8;    // warps per block
constexpr int kBgTile = 32;    // chunks per staged row
constexpr int kBgRowPad = 36;  // bytes per staged row: 9 words, so the 32 lanes'
                               // word reads of their own rows hit 32 banks

__device__ __forceinline__ uint32_t bg_w(uint64_t N) {
    const uint32_t lg = 63u - (uint32_t)__clzll((long long)N);  // floor(log2 N), N >= 2
    return lg ? 31u - (uint32_t)__clz((int)lg) : 0u;             // floor(log2 lg)
}

// One chunk: b = x_i & mask (x_i canonical), key ^= b, x_{i+1} = x_i^2.
// kLimb: the limb-form square (every modulus of the warp has 34..62 bits).
struct BgLane {
    Barrett62 B;
    uint64_t x;
    uint32_t mask, key;
    template <bool kLimb>
    __device__ __forceinline__ uint64_t sqr(uint64_t v) const {
        return kLimb ? B.sqr_limb(v) : B.sqr(v);
    }
    template <bool kLimb>
    __device__ __forceinline__ uint32_t chunk(uint32_t v) {
        key ^= (uint32_t)x & mask;
        x = sqr<kLimb>(x);
        return (v ^ key) & 0xFFu;
    }
    // Four chunks, one per byte of w: the keystream bytes are gathered into
    // one word and XORed in once (key < 2^8: S^0 is a byte, the b_i have at
    // most 5 bits).
    template <bool kLimb>
    __device__ __forceinline__ uint32_t word(uint32_t w) {
        uint32_t ks = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            key ^= (uint32_t)x & mask;
            x = sqr<kLimb>(x);
            ks |= key << (8 * b);
        }
        return w ^ ks;
    }
};

// Encryption key check: N odd, 3 <= N < 2^62 (the range of Barrett62).
__device__ __forceinline__ bool bg_setup_encrypt(uint64_t N, uint64_t r, BgLane &s) {
    const bool ok = (N & 1ull) && N >= 3 && N < (1ull << 62);
    if (!ok) N = 3;
    s.B.set(N, barrett_mu(N));
    s.x = s.B.sqr(r % N);  // x_0 = r^2 mod N
    return ok;
}

// Decryption key check: p != q, both prime, = 3 mod 4, below 2^32, p q < 2^62.
// x_0 = the square root of y taken L times mod p and mod q, joined by
// Garner's formula x_0 = r_p + p ((r_q - r_p) p^-1 mod q).
__device__ __forceinline__ bool bg_setup_decrypt(uint64_t p, uint64_t q, uint64_t y, uint64_t L, BgLane &s) {
    const bool ok = p < (1ull << 32) && q < (1ull << 32) && (p & 3ull) == 3 && (q & 3ull) == 3 && p != q &&
                    p * q < (1ull << 62) && is_prime_u32(p) && is_prime_u32(q);
    uint64_t x0 = 0, N = 3;
    if (ok) {
        const Barrett32 Bp1(p - 1), Bq1(q - 1);      // even moduli: Barrett
        const Mont32 Mp((uint32_t)p), Mq((uint32_t)q);  // odd primes: Montgomery
        const uint64_t ep = Bp1.pow((p + 1) / 4, L);  // ((p+1)/4)^L mod (p-1)
        const uint64_t eq = Bq1.pow((q + 1) / 4, L);
        // y mod N < p q, below p 2^32 and q 2^32: taken to Montgomery form by REDC
        const uint64_t yN = y < p * q ? y : y % (p * q);
        const uint32_t rp = Mp.from(Mp.pow_m(Mp.to_wide(yN), ep));
        const uint32_t rq_m = Mq.pow_m(Mq.to_wide(yN), eq);  // Montgomery forms mod q from here
        const uint32_t pinv_m = Mq.pow_m(Mq.to_any((uint32_t)p), q - 2);  // Fermat: p^(q-2) = p^-1 mod q
        const uint32_t rp_m = Mq.to_any(rp);
        const uint32_t diff_m = rq_m >= rp_m ? rq_m - rp_m : (uint32_t)((uint64_t)rq_m + q - rp_m);
        const uint64_t t = Mq.from(Mq.mul(diff_m, pinv_m));  // (r_q - r_p) p^-1 mod q
        x0 = rp + p * t;                              // < p + p (q - 1) = N
        N = p * q;
    }
    s.B.set(N, barrett_mu(N));
    s.x = x0;
    return ok;
}

// The chunks of one warp's 32 messages (lane = message), after key setup.
template <bool kVec, bool kLimb>
__device__ __forceinline__ void bg_rows(BgLane &s, uint32_t keep, bool live, uint64_t msg, uint64_t m0,
                                        uint32_t rows, uint64_t L, const uint8_t *in, uint8_t *out, uint8_t *tile,
                                        uint8_t *row, uint32_t lane) {
    if constexpr (kVec) {  // L a multiple of 32, rows 16-byte aligned
        if (live) {
            const uint4 *src = reinterpret_cast<const uint4 *>(in + msg * L);
            uint4 *dst = reinterpret_cast<uint4 *>(out + msg * L);
            const uint64_t steps = L / kBgTile;
            for (uint64_t t = 0; t < steps; ++t) {  // each step reads its 32 bytes before writing them
                uint4 a = src[2 * t], b = src[2 * t + 1];
                a.x = s.word<kLimb>(a.x) & keep;
                a.y = s.word<kLimb>(a.y) & keep;
                a.z = s.word<kLimb>(a.z) & keep;
                a.w = s.word<kLimb>(a.w) & keep;
                b.x = s.word<kLimb>(b.x) & keep;
                b.y = s.word<kLimb>(b.y) & keep;
                b.z = s.word<kLimb>(b.z) & keep;
                b.w = s.word<kLimb>(b.w) & keep;
                dst[2 * t] = a;
                dst[2 * t + 1] = b;
            }
        }
    } else {
        for (uint64_t k0 = 0; k0 < L; k0 += kBgTile) {
            const uint32_t width = L - k0 < (uint64_t)kBgTile ? (uint32_t)(L - k0) : (uint32_t)kBgTile;
            __syncwarp();
#pragma unroll 8
            for (uint32_t r = 0; r < rows; ++r)
                if (lane < width) tile[r * kBgRowPad + lane] = in[(m0 + r) * L + k0 + lane];
            __syncwarp();
            if (live) {
                uint32_t *w = reinterpret_cast<uint32_t *>(row);
                if (width == kBgTile) {
#pragma unroll
                    for (int j = 0; j < kBgTile / 4; ++j) w[j] = s.word<kLimb>(w[j]) & keep;
                } else {
                    for (uint32_t j = 0; j < width; ++j) row[j] = (uint8_t)(s.chunk<kLimb>(row[j]) & keep);
                }
            }
            __syncwarp();
#pragma unroll 8
            for (uint32_t r = 0; r < rows; ++r)
                if (lane < width) out[(m0 + r) * L + k0 + lane] = tile[r * kBgRowPad + lane];
        }
    }
}

template <bool kDecrypt, bool kVec>
__global__ void __launch_bounds__(kBgWarps * 32, CI_BG_MIN_BLOCKS)
    k_bg(uint64_t n_msgs, uint64_t L, const uint64_t *__restrict__ key_a, const uint64_t *__restrict__ key_b,
         const uint8_t *__restrict__ S0, const uint64_t *__restrict__ y_in, const uint8_t *in, uint8_t *out,
         uint64_t *__restrict__ y_out, uint32_t *__restrict__ n_rejected) {
    __shared__ __align__(16) uint8_t stage[kBgWarps][32 * kBgRowPad];
    const uint32_t lane = threadIdx.x & 31u;
    uint8_t *tile = stage[threadIdx.x >> 5];
    uint8_t *row = tile + lane * kBgRowPad;
    const uint64_t n_groups = (n_msgs + 31) / 32;
    const uint64_t stride = (uint64_t)gridDim.x * kBgWarps;
    // warp w of block b starts at group w * gridDim.x + b, so a partial last
    // round of warps is spread over every block (and SM)
    for (uint64_t g = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; g < n_groups; g += stride) {
        const uint64_t m0 = g * 32;
        const uint64_t msg = m0 + lane;
        const bool live = msg < n_msgs;
        const uint32_t rows = n_msgs - m0 < 32 ? (uint32_t)(n_msgs - m0) : 32u;
        BgLane s;
        bool ok = false;
        if (live) {
            ok = kDecrypt ? bg_setup_decrypt(key_a[msg], key_b[msg], y_in[msg], L, s)
                          : bg_setup_encrypt(key_a[msg], key_b[msg], s);
            s.mask = ok ? (1u << bg_w(s.B.M)) - 1u : 0u;
            s.key = S0[msg];
            if (!ok && n_rejected) atomicAdd(n_rejected, 1u);
        }
        const uint32_t keep = ok ? 0xFFFFFFFFu : 0u;  // a rejected key's row is written as zeros
        // the same in every lane: the branch never diverges
        if (__all_sync(0xFFFFFFFFu, !live || s.B.M >= (1ull << 33)))
            bg_rows<kVec, true>(s, keep, live, msg, m0, rows, L, in, out, tile, row, lane);
        else
            bg_rows<kVec, false>(s, keep, live, msg, m0, rows, L, in, out, tile, row, lane);
        if (!kDecrypt && live) y_out[msg] = ok ? s.x : 0ull;
    }
}

template <bool kDecrypt, bool kVec>
int bg_grid(uint64_t n_msgs) {
    static int per_sm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bg<kDecrypt, kVec>, kBgWarps * 32, 0);
        if (per_sm <= 0) per_sm = 1;
    });
    const uint64_t blocks = (n_msgs + 31) / 32;  // a block per warp group at most
    return (int)std::min<uint64_t>(blocks, (uint64_t)sm_count() * per_sm);
}

ci_status bg_check(uint64_t n_msgs, uint64_t n_chunks, const void *a, const void *b, const void *S0,
                   const void *y, const void *in, const void *out) {
    if (!a || !b || !S0 || !y) return fail(CI_E_INVAL, "bg: key, S0 and y arrays must be non-null");
    if (n_chunks && (!in || !out)) return fail(CI_E_INVAL, "bg: message and ciphertext must be non-null");
    if (n_chunks > ~0ull / n_msgs) return fail(CI_E_INVAL, "bg: n_msgs * n_chunks overflows");
    return CI_OK;
}

// The per-lane 16-byte path: whole 32-chunk steps and 16-byte aligned rows.
bool bg_vec(uint64_t n_chunks, const void *in, const void *out) {
    return n_chunks % kBgTile == 0 && (reinterpret_cast<uintptr_t>(in) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
}

template <bool kDecrypt>
cudaError_t bg_launch(uint64_t n_msgs, uint64_t L, const uint64_t *a, const uint64_t *b, const uint8_t *S0,
                      const uint64_t *y_in, const uint8_t *in, uint8_t *out, uint64_t *y_out, uint32_t *n_rejected,
                      cudaStream_t stream) {
    if (bg_vec(L, in, out))
        k_bg<kDecrypt, true><<<bg_grid<kDecrypt, true>(n_msgs), kBgWarps * 32, 0, stream>>>(
            n_msgs, L, a, b, S0, y_in, in, out, y_out, n_rejected);
    else
        k_bg<kDecrypt, false><<<bg_grid<kDecrypt, false>(n_msgs), kBgWarps * 32, 0, stream>>>(
            n_msgs, L, a, b, S0, y_in, in, out, y_out, n_rejected);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ci

extern "C" {

ci_status ci_bg_encrypt(uint64_t n_msgs, uint64_t n_chunks, const uint64_t *N_dev, const uint8_t *S0_dev,
                        const uint64_t *r_dev, const uint8_t *msg_dev, uint8_t *cipher_dev, uint64_t *y_dev,
                        uint32_t *n_rejected_dev, void *cuda_stream) {
    ci::TraceRange trace("bg encrypt");
    using namespace ci;
    if (n_msgs == 0) return CI_OK;
    const ci_status st = bg_check(n_msgs, n_chunks, N_dev, r_dev, S0_dev, y_dev, msg_dev, cipher_dev);
    if (st != CI_OK) return st;
    const cudaError_t e = bg_launch<false>(n_msgs, n_chunks, N_dev, r_dev, S0_dev, nullptr, msg_dev, cipher_dev, y_dev,
                                           n_rejected_dev, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? CI_OK : cuda_fail(e, "ci_bg_encrypt launch");
}

ci_status ci_bg_decrypt(uint64_t n_msgs, uint64_t n_chunks, const uint64_t *p_dev, const uint64_t *q_dev,
                        const uint8_t *S0_dev, const uint64_t *y_dev, const uint8_t *cipher_dev, uint8_t *msg_dev,
                        uint32_t *n_rejected_dev, void *cuda_stream) {
    ci::TraceRange trace("bg decrypt");
    using namespace ci;
    if (n_msgs == 0 || n_chunks == 0) return CI_OK;
    const ci_status st = bg_check(n_msgs, n_chunks, p_dev, q_dev, S0_dev, y_dev, cipher_dev, msg_dev);
    if (st != CI_OK) return st;
    const cudaError_t e = bg_launch<true>(n_msgs, n_chunks, p_dev, q_dev, S0_dev, y_dev, cipher_dev, msg_dev, nullptr,
                                          n_rejected_dev, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? CI_OK : cuda_fail(e, "ci_bg_decrypt launch");
}

}  // extern "C"
