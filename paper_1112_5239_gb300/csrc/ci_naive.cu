// ci_naive.cu -- the paper's naive GPU generator (include/ci_prng.h:
// ci_naive_state_bytes, ci_naive_init, ci_naive_generate): Algorithm 3, every
// stream (thread) runs Listing 1 on its own state, without exchange between
// streams.  Listing 1 XORs into the 32-bit x the low and high halves of one
// step of each of three xor-likes with 64-bit words: Marsaglia's xorshift with
// five words (output (y + y + 1) v), xor128 (four words) and xorwow (five
// words and a Weyl counter d += 362437, output d + v).
//
// Layout (P = streams rounded up to 32): fifteen uint64 fields of P lanes
// (xorshift words 0-4, xor128 words 5-8, xorwow words 9-13, d 14), then the
// uint32 field x.  One warp per 32 lanes; outputs are staged in the swizzled
// 32 x 32 shared-memory tile of the main generator and leave as row segments.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "ci_device.cuh"
#include "ci_internal.h"
#include "ci_trace.h"

namespace ci {
namespace {

using namespace dev;

#ifndef CI_NAIVE_MIN_BLOCKS
#define CI_NAIVE_MIN_BLOCKS 1  // resident blocks per SM asked of the register allocator
#endif

constexpr int kNaiveU64 = 15;
enum { N_XS = 0, N_XO = 5, N_XW = 9, N_D = 14 };

struct NaiveLane {
    uint64_t xs[5], xo[4], xw[5], d;
    uint32_t x;
    __device__ __forceinline__ void load(const uint64_t *u, const uint32_t *xf, uint64_t P, uint64_t l) {
#pragma unroll
        for (int w = 0; w < 5; ++w) xs[w] = u[(N_XS + w) * P + l];
#pragma unroll
        for (int w = 0; w < 4; ++w) xo[w] = u[(N_XO + w) * P + l];
#pragma unroll
        for (int w = 0; w < 5; ++w) xw[w] = u[(N_XW + w) * P + l];
        d = u[N_D * P + l];
        x = xf[l];
    }
    __device__ __forceinline__ void store(uint64_t *u, uint32_t *xf, uint64_t P, uint64_t l) const {
#pragma unroll
        for (int w = 0; w < 5; ++w) u[(N_XS + w) * P + l] = xs[w];
#pragma unroll
        for (int w = 0; w < 4; ++w) u[(N_XO + w) * P + l] = xo[w];
#pragma unroll
        for (int w = 0; w < 5; ++w) u[(N_XW + w) * P + l] = xw[w];
        u[N_D * P + l] = d;
        xf[l] = x;
    }
    __device__ __forceinline__ uint32_t next() {
        // xorshift, five words
        uint64_t t = xs[0] ^ (xs[0] >> 7);
        xs[0] = xs[1];
        xs[1] = xs[2];
        xs[2] = xs[3];
        xs[3] = xs[4];
        xs[4] = (xs[4] ^ (xs[4] << 6)) ^ (t ^ (t << 13));
        const uint64_t t1 = (xs[1] + xs[1] + 1ull) * xs[4];
        // xor128
        t = xo[0] ^ (xo[0] << 11);
        xo[0] = xo[1];
        xo[1] = xo[2];
        xo[2] = xo[3];
        xo[3] = (xo[3] ^ (xo[3] >> 19)) ^ (t ^ (t >> 8));
        const uint64_t t2 = xo[3];
        // xorwow
        t = xw[0] ^ (xw[0] >> 2);
        xw[0] = xw[1];
        xw[1] = xw[2];
        xw[2] = xw[3];
        xw[3] = xw[4];
        xw[4] = (xw[4] ^ (xw[4] << 4)) ^ (t ^ (t << 1));
        d += 362437ull;
        const uint64_t t3 = d + xw[4];
        // Listing 1 XORs both 32-bit halves of t1, t2 and t3 into x, which is x
        // XOR both halves of T = t1 ^ t2 ^ t3
        const uint64_t T = t1 ^ t2 ^ t3;
        x ^= (uint32_t)T ^ (uint32_t)(T >> 32);
        return x;
    }
};

struct NaiveView {
    uint64_t *u64;
    uint32_t *x;
    uint64_t P, S;
};

NaiveView naive_view(void *dev, uint64_t S) {
    NaiveView v;
    v.P = (S + 31) / 32 * 32;
    v.S = S;
    v.u64 = static_cast<uint64_t *>(dev);
    v.x = reinterpret_cast<uint32_t *>(v.u64 + kNaiveU64 * v.P);
    return v;
}

// Per-stream parameters from the counter-based splitmix64 draws of stream
// first + l (the paper draws them with ISAAC on the host): draws 0-4 xorshift,
// 5-8 xor128, 9-13 xorwow, 14 d, low half of 15 x; an all-zero word set
// becomes 1, 0, ...
__global__ void __launch_bounds__(256) k_naive_init(NaiveView v, uint64_t seed, uint64_t first) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < v.P; l += stride) {
        uint64_t k = 0, any = 0, w;
        for (int i = 0; i < 5; ++i) any |= (v.u64[(N_XS + i) * v.P + l] = lane_draw(seed, first + l, k++));
        if (!any) v.u64[N_XS * v.P + l] = 1;
        any = 0;
        for (int i = 0; i < 4; ++i) any |= (v.u64[(N_XO + i) * v.P + l] = lane_draw(seed, first + l, k++));
        if (!any) v.u64[N_XO * v.P + l] = 1;
        any = 0;
        for (int i = 0; i < 5; ++i) any |= (v.u64[(N_XW + i) * v.P + l] = lane_draw(seed, first + l, k++));
        if (!any) v.u64[N_XW * v.P + l] = 1;
        v.u64[N_D * v.P + l] = lane_draw(seed, first + l, k++);
        w = lane_draw(seed, first + l, k++);
        v.x[l] = (uint32_t)w;
    }
}

// One warp per 32 lanes; rows r < S of out (row stride n) receive the outputs.
template <bool V4>
__global__ void __launch_bounds__(256, CI_NAIVE_MIN_BLOCKS) k_naive_generate(NaiveView v, uint64_t n, uint32_t *out) {
    __shared__ uint4 tiles[8][256];
    const int lane = threadIdx.x & 31;
    uint4 *tile = tiles[threadIdx.x >> 5];
    uint32_t *tw = reinterpret_cast<uint32_t *>(tile);
    const uint64_t groups = v.P / 32;
    const uint64_t wstride = (uint64_t)gridDim.x * 8;
    // warp w of block b starts at group w * gridDim.x + b: a partial last
    // round of warps is spread over every block (and SM)
    for (uint64_t g = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; g < groups; g += wstride) {
        const uint64_t l = g * 32 + lane, row0 = g * 32;
        NaiveLane L;
        L.load(v.u64, v.x, v.P, l);
        const uint64_t nfull = n - n % 32;
        for (uint64_t i0 = 0; i0 < nfull; i0 += 32) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint4 o;
                o.x = L.next();
                o.y = L.next();
                o.z = L.next();
                o.w = L.next();
                tile[lane * 8 + (q ^ (lane & 7))] = o;
            }
            __syncwarp();
            if (V4) {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int r = 4 * k + lane / 8, c = lane % 8;
                    if (row0 + r < v.S) store16<0>(out + (row0 + r) * n + i0 + 4 * c, tile[r * 8 + (c ^ (r & 7))]);
                }
            } else {
                for (int r = 0; r < 32; ++r)
                    if (row0 + r < v.S) store4<0>(out + (row0 + r) * n + i0 + lane, tw[tile_word<32>(r, lane)]);
            }
            __syncwarp();
        }
        const int rem = (int)(n - nfull);
        if (rem) {
            for (int k = 0; k < rem; ++k) tw[tile_word<32>(lane, k)] = L.next();
            __syncwarp();
            for (int r = 0; r < 32; ++r)
                if (lane < rem && row0 + r < v.S) out[(row0 + r) * n + nfull + lane] = tw[tile_word<32>(r, lane)];
            __syncwarp();
        }
        L.store(v.u64, v.x, v.P, l);
    }
}

template <bool V4>
int naive_grid(uint64_t groups) {
    static int per_sm = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_naive_generate<V4>, 256, 0);
        if (per_sm <= 0) per_sm = 1;
    });
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(groups, (uint64_t)sm_count() * per_sm));  // a block per group at most
}

}  // namespace
}  // namespace ci

extern "C" {

ci_status ci_naive_state_bytes(uint64_t n_streams, uint64_t *bytes) {
    using namespace ci;
    if (!bytes) return fail(CI_E_INVAL, "bytes is NULL");
    if (n_streams == 0 || n_streams > (1ull << 32)) return fail(CI_E_INVAL, "n_streams must be in [1, 2^32]");
    const uint64_t P = (n_streams + 31) / 32 * 32;
    *bytes = (8ull * kNaiveU64 + 4ull) * P;
    return CI_OK;
}

ci_status ci_naive_init(uint64_t n_streams, uint64_t seed, uint64_t first_stream, void *state_dev,
                        uint64_t state_bytes, void *cuda_stream) {
    using namespace ci;
    uint64_t need = 0;
    const ci_status st = ci_naive_state_bytes(n_streams, &need);
    if (st != CI_OK) return st;
    if (!state_dev || state_bytes < need) return fail(CI_E_INVAL, "state buffer NULL or smaller than ci_naive_state_bytes");
    if ((reinterpret_cast<uintptr_t>(state_dev) & 7u) != 0) return fail(CI_E_INVAL, "state buffer not 8-byte aligned");
    if (first_stream >= (1ull << 32) || n_streams > (1ull << 32) - first_stream)
        return fail(CI_E_INVAL, "first_stream + n_streams exceeds 2^32");
    const NaiveView v = naive_view(state_dev, n_streams);
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((v.P + 255) / 256, (uint64_t)sm_count() * 8));
    k_naive_init<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(v, seed, first_stream);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CI_OK : cuda_fail(e, "ci_naive_init launch");
}

ci_status ci_naive_generate(void *state_dev, uint64_t n_streams, uint64_t n_per_stream, uint32_t *out_dev,
                            uint64_t out_capacity_u32, void *cuda_stream) {
    ci::TraceRange trace("naive generate");
    using namespace ci;
    uint64_t need = 0;
    const ci_status st = ci_naive_state_bytes(n_streams, &need);
    if (st != CI_OK) return st;
    if (!state_dev) return fail(CI_E_INVAL, "state buffer is NULL");
    if ((reinterpret_cast<uintptr_t>(state_dev) & 7u) != 0) return fail(CI_E_INVAL, "state buffer not 8-byte aligned");
    if (n_per_stream == 0) return CI_OK;
    if (!out_dev) return fail(CI_E_INVAL, "output is NULL");
    if (n_per_stream > ~0ull / n_streams || out_capacity_u32 < n_streams * n_per_stream)
        return fail(CI_E_INVAL, "out_capacity_u32 is smaller than n_streams * n_per_stream");
    const NaiveView v = naive_view(state_dev, n_streams);
    const uint64_t groups = v.P / 32;
    const bool v4 = (reinterpret_cast<uintptr_t>(out_dev) & 15u) == 0 && n_per_stream % 4 == 0;
    if (v4)
        k_naive_generate<true><<<naive_grid<true>(groups), 256, 0, (cudaStream_t)cuda_stream>>>(v, n_per_stream, out_dev);
    else
        k_naive_generate<false><<<naive_grid<false>(groups), 256, 0, (cudaStream_t)cuda_stream>>>(v, n_per_stream,
                                                                                                   out_dev);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CI_OK : cuda_fail(e, "ci_naive_generate launch");
}

}  // extern "C"
