// ci_kernels.cu -- seeding and generation kernels of the chaotic-iterations
// PRNG (Algorithms 4 and 5 of the paper with Eq. (Oplus)), and their host
// launchers.
//
// The generation kernels themselves are in ci_gen.cuh (instantiated per
// source in ci_gen_*.cu); this file holds seeding and the launch entry points,
// which apply the autotuned launch shape.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "ci_device.cuh"
#include "ci_gen.cuh"
#include "ci_modarith.cuh"
#include "ci_tune.h"

namespace ci {

using namespace dev;

constexpr int kWarpsPerBlock = 8;
constexpr int kBlockThreads = kWarpsPerBlock * 32;

// ------------------------------------------------------------- seeding
// The partner table travels as a kernel parameter (no host-to-device copy
// from pageable memory, which would synchronise the caller's stream).
struct TableParam {
    uint32_t w[kTableBytes / 4];
};

__device__ __forceinline__ void write_table(const DevState &st, const TableParam &tp) {
    if (blockIdx.x == 0 && threadIdx.x < kTableBytes / 4)
        reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(st.table))[threadIdx.x] = tp.w[threadIdx.x];
}

__device__ __forceinline__ void init_xor_lane(const DevState &st, uint64_t seed, uint64_t first, int xl,
                                              uint64_t l) {
    const uint64_t d0 = lane_draw(seed, first + l, 0);
    const uint64_t d1 = lane_draw(seed, first + l, 1);
    const uint64_t d2 = lane_draw(seed, first + l, 2);
    uint32_t a, b = 0, c = 0, d = 0;
    if (xl == CI_XL_XOR128) {
        a = (uint32_t)d0;
        b = (uint32_t)(d0 >> 32);
        c = (uint32_t)d1;
        d = (uint32_t)(d1 >> 32);
        if ((a | b | c | d) == 0u) a = 1u;
    } else if (xl == CI_XL_XOR64) {
        a = (uint32_t)d0;
        b = (uint32_t)(d0 >> 32);
        if ((a | b) == 0u) a = 1u;
    } else {
        a = (uint32_t)d0;
        if (a == 0u) a = 1u;
    }
    st.u32[F_A * st.P + l] = a;
    st.u32[F_B * st.P + l] = b;
    st.u32[F_C * st.P + l] = c;
    st.u32[F_D * st.P + l] = d;
    st.u32[F_X * st.P + l] = (uint32_t)d2;
    st.u32[F_SLOT * st.P + l] = (uint32_t)(d2 >> 32);
    st.u32[F_SEL * st.P + l] = 0u;
    st.u32[F_P * st.P + l] = 0u;
    st.u32[F_Q * st.P + l] = 0u;
}

__global__ void __launch_bounds__(256) k_init_xor(DevState st, TableParam tp, uint64_t seed, uint64_t first, int xl) {
    write_table(st, tp);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < st.P; l += stride)
        init_xor_lane(st, seed, first, xl, l);
}

// Blum prime candidate from a draw: 2^30 + (d >> 34), forced to 3 mod 4.
__device__ __forceinline__ uint32_t blum_candidate(uint64_t d) {
    return (uint32_t)((1ull << 30) + (d >> 34)) | 3u;
}

__device__ void init_bbs_lane(const DevState &st, uint64_t seed, uint64_t first, uint64_t l) {
    uint64_t k = 0, d;
    uint32_t p, q;
    do {
        d = lane_draw(seed, first + l, k++);
        p = blum_candidate(d);
    } while (!is_prime_u32(p));
    do {
        d = lane_draw(seed, first + l, k++);
        q = blum_candidate(d);
    } while (q == p || !is_prime_u32(q));
    const uint64_t M = (uint64_t)p * q;
    uint64_t v;
    do {
        d = lane_draw(seed, first + l, k++);
        v = 2ull + d % (M - 2ull);
    } while (v % p == 0ull || v % q == 0ull);  // gcd(v, p q) = 1
    d = lane_draw(seed, first + l, k++);
    for (int f = F_A; f <= F_D; ++f) st.u32[f * st.P + l] = 0u;
    st.u32[F_X * st.P + l] = (uint32_t)d;
    st.u32[F_SLOT * st.P + l] = (uint32_t)(d >> 32);
    st.u32[F_SEL * st.P + l] = (uint32_t)(v & 7u) | ((uint32_t)((v >> 3) & 7u) << 8);
    st.u32[F_P * st.P + l] = p;
    st.u32[F_Q * st.P + l] = q;
    st.u64[G_Y * st.P + l] = v;
    st.u64[G_M * st.P + l] = M;
    st.u64[G_MU * st.P + l] = barrett_mu(M);
}

__global__ void __launch_bounds__(256) k_init_bbs(DevState st, TableParam tp, uint64_t seed, uint64_t first) {
    write_table(st, tp);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < st.P; l += stride)
        init_bbs_lane(st, seed, first, l);
}

// Algorithm 5 as printed: eight generators per lane, Blum primes p != q from
// candidates (128 + draw mod 128) | 3 (odd, < 256: prime iff no divisor in
// 3..13), a seed coprime to M, then x and the slot.
__device__ __forceinline__ bool is_prime_below_256(uint32_t c) {  // c odd, >= 131
    return c % 3u && c % 5u && c % 7u && c % 11u && c % 13u;
}

__device__ void init_bbs16_lane(const DevState &st, uint64_t seed, uint64_t first, uint64_t l) {
    uint64_t k = 0, d;
    for (int g = 0; g < 8; ++g) {
        uint32_t p, q;
        do {
            d = lane_draw(seed, first + l, k++);
            p = (uint32_t)(128u + d % 128u) | 3u;
        } while (!is_prime_below_256(p));
        do {
            d = lane_draw(seed, first + l, k++);
            q = (uint32_t)(128u + d % 128u) | 3u;
        } while (q == p || !is_prime_below_256(q));
        const uint32_t M = p * q;
        uint32_t v;
        do {
            d = lane_draw(seed, first + l, k++);
            v = 2u + (uint32_t)(d % (uint64_t)(M - 2u));
        } while (v % p == 0u || v % q == 0u);
        st.u32[(F_Y16 + g) * st.P + l] = v;
        st.u32[(F_M16 + g) * st.P + l] = M;
    }
    d = lane_draw(seed, first + l, k++);
    for (int f = F_A; f <= F_D; ++f) st.u32[f * st.P + l] = 0u;
    st.u32[F_X * st.P + l] = (uint32_t)d;
    st.u32[F_SLOT * st.P + l] = (uint32_t)(d >> 32);
    st.u32[F_SEL * st.P + l] = 0u;
    st.u32[F_P * st.P + l] = 0u;
    st.u32[F_Q * st.P + l] = 0u;
}

__global__ void __launch_bounds__(256) k_init_bbs16(DevState st, TableParam tp, uint64_t seed, uint64_t first) {
    write_table(st, tp);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < st.P; l += stride)
        init_bbs16_lane(st, seed, first, l);
}

// Seeding of many states in one launch: thread g takes global lane g, finds
// its task (largest lane prefix <= g) and seeds that lane; the first lanes of
// each task also write its partner table.
__global__ void __launch_bounds__(256) k_init_batched(const InitTask *tasks, uint32_t n_tasks, uint64_t total) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
        uint32_t lo = 0, hi = n_tasks;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (tasks[mid].prefix <= g)
                lo = mid;
            else
                hi = mid;
        }
        const InitTask &T = tasks[lo];
        const uint64_t l = g - T.prefix;
        for (uint64_t w = l; w < kTableBytes / 4; w += T.st.P)
            reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(T.st.table))[w] = T.table[w];
        if (T.variant == CI_VAR_BBS)
            init_bbs_lane(T.st, T.seed, T.first, l);
        else if (T.variant == CI_VAR_BBS16)
            init_bbs16_lane(T.st, T.seed, T.first, l);
        else
            init_xor_lane(T.st, T.seed, T.first, T.xl, l);
    }
}

cudaError_t launch_init_batched(const InitTask *dev_tasks, uint32_t n_tasks, uint64_t total_lanes,
                                cudaStream_t stream) {
    if (n_tasks == 0 || total_lanes == 0) return cudaSuccess;
    const uint64_t blocks = (total_lanes + kBlockThreads - 1) / kBlockThreads;
    const unsigned grid = (unsigned)(blocks < 65535 ? blocks : 65535);
    k_init_batched<<<grid, kBlockThreads, 0, stream>>>(dev_tasks, n_tasks, total_lanes);
    return cudaGetLastError();
}

// ------------------------------------------------------------ launchers
// SM count of the current device, looked up once per device: one process may
// drive GPUs of different models.
int sm_count() {
    constexpr int kMaxDevices = 64;
    static std::atomic<int> counts[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    const bool cached = dev >= 0 && dev < kMaxDevices;
    if (cached) {
        const int c = counts[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int count = 0;
    if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || count <= 0) count = 1;
    if (cached) counts[dev].store(count, std::memory_order_relaxed);
    return count;
}

cudaError_t launch_init(const ci_states_s &h, uint64_t seed, uint64_t first, cudaStream_t stream) {
    const DevState st = h.view();
    const uint64_t blocks = (h.P + kBlockThreads - 1) / kBlockThreads;
    const unsigned grid = (unsigned)(blocks < 65535 ? blocks : 65535);
    TableParam tp;
    std::memcpy(tp.w, h.table, kTableBytes);
    if (h.variant == CI_VAR_BBS)
        k_init_bbs<<<grid, kBlockThreads, 0, stream>>>(st, tp, seed, first);
    else if (h.variant == CI_VAR_BBS16)
        k_init_bbs16<<<grid, kBlockThreads, 0, stream>>>(st, tp, seed, first);
    else
        k_init_xor<<<grid, kBlockThreads, 0, stream>>>(st, tp, seed, first, h.xl);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's entry-point lookup, so the
// library does not link libcuda itself.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool make_out_tensor_map(CUtensorMap *map, uint32_t *out, uint64_t rows, uint64_t cols) {
    // TMA: base 16-byte aligned, row stride a multiple of 16 bytes (cols % 4),
    // int32 coordinates; box 32 x 32 words, 128-byte swizzle
    if ((reinterpret_cast<uintptr_t>(out) & 15u) || cols % 4 || cols < 32 || rows == 0 || cols >= (1ull << 31) ||
        rows >= (1ull << 31))
        return false;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 4ull};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t elem[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, out, dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

cudaError_t launch_with(const ci_states_s &h, int sink, const TuneChoice &c, uint64_t n, uint32_t *out,
                        uint64_t *counts, cudaStream_t stream) {
    const DevState st = h.view();
    if (h.variant == CI_VAR_BBS) return gen_bbs(sink, c, st, n, out, counts, stream);
    if (h.variant == CI_VAR_BBS16) return gen_bbs16(sink, c, st, n, out, counts, stream);
    if (h.xl == CI_XL_XORSHIFT32) return gen_xs32(sink, c, st, n, out, counts, stream);
    if (h.xl == CI_XL_XOR64) return gen_xor64(sink, c, st, n, out, counts, stream);
    return gen_xor128(sink, c, st, n, out, counts, stream);
}

static int src_kind(const ci_states_s &h) {
    if (h.variant == CI_VAR_BBS16) return SK_BBS16;
    if (h.variant == CI_VAR_BBS) return SK_BBS;
    return h.xl == CI_XL_XORSHIFT32 ? SK_XS32 : h.xl == CI_XL_XOR64 ? SK_XOR64 : SK_XOR128;
}

cudaError_t launch_generate(const ci_states_s &h, uint64_t n, uint32_t *out, cudaStream_t stream) {
    const bool v4 = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) && (n % 4 == 0);
    const int sink = v4 ? SINK_V4 : SINK_SCALAR;
    return launch_with(h, sink, tuned(src_kind(h), sink), n, out, nullptr, stream);
}

cudaError_t launch_fused_qc(const ci_states_s &h, uint64_t n, uint64_t *counts, cudaStream_t stream) {
    return launch_with(h, SINK_QC, tuned(src_kind(h), SINK_QC), n, nullptr, counts, stream);
}

cudaError_t launch_digest(const ci_states_s &h, uint64_t n, uint64_t *digest, cudaStream_t stream) {
    return launch_with(h, SINK_DIGEST, tuned(src_kind(h), SINK_DIGEST), n, nullptr, digest, stream);
}

}  // namespace ci
