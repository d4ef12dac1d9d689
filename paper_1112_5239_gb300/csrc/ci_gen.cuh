// ci_gen.cuh -- the generation kernel template and its launch-shape
// dispatch, instantiated per strategy source in ci_gen_<source>.cu so the
// instantiations compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "ci_device.cuh"
#include "ci_tune.h"

namespace ci {

// One warp per group of 32 lanes, W warps per block, a persistent grid whose
// warps stride over the warp groups; written sinks stage a 32 x KT tile per
// warp in dynamic shared memory.  Warp w of block b starts at group
// w * gridDim.x + b: with fewer groups than resident warps, the idle warps are
// spread over all blocks (hence all SMs) instead of leaving whole blocks idle.
template <class Src, int SINK, int W, class TC>
__global__ void __launch_bounds__(W * 32) k_generate(DevState st, uint64_t n, uint32_t *out, uint64_t *counts) {
    extern __shared__ uint4 dyn_tiles[];
    const int w = threadIdx.x >> 5;
    uint4 *tile = dyn_tiles + (SINK >= dev::SINK_QC ? 0 : w * TC::KT * 8);
    const uint64_t ngroups = st.P / 32;
    const uint64_t gstride = (uint64_t)gridDim.x * W;
    for (uint64_t g = (uint64_t)w * gridDim.x + blockIdx.x; g < ngroups; g += gstride)
        dev::warp_task<Src, SINK, TC>(st, g, n, out, n, 0, counts, tile);
}

// Written sink through TMA bulk tensor stores (xor sources, store policy 2).
template <class Src, int W>
__global__ void __launch_bounds__(W * 32) k_generate_tma(DevState st, uint64_t n, uint32_t *out,
                                                         const __grid_constant__ CUtensorMap map) {
    extern __shared__ uint4 tma_tiles[];
    // the 128-byte swizzle needs 1024-byte aligned tiles: round the base up
    // (the launch allocates 1 KB of slack)
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tma_tiles);
    uint4 *base = reinterpret_cast<uint4 *>(reinterpret_cast<char *>(tma_tiles) + ((1024u - (sbase & 1023u)) & 1023u));
    const int w = threadIdx.x >> 5;
    uint4 *tiles = base + w * 512;  // two 4 KB tiles per warp
    const uint64_t ngroups = st.P / 32;
    const uint64_t gstride = (uint64_t)gridDim.x * W;
    for (uint64_t g = (uint64_t)w * gridDim.x + blockIdx.x; g < ngroups; g += gstride)  // as in k_generate
        dev::warp_task_tma<Src>(st, g, n, &map, out, n, 0, tiles);
    if ((threadIdx.x & 31) == 0) dev::tma_wait_all();  // every store complete before the block exits
    __syncwarp();
}

// Tensor map over out[rows][cols] (uint32, row stride cols words) with a
// 32 x 32 box and the 128-byte swizzle; false when TMA cannot be used (then
// the caller takes the 16-byte-store path).
bool make_out_tensor_map(CUtensorMap *map, uint32_t *out, uint64_t rows, uint64_t cols);

template <class Src, int W>
static cudaError_t launch_gen_tma(const DevState &st, uint64_t n, uint32_t *out, cudaStream_t stream, bool *used) {
    *used = false;
    CUtensorMap map;
    if (!make_out_tensor_map(&map, out, st.S, n)) return cudaSuccess;
    auto kern = k_generate_tma<Src, W>;
    const size_t smem = (size_t)W * 2 * 4096 + 1024;  // + slack for the 1024-byte alignment of the base
    static std::once_flag once;
    static int per_sm = 1;
    std::call_once(once, [&] {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int ps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kern, W * 32, smem) == cudaSuccess && ps > 0)
            per_sm = ps;
    });
    const uint64_t cap = (uint64_t)sm_count() * per_sm;
    const uint64_t need = st.P / 32;  // a block per group at most (the warps spread over the blocks)
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    *used = true;
    if (grid == 0) return cudaSuccess;
    kern<<<grid, W * 32, smem, stream>>>(st, n, out, map);
    return cudaGetLastError();
}

template <class Src, int SINK, int W, class TC>
static cudaError_t launch_gen_t(const DevState &st, uint64_t n, uint32_t *out, uint64_t *counts,
                                cudaStream_t stream) {
    auto kern = k_generate<Src, SINK, W, TC>;
    const size_t smem = SINK >= dev::SINK_QC ? 0 : (size_t)W * TC::KT * 8 * sizeof(uint4);
    static std::once_flag once;
    static int per_sm = 1;
    std::call_once(once, [&] {
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int ps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kern, W * 32, smem) == cudaSuccess && ps > 0)
            per_sm = ps;
    });
    const uint64_t cap = (uint64_t)sm_count() * per_sm;
    const uint64_t need = st.P / 32;  // a block per group at most (the warps spread over the blocks)
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    if (grid == 0) return cudaSuccess;
    kern<<<grid, W * 32, smem, stream>>>(st, n, out, counts);
    return cudaGetLastError();
}

template <class Src, int SINK, int W>
static cudaError_t gen_tile(const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out, uint64_t *counts,
                            cudaStream_t stream) {
    if constexpr (SINK == dev::SINK_V4 && !Src::kHeavy) {
        if (c.cache_policy == 2) {
            bool used = false;
            const cudaError_t e = launch_gen_tma<Src, W>(st, n, out, stream, &used);
            if (used || e != cudaSuccess) return e;
            return launch_gen_t<Src, SINK, W, dev::TileCfg<32, 0>>(st, n, out, counts, stream);
        }
        if (c.tile_depth == 64)
            return c.cache_policy ? launch_gen_t<Src, SINK, W, dev::TileCfg<64, 1>>(st, n, out, counts, stream)
                                  : launch_gen_t<Src, SINK, W, dev::TileCfg<64, 0>>(st, n, out, counts, stream);
        return c.cache_policy ? launch_gen_t<Src, SINK, W, dev::TileCfg<32, 1>>(st, n, out, counts, stream)
                              : launch_gen_t<Src, SINK, W, dev::TileCfg<32, 0>>(st, n, out, counts, stream);
    } else if constexpr (SINK == dev::SINK_V4) {
        return c.cache_policy ? launch_gen_t<Src, SINK, W, dev::TileCfg<32, 1>>(st, n, out, counts, stream)
                              : launch_gen_t<Src, SINK, W, dev::TileCfg<32, 0>>(st, n, out, counts, stream);
    } else {
        return launch_gen_t<Src, SINK, W, dev::TileDefault>(st, n, out, counts, stream);
    }
}

template <class Src, int SINK>
static cudaError_t gen_warps(const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out, uint64_t *counts,
                             cudaStream_t stream) {
    switch (c.warps_per_block) {
        case 4:
            return gen_tile<Src, SINK, 4>(c, st, n, out, counts, stream);
        case 16:
            return gen_tile<Src, SINK, 16>(c, st, n, out, counts, stream);
        default:
            return gen_tile<Src, SINK, 8>(c, st, n, out, counts, stream);
    }
}

template <class Src>
static cudaError_t gen_source(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                              uint64_t *counts, cudaStream_t stream) {
    switch (sink) {
        case dev::SINK_V4:
            return gen_warps<Src, dev::SINK_V4>(c, st, n, out, counts, stream);
        case dev::SINK_SCALAR:
            return gen_warps<Src, dev::SINK_SCALAR>(c, st, n, out, counts, stream);
        case dev::SINK_QC:
            return gen_warps<Src, dev::SINK_QC>(c, st, n, out, counts, stream);
        default:
            return gen_warps<Src, dev::SINK_DIGEST>(c, st, n, out, counts, stream);
    }
}

}  // namespace ci
