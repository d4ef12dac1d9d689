// ci_tune.h -- launch-shape choices picked by the autotuner (ci_tune.cu) and
// consulted by every generation launch.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "ci_internal.h"

namespace ci {

struct TuneChoice {
    uint32_t warps_per_block;  // 4, 8 or 16
    uint32_t tile_depth;       // written sinks: outputs per stream per staging flush, 32 or 64
    uint32_t cache_policy;     // written sinks: 0 streaming (evict-first) stores, 1 write-back
};

enum SrcKind { SK_XOR128 = 0, SK_XS32 = 1, SK_BBS = 2, SK_BBS16 = 3, SK_XOR64 = 4 };
constexpr int kSrcKinds = 5;

// Current choice for a (source kind, SINK_*) pair.
TuneChoice tuned(int src, int sink);
// Warps per block of the batched persistent kernel.
int tuned_batch_warps();

cudaError_t gen_xor128(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                       uint64_t *counts, cudaStream_t stream);
cudaError_t gen_xs32(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                     uint64_t *counts, cudaStream_t stream);
cudaError_t gen_bbs(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                    uint64_t *counts, cudaStream_t stream);
cudaError_t gen_xor64(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                      uint64_t *counts, cudaStream_t stream);
cudaError_t gen_bbs16(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                      uint64_t *counts, cudaStream_t stream);

// Generation launch for handle h with an explicit choice (the tuner) or the
// tuned one.
cudaError_t launch_with(const ci_states_s &h, int sink, const TuneChoice &c, uint64_t n, uint32_t *out,
                        uint64_t *counts, cudaStream_t stream);

}  // namespace ci
