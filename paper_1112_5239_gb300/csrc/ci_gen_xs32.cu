// ci_gen_xs32.cu -- generation kernels driven by Algorithm 2 XORshift (all sinks and launch
// shapes the autotuner may pick).
#include "ci_gen.cuh"

namespace ci {

cudaError_t gen_xs32(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out, uint64_t *counts,
                   cudaStream_t stream) {
    return gen_source<dev::SrcXorshift32>(sink, c, st, n, out, counts, stream);
}

}  // namespace ci
