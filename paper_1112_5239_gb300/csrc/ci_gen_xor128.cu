// ci_gen_xor128.cu -- generation kernels driven by the 32-bit xor128 (all sinks and launch
// shapes the autotuner may pick).
#include "ci_gen.cuh"

namespace ci {

cudaError_t gen_xor128(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out, uint64_t *counts,
                   cudaStream_t stream) {
    return gen_source<dev::SrcXor128>(sink, c, st, n, out, counts, stream);
}

}  // namespace ci
