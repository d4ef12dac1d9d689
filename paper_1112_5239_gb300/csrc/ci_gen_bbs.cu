// ci_gen_bbs.cu -- generation kernels driven by BBS (Algorithm 5) (all sinks and launch
// shapes the autotuner may pick).
#include "ci_gen.cuh"

namespace ci {

cudaError_t gen_bbs(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out, uint64_t *counts,
                   cudaStream_t stream) {
    return gen_source<dev::SrcBbs>(sink, c, st, n, out, counts, stream);
}

}  // namespace ci
