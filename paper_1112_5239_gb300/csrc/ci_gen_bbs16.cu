// ci_gen_bbs16.cu -- generation kernels driven by Algorithm 5 as printed
// (eight 16-bit-modulus BBS generators per stream).
#include "ci_gen.cuh"

namespace ci {

cudaError_t gen_bbs16(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                      uint64_t *counts, cudaStream_t stream) {
    return gen_source<dev::SrcBbs16>(sink, c, st, n, out, counts, stream);
}

}  // namespace ci
