// ci_gen_xor64.cu -- generation kernels driven by xor64 (the 64-bit xorshift
// of the paper's Sec. 7 measurements).
#include "ci_gen.cuh"

namespace ci {

cudaError_t gen_xor64(int sink, const TuneChoice &c, const DevState &st, uint64_t n, uint32_t *out,
                      uint64_t *counts, cudaStream_t stream) {
    return gen_source<dev::SrcXor64>(sink, c, st, n, out, counts, stream);
}

}  // namespace ci
