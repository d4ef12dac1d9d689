// ci_split.h -- time-parallel generation (ci_split.cu), shared by the C ABI
// (ci_generate_split, ci_generate_bbs) and the serving loop's split jobs (not
// part of the C ABI).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "ci_internal.h"

namespace ci {

constexpr uint32_t kSplitMaxSegments = 8192;

// Segment count for n iterations of h (requested == 0: from the GPU size);
// 1 means unsplit.
uint64_t split_segments(const ci_states_s &h, uint64_t n, uint64_t requested);

// Segment count ci_generate_bbs (and the BBS consumer calls) use on their
// own for CI_VAR_BBS states, 1 for others.  Written sink, and consumer sinks
// whose outputs fit the scratch (2^29 words; they are written, fixed up and
// reduced): from the GPU size and the form split_launch takes (one launch
// from 12 warp groups per SM on, three launches below); larger consumer
// calls, which generate twice: > 1 only for states that fill less than about
// two waves of resident warps.
uint64_t split_auto_bbs(const ci_states_s &h, uint64_t n, int sink);

// Segment count the single-call entry points use on their own for `sink`
// (CI_SINK_*): split_auto_bbs for CI_VAR_BBS; for xor-like states only with
// no more warp groups than SMs (and segments of at least 1024 iterations);
// for CI_VAR_BBS16 likewise (segments of at least 256); 1 otherwise.
uint64_t split_auto(const ci_states_s &h, uint64_t n, int sink);

// n iterations of h as K segments into `sink` (written: out[r * ld + col0 + i];
// consumers: aux[r]), with results equal to one sequential call.  Calls on
// different streams are independent (no shared queue or lock).

ci_status split_launch(const ci_states_s &h, uint64_t n, int sink, uint32_t *out, uint64_t ld, uint64_t col0,
                       uint64_t *aux, uint64_t K, cudaStream_t stream);

// Builds the jump tables for the current device (blocks once on `stream`).
cudaError_t split_prepare(cudaStream_t stream);

}  // namespace ci
