// ci_batch.h -- device work queue of the batched persistent kernel (shared by
// the batch API and the serving loop; not part of the C ABI).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "ci_internal.h"

namespace ci {

// Source kinds of a task.
enum TaskKind : uint32_t { K_XOR128 = 0, K_XS32 = 1, K_BBS = 2, K_BBS16 = 3, K_XOR64 = 4 };

// One queue entry: warp groups [g0, g0 + ngroups) of one state, each advanced
// by n iterations; written outputs of row r go to out[r * ld + col0 + i].
// Work unit u (a global index) belongs to the task with the largest prefix
// <= u and is warp group g0 + (u - prefix).
struct BatchTask {
    DevState st;
    uint32_t *out;
    uint64_t *aux;      // quarter-circle counts (+=) or digests (=)
    uint64_t ld, col0, n;
    uint64_t g0, ngroups;
    uint64_t prefix;
    uint32_t kind, sink;
};

// Queue header, copied to the device in front of the tasks.  The cursor is
// zero in every upload; warps claim units with atomicAdd on it.
struct BatchHeader {
    uint64_t total_units;
    uint64_t cursor;
    uint32_t n_tasks;
    uint32_t reserved[3];
};

static_assert(sizeof(BatchHeader) == 32, "header layout");

// Launch geometry of the persistent batched kernel.
struct BatchGeometry {
    void *func;          // kernel entry (k_batched<W>)
    unsigned grid, block;
};

BatchGeometry batch_geometry(int warps_per_block);

// Cost of one output of a task kind relative to xor128 (used to order the
// queue longest-first).
double kind_cost(uint32_t kind);

// Fills a task for `n` iterations of all of h's warp groups (col0 = 0, ld = n)
// and returns the SINK_* it uses.  `sink_abi` is CI_SINK_*.
BatchTask make_task(const ci_states_s &h, uint64_t n, int sink_abi, uint32_t *out, uint64_t *aux,
                    uint64_t ld, uint64_t col0);

// Uploads `tasks` (sorted and packed here) to one of b's two queue slots and
// replays that slot's graph on `stream`; waits first for the launch that
// last used the slot.
// With sort == false the tasks keep their order (serving waves, whose slices
// are already bounded in length).
ci_status batch_launch_tasks(ci_batch_s *b, BatchTask *tasks, uint32_t n_tasks, cudaStream_t stream,
                             bool sort = true);

// Sorts tasks longest-first, assigns prefixes, writes header + tasks to
// `staging` (capacity checked by the caller) and returns the bytes to upload.
uint64_t pack_queue(BatchTask *tasks, uint32_t n_tasks, void *staging, bool sort = true);

}  // namespace ci
