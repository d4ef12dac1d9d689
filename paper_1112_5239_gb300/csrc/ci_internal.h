// ci_internal.h -- host-side structures shared by the library's translation
// units (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "ci_prng.h"

namespace ci {

// Device state layout (see ci_export_state in ci_prng.h).
constexpr int kTableBytes = 512;     // partner table u8[16][32]
constexpr int kU32Fields = 9;        // a b c d x slot sel p q
constexpr int kU32FieldsBbs16 = 25;  // ... then y16[8], m16[8] (CI_VAR_BBS16)
constexpr int kU64Fields = 3;        // y M mu (BBS only)
enum U32Field { F_A = 0, F_B = 1, F_C = 2, F_D = 3, F_X = 4, F_SLOT = 5, F_SEL = 6, F_P = 7, F_Q = 8, F_Y16 = 9, F_M16 = 17 };
enum U64Field { G_Y = 0, G_M = 1, G_MU = 2 };

// Device view of one handle's state, passed to kernels by value.
struct DevState {
    const uint8_t *table;  // [16][32]
    uint32_t *u32;         // field f at u32 + f * P
    uint64_t *u64;         // field g at u64 + g * P (BBS)
    uint64_t P;            // lanes (multiple of 32)
    uint64_t S;            // streams returned
    unsigned long long *check;  // bounds-check status word (CI_CHECKED builds), else null
};

// Bounds checks of the CI_CHECKED build.  A failed check stores
// (id << 56) | (index & (2^56 - 1)) in the status word of the device (the
// first failure wins) and the warp skips the work the check guards.
enum CheckId : uint32_t {
    CHK_GROUP = 1,      // warp group beyond the state's lanes
    CHK_COLS = 2,       // written columns beyond the row length
    CHK_TMA_ALIGN = 3,  // TMA store column not a multiple of 4 words
    CHK_V4_ALIGN = 4,   // 16-byte stores with unaligned columns or row length
    CHK_UNIT = 5,       // batch unit beyond its task's warp groups
    CHK_SEGMENT = 6,    // split segment index beyond the segment count
    CHK_SEG_COLS = 7,   // split segment's columns beyond the row length
    CHK_PROBE = 8,      // the deliberate failure of ci_check_probe
};

// Status word of the current device (CI_CHECKED builds: allocated on first use;
// otherwise null).
unsigned long long *check_word();
// Run by every synchronous entry point before it returns rc: in CI_CHECKED
// builds it waits for `stream`, reads and clears the status word and turns a
// recorded failure into CI_E_INVAL; otherwise it returns rc unchanged.
ci_status check_epilogue(cudaStream_t stream, ci_status rc);

uint64_t state_bytes_for(int variant, uint64_t P);

// One state to seed in a batched initialisation launch; lanes of all tasks
// form one index space (task t owns [prefix, prefix + st.P)).
struct InitTask {
    DevState st;
    uint64_t seed, first, prefix;
    int32_t variant, xl;
    uint32_t table[kTableBytes / 4];
};

}  // namespace ci

struct ci_states_s {
    uint32_t magic;
    int32_t variant, xl;
    uint32_t C;
    uint64_t S, P;
    uint64_t bytes;
    void *dev;
    bool owns;
    uint8_t comb[16 * 32];
    uint8_t table[ci::kTableBytes];
    ci::DevState view() const;
};

namespace ci {

constexpr uint32_t kMagic = 0xC1C1A05Eu;

// Thread-local error message; returns `st` for tail calls.
ci_status fail(ci_status st, const std::string &msg);
ci_status cuda_fail(cudaError_t e, const char *what);
bool valid_handle(const ci_states s);

// Kernel launchers (ci_kernels.cu).  All asynchronous on `stream`.
cudaError_t launch_init(const ci_states_s &h, uint64_t seed, uint64_t first_stream, cudaStream_t stream);
cudaError_t launch_generate(const ci_states_s &h, uint64_t n, uint32_t *out, cudaStream_t stream);
cudaError_t launch_fused_qc(const ci_states_s &h, uint64_t n, uint64_t *counts, cudaStream_t stream);
cudaError_t launch_digest(const ci_states_s &h, uint64_t n, uint64_t *digest, cudaStream_t stream);
cudaError_t launch_init_batched(const InitTask *dev_tasks, uint32_t n_tasks, uint64_t total_lanes,
                                cudaStream_t stream);

// Validates params and builds a handle over `dev` (which must hold
// state_bytes_for(...) bytes) without seeding it; fill_init_task describes the
// seeding for a batched launch.
ci_status prepare_handle(const ci_params *p, uint64_t S, void *dev, uint64_t bytes, bool owns, ci_states *out);
void fill_init_task(const ci_states_s &h, uint64_t seed, uint64_t first, uint64_t prefix, InitTask *t);

int sm_count();

}  // namespace ci
