// ci_api.cu -- the C ABI (include/ci_prng.h): argument checks, state handles,
// combination arrays, checkpoint export/import.  Every entry point returns a
// ci_status and records a message for ci_last_error() on failure.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ci_device.cuh"
#include "ci_split.h"
#include "ci_internal.h"
#include "ci_trace.h"

namespace ci {

static thread_local std::string g_err;

ci_status fail(ci_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

ci_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return CI_E_CUDA;
}

bool valid_handle(const ci_states s) { return s != nullptr && s->magic == kMagic; }

uint64_t state_bytes_for(int variant, uint64_t P) {
    return (uint64_t)kTableBytes + 4ull * (variant == CI_VAR_BBS16 ? kU32FieldsBbs16 : kU32Fields) * P +
           (variant == CI_VAR_BBS ? 8ull * kU64Fields * P : 0ull);
}

// splitmix64 (Steele, Lea & Flood 2014) on the host, for the combination
// arrays: draw i of seed s is mix(s + (i + 1) * golden gamma).
static uint64_t host_draw(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Fisher-Yates shuffle of 0..C-1, consuming draws ctr, ctr+1, ...
static void shuffle(uint32_t C, uint64_t seed, uint64_t &ctr, uint8_t *a) {
    for (uint32_t i = 0; i < C; ++i) a[i] = (uint8_t)i;
    for (uint32_t i = C; i-- > 1;) {
        const uint32_t j = (uint32_t)(host_draw(seed, ctr++) % (uint64_t)(i + 1));
        const uint8_t t = a[i];
        a[i] = a[j];
        a[j] = t;
    }
}

// Combination arrays (Alg. 4: two, Alg. 5: sixteen permutations of [0, C)).
// For the xor variant the second array is redrawn until it differs from the
// first at every position (an equal pair of partners cancels in the XOR).
static void derive_comb(int variant, uint32_t C, uint64_t seed, uint8_t *comb) {
    uint64_t ctr = 0;
    if (variant != CI_VAR_XOR) {
        for (int a = 0; a < 16; ++a) shuffle(C, seed, ctr, comb + a * C);
        return;
    }
    shuffle(C, seed, ctr, comb);
    for (;;) {
        shuffle(C, seed, ctr, comb + C);
        if (C == 1) return;
        bool distinct = true;
        for (uint32_t j = 0; j < C; ++j) distinct = distinct && comb[j] != comb[C + j];
        if (distinct) return;
    }
}

// Partner table: lane j of a warp, array a -> lane (j - j % C) + comb[a][j % C].
static void build_table(int variant, uint32_t C, const uint8_t *comb, uint8_t *table) {
    std::memset(table, 0, kTableBytes);
    const int arrays = variant == CI_VAR_XOR ? 2 : 16;
    for (int a = 0; a < arrays; ++a)
        for (uint32_t j = 0; j < 32; ++j) table[a * 32 + j] = (uint8_t)((j & ~(C - 1)) + comb[a * C + (j & (C - 1))]);
}

static ci_status check_params(const ci_params *p, uint64_t S) {
    if (!p) return fail(CI_E_INVAL, "params is NULL");
    if (p->variant != CI_VAR_XOR && p->variant != CI_VAR_BBS && p->variant != CI_VAR_BBS16)
        return fail(CI_E_INVAL, "unknown variant");
    if (p->variant == CI_VAR_XOR && p->xl != CI_XL_XOR128 && p->xl != CI_XL_XORSHIFT32 && p->xl != CI_XL_XOR64)
        return fail(CI_E_INVAL, "unknown xor-like generator");
    const uint32_t C = p->comb_size;
    if (C < 1 || C > 32 || (C & (C - 1)) != 0) return fail(CI_E_INVAL, "comb_size must be 1, 2, 4, 8, 16 or 32");
    if (p->flags != 0) return fail(CI_E_INVAL, "flags must be 0");
    if (S < 1 || S > (1ull << 32)) return fail(CI_E_INVAL, "n_streams must be in [1, 2^32]");
    if ((p->first_stream & 31ull) != 0 || p->first_stream > (1ull << 32) - S)
        return fail(CI_E_INVAL, "first_stream must be a multiple of 32 with first_stream + n_streams <= 2^32");
    if (p->comb) {
        const uint32_t n = (p->variant == CI_VAR_XOR ? 2u : 16u) * C;
        for (uint32_t i = 0; i < n; ++i)
            if (p->comb[i] >= C) return fail(CI_E_INVAL, "combination array entry >= comb_size");
    }
    return CI_OK;
}

static uint64_t lanes_for(uint64_t S) { return (S + 31ull) & ~31ull; }

ci_status prepare_handle(const ci_params *p, uint64_t S, void *dev, uint64_t bytes, bool owns, ci_states *out) {
    ci_states_s *h = new (std::nothrow) ci_states_s();
    if (!h) return fail(CI_E_NOMEM, "host allocation failed");
    h->magic = kMagic;
    h->variant = p->variant;
    h->xl = p->variant == CI_VAR_XOR ? p->xl : 0;
    h->C = p->comb_size;
    h->S = S;
    h->P = lanes_for(S);
    h->bytes = bytes;
    h->dev = dev;
    h->owns = owns;
    std::memset(h->comb, 0, sizeof h->comb);
    const uint32_t ncomb = (p->variant == CI_VAR_XOR ? 2u : 16u) * h->C;
    if (p->comb)
        std::memcpy(h->comb, p->comb, ncomb);
    else
        derive_comb(p->variant, h->C, p->comb_seed, h->comb);
    build_table(p->variant, h->C, h->comb, h->table);
    *out = h;
    return CI_OK;
}

void fill_init_task(const ci_states_s &h, uint64_t seed, uint64_t first, uint64_t prefix, InitTask *t) {
    t->st = h.view();
    t->seed = seed;
    t->first = first;
    t->prefix = prefix;
    t->variant = h.variant;
    t->xl = h.xl;
    std::memcpy(t->table, h.table, kTableBytes);
}

static ci_status make_handle(const ci_params *p, uint64_t S, void *dev, uint64_t bytes, bool owns,
                             cudaStream_t stream, ci_states *out) {
    ci_states h = nullptr;
    ci_status st = prepare_handle(p, S, dev, bytes, owns, &h);
    if (st != CI_OK) return st;
    cudaError_t e = launch_init(*h, p->seed, p->first_stream, stream);  // also writes the partner table
    if (e != cudaSuccess) {
        h->magic = 0;
        delete h;
        return cuda_fail(e, "state initialisation");
    }
    *out = h;
    return CI_OK;
}

}  // namespace ci

ci::DevState ci_states_s::view() const {
    ci::DevState s;
    uint8_t *base = static_cast<uint8_t *>(dev);
    s.table = base;
    s.u32 = reinterpret_cast<uint32_t *>(base + ci::kTableBytes);
    s.u64 = variant == CI_VAR_BBS ? reinterpret_cast<uint64_t *>(base + ci::kTableBytes + 4ull * ci::kU32Fields * P)
                                  : nullptr;
    s.P = P;
    s.S = S;
    s.check = ci::check_word();
    return s;
}

// ------------------------------------------------- bounds-checked build
namespace ci {

#ifdef CI_CHECKED
namespace {

std::mutex g_check_mu;
unsigned long long *g_check_words[64];  // per device, allocated on first use

// The one deliberate failure: a check whose condition is false, so the status
// path can be tested without any out-of-range access.
__global__ void k_check_probe(DevState st) { CI_WARP_CHECK(st, false, CHK_PROBE, 0); }

const char *check_name(unsigned id) {
    switch (id) {
        case CHK_GROUP: return "warp group beyond the state's lanes";
        case CHK_COLS: return "written columns beyond the row length";
        case CHK_TMA_ALIGN: return "TMA store column not a multiple of 4 words";
        case CHK_V4_ALIGN: return "16-byte stores with unaligned columns or row length";
        case CHK_UNIT: return "batch unit beyond its task's warp groups";
        case CHK_SEGMENT: return "split segment index beyond the segment count";
        case CHK_SEG_COLS: return "split segment's columns beyond the row length";
        case CHK_PROBE: return "probe";
        default: return "unknown check";
    }
}

// Waits for `stream`, then reads and clears the current device's status word.
ci_status read_clear(cudaStream_t stream, unsigned long long *value) {
    *value = 0;
    unsigned long long *w = check_word();
    if (!w) return fail(CI_E_CUDA, "no bounds-check status word on this device");
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaMemcpy(value, w, sizeof *value, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && *value) e = cudaMemsetAsync(w, 0, sizeof *value, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e == cudaSuccess ? CI_OK : cuda_fail(e, "bounds-check status read");
}

}  // namespace

unsigned long long *check_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_check_mu);
    if (!g_check_words[dev]) {
        void *p = nullptr;
        if (cudaMalloc(&p, sizeof(unsigned long long)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(unsigned long long)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            cudaFree(p);
            return nullptr;
        }
        g_check_words[dev] = static_cast<unsigned long long *>(p);
    }
    return g_check_words[dev];
}

ci_status check_epilogue(cudaStream_t stream, ci_status rc) {
    if (rc != CI_OK) return rc;
    unsigned long long v = 0;
    const ci_status st = read_clear(stream, &v);
    if (st != CI_OK) return st;
    if (v)
        return fail(CI_E_INVAL, std::string("bounds check failed: ") + check_name((unsigned)(v >> 56)) + " (index " +
                                    std::to_string(v & ((1ull << 56) - 1)) + ")");
    return CI_OK;
}
#else
unsigned long long *check_word() { return nullptr; }
ci_status check_epilogue(cudaStream_t, ci_status rc) { return rc; }
#endif

}  // namespace ci

using namespace ci;

extern "C" {

ci_status ci_state_bytes(const ci_params *params, uint64_t n_streams, uint64_t *bytes) {
    ci_status st = check_params(params, n_streams);
    if (st != CI_OK) return st;
    if (!bytes) return fail(CI_E_INVAL, "bytes is NULL");
    *bytes = state_bytes_for(params->variant, lanes_for(n_streams));
    return CI_OK;
}

// Host-side fault injection for the error paths (CI_FAULT="alloc_fail@N"):
// the N-th state allocation since CI_FAULT took its current value fails with
// CI_E_NOMEM before anything touches the device.  The server's own hooks
// (queue_full, reject_admit, launch_fail) share the variable and are read
// when a server is created.
static bool injected_alloc_failure() {
    static std::mutex m;
    static std::string spec;
    static uint64_t count = 0;
    const char *env = std::getenv("CI_FAULT");
    std::lock_guard<std::mutex> g(m);
    const std::string now = env ? env : "";
    if (now != spec) {
        spec = now;
        count = 0;
    }
    const size_t at = spec.find("alloc_fail@");
    if (at == std::string::npos) return false;
    const uint64_t n = std::strtoull(spec.c_str() + at + 11, nullptr, 10);
    return ++count == n;
}

ci_status ci_init_states(const ci_params *params, uint64_t n_streams, void *cuda_stream, ci_states *out) {
    if (!out) return fail(CI_E_INVAL, "out is NULL");
    *out = nullptr;
    ci_status st = check_params(params, n_streams);
    if (st != CI_OK) return st;
    const uint64_t bytes = state_bytes_for(params->variant, lanes_for(n_streams));
    if (injected_alloc_failure()) return fail(CI_E_NOMEM, "injected allocation failure (CI_FAULT alloc_fail)");
    void *dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? CI_E_NOMEM : CI_E_CUDA,
                    std::string("cudaMalloc of the state: ") + cudaGetErrorString(e));
    }
    st = make_handle(params, n_streams, dev, bytes, true, static_cast<cudaStream_t>(cuda_stream), out);
    if (st != CI_OK) cudaFree(dev);
    return st;
}

ci_status ci_init_states_at(const ci_params *params, uint64_t n_streams, void *state_dev, uint64_t state_bytes,
                            void *cuda_stream, ci_states *out) {
    if (!out) return fail(CI_E_INVAL, "out is NULL");
    *out = nullptr;
    ci_status st = check_params(params, n_streams);
    if (st != CI_OK) return st;
    const uint64_t need = state_bytes_for(params->variant, lanes_for(n_streams));
    if (!state_dev || (reinterpret_cast<uintptr_t>(state_dev) & 255u) != 0)
        return fail(CI_E_INVAL, "state_dev must be a non-NULL 256-byte aligned device address");
    if (state_bytes < need) return fail(CI_E_INVAL, "state_bytes smaller than ci_state_bytes()");
    return make_handle(params, n_streams, state_dev, need, false, static_cast<cudaStream_t>(cuda_stream), out);
}

ci_status ci_init_states_many(const ci_params *params, const uint64_t *n_streams, uint32_t n, void *cuda_stream,
                              ci_states *out) {
    if (n == 0) return CI_OK;
    if (!params || !n_streams || !out) return fail(CI_E_INVAL, "NULL argument");
    for (uint32_t i = 0; i < n; ++i) out[i] = nullptr;
    for (uint32_t i = 0; i < n; ++i) {
        ci_status st = check_params(&params[i], n_streams[i]);
        if (st != CI_OK) return fail(st, "item " + std::to_string(i) + ": " + g_err);
    }
    cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    std::vector<InitTask> tasks(n);
    uint64_t lanes = 0;
    ci_status rc = CI_OK;
    for (uint32_t i = 0; i < n && rc == CI_OK; ++i) {
        const uint64_t bytes = state_bytes_for(params[i].variant, lanes_for(n_streams[i]));
        if (injected_alloc_failure()) {
            rc = fail(CI_E_NOMEM, "item " + std::to_string(i) + ": injected allocation failure (CI_FAULT alloc_fail)");
            break;
        }
        void *dev = nullptr;
        cudaError_t e = cudaMalloc(&dev, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(e == cudaErrorMemoryAllocation ? CI_E_NOMEM : CI_E_CUDA, "cudaMalloc of a state");
            break;
        }
        rc = prepare_handle(&params[i], n_streams[i], dev, bytes, true, &out[i]);
        if (rc != CI_OK) {
            cudaFree(dev);
            break;
        }
        fill_init_task(*out[i], params[i].seed, params[i].first_stream, lanes, &tasks[i]);
        lanes += out[i]->P;
    }
    InitTask *dtasks = nullptr;
    if (rc == CI_OK) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&dtasks), sizeof(InitTask) * n, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dtasks, tasks.data(), sizeof(InitTask) * n, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = launch_init_batched(dtasks, n, lanes, cs);
        if (dtasks) cudaFreeAsync(dtasks, cs);
        if (e != cudaSuccess) rc = cuda_fail(e, "batched state initialisation");
    }
    if (rc != CI_OK) {
        for (uint32_t i = 0; i < n; ++i) {
            if (out[i]) ci_free_states(out[i]);
            out[i] = nullptr;
        }
    }
    return rc;
}

ci_status ci_free_states(ci_states s) {
    if (!s) return CI_OK;
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    s->magic = 0;
    cudaError_t e = cudaSuccess;
    if (s->owns) e = cudaFree(s->dev);
    delete s;
    return e == cudaSuccess ? CI_OK : cuda_fail(e, "cudaFree of the state");
}

ci_status ci_states_query(ci_states s, ci_states_desc *out) {
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    if (!out) return fail(CI_E_INVAL, "out is NULL");
    std::memset(out, 0, sizeof *out);
    out->variant = s->variant;
    out->xl = s->xl;
    out->comb_size = s->C;
    out->n_streams = s->S;
    out->n_lanes = s->P;
    out->state_bytes = s->bytes;
    out->state_dev = s->dev;
    std::memcpy(out->comb, s->comb, sizeof out->comb);
    return CI_OK;
}

static ci_status check_out(ci_states s, uint64_t n, const void *out, uint64_t cap) {
    if (!out) return fail(CI_E_INVAL, "out_dev is NULL");
    if (n > 0 && s->S > UINT64_MAX / n) return fail(CI_E_INVAL, "n_streams * n_per_stream overflows");
    if (cap < s->S * n) return fail(CI_E_INVAL, "out_capacity_u32 < n_streams * n_per_stream");
    return CI_OK;
}

ci_status ci_generate(ci_states s, uint64_t n, uint32_t *out, uint64_t cap, void *stream) {
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    TraceRange trace("ci_generate");
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    if (s->variant != CI_VAR_XOR) return fail(CI_E_STATE, "ci_generate needs an xor-variant state (use ci_generate_bbs)");
    if (n == 0) return CI_OK;
    ci_status st = check_out(s, n, out, cap);
    if (st != CI_OK) return st;
    // A narrow state is a few serial chains: run it as time segments (identical results).
    const uint64_t K = split_auto(*s, n, CI_SINK_WRITTEN);
    if (K > 1) return check_epilogue(cs, split_launch(*s, n, CI_SINK_WRITTEN, out, n, 0, nullptr, K, cs));
    cudaError_t e = launch_generate(*s, n, out, cs);
    return check_epilogue(cs, e == cudaSuccess ? CI_OK : cuda_fail(e, "generation kernel launch"));
}

ci_status ci_generate_bbs(ci_states s, uint64_t n, uint32_t *out, uint64_t cap, void *stream) {
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    TraceRange trace("ci_generate_bbs");
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    if (s->variant == CI_VAR_XOR) return fail(CI_E_STATE, "ci_generate_bbs needs a BBS-variant state (use ci_generate)");
    if (n == 0) return CI_OK;
    ci_status st = check_out(s, n, out, cap);
    if (st != CI_OK) return st;
    // Few streams leave most SMs idle on their serial squaring chains: run the
    // call as time segments instead (identical results).
    const uint64_t K = split_auto(*s, n, CI_SINK_WRITTEN);
    if (K > 1) return check_epilogue(cs, split_launch(*s, n, CI_SINK_WRITTEN, out, n, 0, nullptr, K, cs));
    cudaError_t e = launch_generate(*s, n, out, cs);
    return check_epilogue(cs, e == cudaSuccess ? CI_OK : cuda_fail(e, "BBS generation kernel launch"));
}

ci_status ci_generate_fused_qc(ci_states s, uint64_t n, uint64_t *counts, void *stream) {
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    TraceRange trace("ci_generate_fused_qc");
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    if (n & 1ull) return fail(CI_E_INVAL, "n_per_stream must be even (outputs are consumed in pairs)");
    if (n == 0) return CI_OK;
    if (!counts) return fail(CI_E_INVAL, "counts_dev is NULL");
    const uint64_t K = split_auto(*s, n, CI_SINK_QC);
    if (K > 1) return check_epilogue(cs, split_launch(*s, n, CI_SINK_QC, nullptr, n, 0, counts, K, cs));
    cudaError_t e = launch_fused_qc(*s, n, counts, cs);
    return check_epilogue(cs, e == cudaSuccess ? CI_OK : cuda_fail(e, "fused generation kernel launch"));
}

ci_status ci_generate_digest(ci_states s, uint64_t n, uint64_t *digest, void *stream) {
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    TraceRange trace("ci_generate_digest");
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    if (n == 0) return CI_OK;
    if (!digest) return fail(CI_E_INVAL, "digest_dev is NULL");
    const uint64_t K = split_auto(*s, n, CI_SINK_DIGEST);
    if (K > 1) return check_epilogue(cs, split_launch(*s, n, CI_SINK_DIGEST, nullptr, n, 0, digest, K, cs));
    cudaError_t e = launch_digest(*s, n, digest, cs);
    return check_epilogue(cs, e == cudaSuccess ? CI_OK : cuda_fail(e, "digest kernel launch"));
}

ci_status ci_export_state(ci_states s, void *host_buf, uint64_t bytes, void *stream) {
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    if (!host_buf || bytes != s->bytes) return fail(CI_E_INVAL, "host_buf NULL or bytes != state_bytes");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(host_buf, s->dev, bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    return e == cudaSuccess ? CI_OK : cuda_fail(e, "state export");
}

// The per-lane rules an imported state must follow (see ci_import_state).
static ci_status check_import(const ci_states_s &h, const uint8_t *buf) {
    const uint64_t P = h.P;
    const uint32_t *u32 = reinterpret_cast<const uint32_t *>(buf + kTableBytes);
    if (h.variant == CI_VAR_BBS) {
        const uint64_t *u64 = reinterpret_cast<const uint64_t *>(buf + kTableBytes + 4ull * kU32Fields * P);
        for (uint64_t l = 0; l < P; ++l) {
            const uint64_t y = u64[G_Y * P + l], M = u64[G_M * P + l], mu = u64[G_MU * P + l];
            const uint64_t p = u32[F_P * P + l], q = u32[F_Q * P + l];
            const uint32_t n = M ? dev::bit_length64(M) : 0;
            if (n < 33 || n > 62 || !(M & 1ull) || p * q != M)
                return fail(CI_E_INVAL, "imported BBS lane " + std::to_string(l) + ": M must be p q of 33 to 62 bits");
            if (y >= M || mu != dev::barrett_mu(M))
                return fail(CI_E_INVAL, "imported BBS lane " + std::to_string(l) + ": y >= M or a wrong reciprocal");
        }
    } else if (h.variant == CI_VAR_BBS16) {
        for (uint64_t l = 0; l < P; ++l)
            for (int g = 0; g < 8; ++g) {
                const uint32_t y = u32[(F_Y16 + g) * P + l], M = u32[(F_M16 + g) * P + l];
                if (M < 3 || M >= (1u << 16) || y >= M)
                    return fail(CI_E_INVAL, "imported Algorithm 5 lane " + std::to_string(l) +
                                                ": a modulus outside [3, 2^16) or a state above it");
            }
    }
    return CI_OK;
}

ci_status ci_import_state(ci_states s, const void *host_buf, uint64_t bytes, void *stream) {
    if (!valid_handle(s)) return fail(CI_E_STATE, "not a live ci_states handle");
    if (!host_buf || bytes != s->bytes) return fail(CI_E_INVAL, "host_buf NULL or bytes != state_bytes");
    const ci_status chk = check_import(*s, static_cast<const uint8_t *>(host_buf));
    if (chk != CI_OK) return chk;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(s->dev, host_buf, bytes, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(e, "state import");
    std::memcpy(s->table, host_buf, kTableBytes);
    return CI_OK;
}

ci_status ci_check_status(uint64_t *word, void *stream) {
    if (!word) return fail(CI_E_INVAL, "word is NULL");
    *word = 0;
#ifdef CI_CHECKED
    unsigned long long v = 0;
    const ci_status st = read_clear(static_cast<cudaStream_t>(stream), &v);
    *word = v;
    return st;
#else
    (void)stream;
    return fail(CI_E_STATE, "bounds checks are compiled only into the CI_CHECKED build");
#endif
}

ci_status ci_check_probe(void *stream) {
#ifdef CI_CHECKED
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    DevState st{};
    st.check = check_word();
    if (!st.check) return fail(CI_E_CUDA, "no bounds-check status word on this device");
    k_check_probe<<<1, 32, 0, cs>>>(st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "probe kernel launch");
    return check_epilogue(cs, CI_OK);
#else
    (void)stream;
    return fail(CI_E_STATE, "bounds checks are compiled only into the CI_CHECKED build");
#endif
}

const char *ci_last_error(void) { return g_err.c_str(); }

uint32_t ci_version(void) { return 10000u; }

}  // extern "C"
