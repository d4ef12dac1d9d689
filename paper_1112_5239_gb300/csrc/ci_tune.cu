// ci_tune.cu -- the autotuner: times every allowed launch shape of each
// (strategy source, sink) generation kernel and of the batched persistent
// kernel on representative synthetic problems, and installs the fastest.
// Launch shapes never change results (tests check every shape against the
// oracle), only speed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <mutex>
#include <vector>

#include "ci_batch.h"
#include "ci_device.cuh"
#include "ci_tune.h"

namespace ci {

static std::mutex g_tune_mu;
static ci_tune_table g_table = [] {
    ci_tune_table t;
    std::memset(&t, 0, sizeof t);
    for (int s = 0; s < kSrcKinds; ++s)
        for (int k = 0; k < 4; ++k) {
            t.choice[s][k].warps_per_block = 8;
            t.choice[s][k].tile_depth = 32;
            t.choice[s][k].cache_policy = 0;
        }
    t.batch_warps_per_block = 8;
    return t;
}();

TuneChoice tuned(int src, int sink) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const ci_tune_choice &c = g_table.choice[src][sink];
    return TuneChoice{c.warps_per_block, c.tile_depth, c.cache_policy};
}

int tuned_batch_warps() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (int)g_table.batch_warps_per_block;
}

static bool valid_choice(int src, int sink, const ci_tune_choice &c) {
    if (c.warps_per_block != 4 && c.warps_per_block != 8 && c.warps_per_block != 16) return false;
    if (c.cache_policy > 2) return false;
    if (c.tile_depth != 32 && c.tile_depth != 64) return false;
    const bool xor_src = src == SK_XOR128 || src == SK_XS32 || src == SK_XOR64;
    if (c.tile_depth == 64 && !(sink == dev::SINK_V4 && xor_src)) return false;
    if (c.cache_policy == 1 && sink != dev::SINK_V4) return false;
    if (c.cache_policy == 2 && !(sink == dev::SINK_V4 && xor_src && c.tile_depth == 32)) return false;
    return true;
}

// Candidate shapes of one (source, sink) class.
static std::vector<ci_tune_choice> candidates(int src, int sink) {
    std::vector<ci_tune_choice> v;
    for (uint32_t w : {4u, 8u, 16u})
        for (uint32_t kt : {32u, 64u})
            for (uint32_t cp : {0u, 1u, 2u}) {
                ci_tune_choice c;
                std::memset(&c, 0, sizeof c);
                c.warps_per_block = w;
                c.tile_depth = kt;
                c.cache_policy = cp;
                if (valid_choice(src, sink, c)) v.push_back(c);
            }
    return v;
}

// Median of reps - 1 timed launches (the first launch is the warm-up).
static float time_launches(cudaStream_t s, int reps, const std::function<cudaError_t()> &fn, cudaError_t *err) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<float> t;
    for (int r = 0; r < reps && *err == cudaSuccess; ++r) {
        cudaEventRecord(a, s);
        *err = fn();
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) t.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (t.empty()) return 1e30f;
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace ci

using namespace ci;

extern "C" {

ci_status ci_tune_get(ci_tune_table *out) {
    if (!out) return fail(CI_E_INVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *out = g_table;
    return CI_OK;
}

ci_status ci_tune_set(const ci_tune_table *in) {
    if (!in) return fail(CI_E_INVAL, "in is NULL");
    for (int s = 0; s < kSrcKinds; ++s)
        for (int k = 0; k < 4; ++k)
            if (!valid_choice(s, k, in->choice[s][k])) return fail(CI_E_INVAL, "launch shape not allowed for its class");
    if (in->batch_warps_per_block != 4 && in->batch_warps_per_block != 8 && in->batch_warps_per_block != 16)
        return fail(CI_E_INVAL, "batch_warps_per_block must be 4, 8 or 16");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table = *in;
    return CI_OK;
}

ci_status ci_autotune(uint32_t flags, void *cuda_stream, ci_tune_table *out) {
    if (flags != 0) return fail(CI_E_INVAL, "flags must be 0");
    cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    ci_tune_table table;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        table = g_table;
    }
    // Representative problems: xor sources 2^20 streams (written: 256 outputs
    // per stream, a 1 GiB launch; consumers: 1024), BBS sources 2^16 x 1024
    // (at 128 outputs the shapes' times were within noise of each other and
    // the pick could be 4 % slower on long calls).
    const uint64_t S_xor = 1ull << 20, S_bbs = 1ull << 16;
    const uint64_t L_written = 256, L_fused = 1024, L_bbs = 1024;
    ci_params p;
    std::memset(&p, 0, sizeof p);
    p.comb_size = 32;
    p.seed = 12345;
    ci_states hs[kSrcKinds] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    const uint64_t S_of[kSrcKinds] = {S_xor, S_xor, S_bbs, S_bbs, S_xor};
    ci_status rc = CI_OK;
    for (int s = 0; s < kSrcKinds && rc == CI_OK; ++s) {
        p.variant = s == SK_BBS ? CI_VAR_BBS : (s == SK_BBS16 ? CI_VAR_BBS16 : CI_VAR_XOR);
        p.xl = s == SK_XS32 ? CI_XL_XORSHIFT32 : s == SK_XOR64 ? CI_XL_XOR64 : CI_XL_XOR128;
        rc = ci_init_states(&p, S_of[s], cuda_stream, &hs[s]);
    }
    uint32_t *out_dev = nullptr;
    uint64_t *aux_dev = nullptr;
    cudaError_t e = cudaSuccess;
    if (rc == CI_OK) e = cudaMalloc(&out_dev, S_xor * L_written * 4 + 64);
    if (rc == CI_OK && e == cudaSuccess) e = cudaMalloc(&aux_dev, S_xor * 8);
    if (rc == CI_OK && e != cudaSuccess) rc = cuda_fail(e, "autotuner buffers");
    for (int s = 0; s < kSrcKinds && rc == CI_OK; ++s) {
        for (int k = 0; k < 4 && rc == CI_OK; ++k) {
            const bool bbs_src = s == SK_BBS || s == SK_BBS16;
            const uint64_t L = bbs_src ? L_bbs : (k <= dev::SINK_SCALAR ? L_written : L_fused);
            // the unaligned written sink runs on an output offset by one word
            uint32_t *o = k == dev::SINK_SCALAR ? out_dev + 1 : out_dev;
            float best = 1e30f;
            ci_tune_choice pick = table.choice[s][k];
            for (const ci_tune_choice &c : candidates(s, k)) {
                const TuneChoice tc{c.warps_per_block, c.tile_depth, c.cache_policy};
                const float ms = time_launches(cs, 6, [&] { return launch_with(*hs[s], k, tc, L, o, aux_dev, cs); }, &e);
                if (e != cudaSuccess) break;
                if (ms < best) {
                    best = ms;
                    pick = c;
                    pick.ms = ms;
                }
            }
            if (e != cudaSuccess) rc = cuda_fail(e, "autotuner launch");
            table.choice[s][k] = pick;
        }
    }
    // the batched persistent kernel: a mixed batch of small and large requests
    if (rc == CI_OK) {
        float best = 1e30f;
        std::vector<ci_states> small;
        std::vector<ci_batch_item> items;
        for (int i = 0; i < 64 && rc == CI_OK; ++i) {
            ci_params q = p;
            q.variant = (i % 5 == 0) ? CI_VAR_BBS : CI_VAR_XOR;
            q.xl = CI_XL_XOR128;
            q.seed = 777 + i;
            ci_states h = nullptr;
            rc = ci_init_states(&q, 1 + (uint64_t)(i * 997) % 4096, cuda_stream, &h);
            if (rc != CI_OK) break;
            small.push_back(h);
            ci_batch_item it;
            std::memset(&it, 0, sizeof it);
            it.states = h;
            it.n_per_stream = q.variant == CI_VAR_BBS ? 64 : 64 + (uint64_t)(i * 131) % 2048;
            it.sink = CI_SINK_DIGEST;
            it.aux_dev = aux_dev;  // digests overwrite: the values are not read
            items.push_back(it);
        }
        // items share aux_dev: digests of different handles land on the same
        // words, which is harmless for timing
        uint32_t best_w = table.batch_warps_per_block;
        for (uint32_t w : {4u, 8u, 16u}) {
            if (rc != CI_OK) break;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_table.batch_warps_per_block = w;
            }
            ci_batch b = nullptr;  // its kernel shape is read from the table at creation
            rc = ci_batch_create((uint32_t)items.size(), &b);
            if (rc != CI_OK) break;
            const float ms = time_launches(cs, 4, [&] {
                return ci_batch_run(b, items.data(), (uint32_t)items.size(), cuda_stream) == CI_OK ? cudaSuccess
                                                                                                   : cudaErrorUnknown;
            }, &e);
            ci_batch_destroy(b);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "autotuner batch launch");
                break;
            }
            if (ms < best) {
                best = ms;
                best_w = w;
            }
        }
        table.batch_warps_per_block = best_w;
        table.batch_ms = best;
        for (ci_states h : small) ci_free_states(h);
    }
    cudaStreamSynchronize(cs);
    if (out_dev) cudaFree(out_dev);
    if (aux_dev) cudaFree(aux_dev);
    for (ci_states h : hs)
        if (h) ci_free_states(h);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (rc == CI_OK)
            g_table = table;
        else
            g_table.batch_warps_per_block = table.batch_warps_per_block;
    }
    if (rc == CI_OK && out) *out = table;
    return rc;
}

}  // extern "C"
