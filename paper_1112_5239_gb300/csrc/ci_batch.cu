// ci_batch.cu -- the batched persistent kernel: one launch drains a device
// work queue of (state, warp group, length) units for many requests of
// uneven stream counts, lengths and variants; plus the C ABI around it
// (ci_batch_create / ci_batch_run / ci_batch_destroy), which replays a CUDA
// graph (queue upload -> persistent kernel) per batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "ci_batch.h"
#include "ci_device.cuh"
#include "ci_trace.h"
#include "ci_tune.h"

namespace ci {

using namespace dev;

template <class Src>
__device__ __forceinline__ void run_sink(const BatchTask &T, uint64_t g, uint4 *tile) {
    switch (T.sink) {
        case SINK_V4:
            warp_task<Src, SINK_V4>(T.st, g, T.n, T.out, T.ld, T.col0, T.aux, tile);
            break;
        case SINK_SCALAR:
            warp_task<Src, SINK_SCALAR>(T.st, g, T.n, T.out, T.ld, T.col0, T.aux, tile);
            break;
        case SINK_QC:
            warp_task<Src, SINK_QC>(T.st, g, T.n, T.out, T.ld, T.col0, T.aux, tile);
            break;
        default:
            warp_task<Src, SINK_DIGEST>(T.st, g, T.n, T.out, T.ld, T.col0, T.aux, tile);
            break;
    }
}

// Persistent: every warp loops claiming one unit at a time from the cursor
// until the queue is empty.  Units are handed out in queue order, and the
// host orders tasks longest-first, so long serial chains start early.
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_batched(BatchHeader *hdr, const BatchTask *tasks) {
    __shared__ uint4 tiles[WARPS][256];
    const int lane = threadIdx.x & 31;
    uint4 *tile = tiles[threadIdx.x >> 5];
    const uint64_t total = hdr->total_units;
    const uint32_t nt = hdr->n_tasks;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(reinterpret_cast<unsigned long long *>(&hdr->cursor), 1ull);
        u = __shfl_sync(kFull, u, 0);
        if (u >= total) break;
        uint32_t lo = 0, hi = nt;  // tasks[lo].prefix <= u < tasks[hi].prefix
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (tasks[mid].prefix <= u)
                lo = mid;
            else
                hi = mid;
        }
        const BatchTask T = tasks[lo];
        CI_WARP_CHECK(T.st, u - T.prefix < T.ngroups, CHK_UNIT, u);
        const uint64_t g = T.g0 + (u - T.prefix);
        if (T.kind == K_BBS)
            run_sink<SrcBbs>(T, g, tile);
        else if (T.kind == K_BBS16)
            run_sink<SrcBbs16>(T, g, tile);
        else if (T.kind == K_XS32)
            run_sink<SrcXorshift32>(T, g, tile);
        else if (T.kind == K_XOR64)
            run_sink<SrcXor64>(T, g, tile);
        else
            run_sink<SrcXor128>(T, g, tile);
    }
}

template <int W>
static BatchGeometry geometry_for() {
    BatchGeometry g;
    g.func = reinterpret_cast<void *>(k_batched<W>);
    g.block = W * 32;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<W>, W * 32, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    g.grid = (unsigned)(sm_count() * per_sm);
    return g;
}

BatchGeometry batch_geometry(int warps_per_block) {
    switch (warps_per_block) {
        case 4:
            return geometry_for<4>();
        case 16:
            return geometry_for<16>();
        default:
            return geometry_for<8>();
    }
}

double kind_cost(uint32_t kind) {
    // measured ratios of per-output cost (BBS: 11 Barrett squarings per
    // output; BBS16: 12 32-bit Barrett squarings)
    return kind == K_BBS ? 40.0 : kind == K_BBS16 ? 8.0 : 1.0;
}

BatchTask make_task(const ci_states_s &h, uint64_t n, int sink_abi, uint32_t *out, uint64_t *aux, uint64_t ld,
                    uint64_t col0) {
    BatchTask t;
    std::memset(&t, 0, sizeof t);
    t.st = h.view();
    t.out = out;
    t.aux = aux;
    t.ld = ld;
    t.col0 = col0;
    t.n = n;
    t.g0 = 0;
    t.ngroups = h.P / 32;
    t.kind = h.variant == CI_VAR_BBS     ? K_BBS
             : h.variant == CI_VAR_BBS16 ? K_BBS16
             : (h.xl == CI_XL_XORSHIFT32 ? K_XS32 : h.xl == CI_XL_XOR64 ? K_XOR64 : K_XOR128);
    if (sink_abi == CI_SINK_QC)
        t.sink = SINK_QC;
    else if (sink_abi == CI_SINK_DIGEST)
        t.sink = SINK_DIGEST;
    else {
        const bool v4 = (reinterpret_cast<uintptr_t>(out) & 15u) == 0 && ld % 4 == 0 && col0 % 4 == 0;
        t.sink = v4 ? SINK_V4 : SINK_SCALAR;
    }
    return t;
}

uint64_t pack_queue(BatchTask *tasks, uint32_t n_tasks, void *staging, bool sort) {
    if (sort)
        std::stable_sort(tasks, tasks + n_tasks, [](const BatchTask &a, const BatchTask &b) {
            return (double)a.n * kind_cost(a.kind) > (double)b.n * kind_cost(b.kind);
        });
    uint64_t prefix = 0;
    for (uint32_t i = 0; i < n_tasks; ++i) {
        tasks[i].prefix = prefix;
        prefix += tasks[i].ngroups;
    }
    BatchHeader hdr;
    std::memset(&hdr, 0, sizeof hdr);
    hdr.total_units = prefix;
    hdr.cursor = 0;
    hdr.n_tasks = n_tasks;
    std::memcpy(staging, &hdr, sizeof hdr);
    std::memcpy(static_cast<char *>(staging) + sizeof hdr, tasks, sizeof(BatchTask) * n_tasks);
    return sizeof hdr + sizeof(BatchTask) * (uint64_t)n_tasks;
}

}  // namespace ci

// --------------------------------------------------------------- C ABI
using namespace ci;

struct ci_batch_s {
    uint32_t magic;
    uint32_t max_items;
    uint64_t bytes;
    void *dev[2] = {nullptr, nullptr};
    void *host[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool pending[2] = {false, false};
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaGraphNode_t copy_node[2] = {nullptr, nullptr};
    int slot = 0;
    BatchGeometry geo;
    std::vector<BatchTask> tasks;
};

static constexpr uint32_t kBatchMagic = 0xBA7C4ED1u;

static void batch_release(ci_batch_s *b) {
    for (int i = 0; i < 2; ++i) {
        if (b->pending[i]) cudaEventSynchronize(b->done[i]);
        if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
        if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
        if (b->done[i]) cudaEventDestroy(b->done[i]);
        if (b->dev[i]) cudaFree(b->dev[i]);
        if (b->host[i]) cudaFreeHost(b->host[i]);
    }
    b->magic = 0;
    delete b;
}

// Graph for slot i: H2D upload of header + tasks, then the persistent kernel.
static cudaError_t build_graph(ci_batch_s *b, int i) {
    cudaError_t e = cudaGraphCreate(&b->graph[i], 0);
    if (e != cudaSuccess) return e;
    e = cudaGraphAddMemcpyNode1D(&b->copy_node[i], b->graph[i], nullptr, 0, b->dev[i], b->host[i],
                                 sizeof(BatchHeader), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    BatchHeader *hdr = static_cast<BatchHeader *>(b->dev[i]);
    BatchTask *tasks = reinterpret_cast<BatchTask *>(static_cast<char *>(b->dev[i]) + sizeof(BatchHeader));
    void *args[2] = {&hdr, &tasks};
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.func = b->geo.func;
    kp.gridDim = dim3(b->geo.grid);
    kp.blockDim = dim3(b->geo.block);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    cudaGraphNode_t kn;
    e = cudaGraphAddKernelNode(&kn, b->graph[i], &b->copy_node[i], 1, &kp);
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(&b->exec[i], b->graph[i], 0);
}

namespace ci {

ci_status batch_launch_tasks(ci_batch_s *b, BatchTask *tasks, uint32_t n_tasks, cudaStream_t cs, bool sort) {
    TraceRange trace("batch launch");
    if (n_tasks == 0) return CI_OK;
    if (n_tasks > b->max_items) return fail(CI_E_INVAL, "more tasks than the batch's max_items");
    const int s = b->slot;
    b->slot ^= 1;
    if (b->pending[s]) {
        cudaError_t e = cudaEventSynchronize(b->done[s]);
        if (e != cudaSuccess) return cuda_fail(e, "waiting for the previous batch");
        b->pending[s] = false;
    }
    const uint64_t bytes = pack_queue(tasks, n_tasks, b->host[s], sort);
    cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(b->exec[s], b->copy_node[s], b->dev[s], b->host[s], bytes,
                                                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec[s], cs);
    if (e == cudaSuccess) e = cudaEventRecord(b->done[s], cs);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    b->pending[s] = true;
    return CI_OK;
}

}  // namespace ci

extern "C" {

ci_status ci_batch_create(uint32_t max_items, ci_batch *out) {
    if (!out) return fail(CI_E_INVAL, "out is NULL");
    *out = nullptr;
    if (max_items < 1 || max_items > (1u << 24)) return fail(CI_E_INVAL, "max_items must be in [1, 2^24]");
    ci_batch_s *b = new (std::nothrow) ci_batch_s();
    if (!b) return fail(CI_E_NOMEM, "host allocation failed");
    b->magic = kBatchMagic;
    b->max_items = max_items;
    b->bytes = sizeof(BatchHeader) + sizeof(BatchTask) * (uint64_t)max_items;
    b->geo = batch_geometry(tuned_batch_warps());
    b->tasks.reserve(max_items);
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaMalloc(&b->dev[i], b->bytes);
        if (e == cudaSuccess) e = cudaHostAlloc(&b->host[i], b->bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = build_graph(b, i);
        if (e != cudaSuccess) {
            cudaGetLastError();
            batch_release(b);
            return e == cudaErrorMemoryAllocation ? fail(CI_E_NOMEM, "batch queue allocation failed")
                                                  : cuda_fail(e, "batch creation");
        }
    }
    *out = b;
    return CI_OK;
}

ci_status ci_batch_run(ci_batch b, const ci_batch_item *items, uint32_t n_items, void *cuda_stream) {
    if (!b || b->magic != kBatchMagic) return fail(CI_E_STATE, "not a live ci_batch");
    if (n_items > b->max_items) return fail(CI_E_INVAL, "n_items exceeds the batch's max_items");
    if (n_items > 0 && !items) return fail(CI_E_INVAL, "items is NULL");
    std::unordered_set<const void *> seen;
    b->tasks.clear();
    for (uint32_t i = 0; i < n_items; ++i) {
        const ci_batch_item &it = items[i];
        if (!valid_handle(it.states)) return fail(CI_E_STATE, "item " + std::to_string(i) + ": not a live handle");
        if (!seen.insert(it.states).second)
            return fail(CI_E_INVAL, "item " + std::to_string(i) + ": a handle may appear once per batch");
        const ci_states_s &h = *it.states;
        const uint64_t n = it.n_per_stream;
        if (it.sink == CI_SINK_WRITTEN) {
            if (n > 0 && !it.out_dev) return fail(CI_E_INVAL, "item " + std::to_string(i) + ": out_dev is NULL");
            if (n > 0 && (h.S > UINT64_MAX / n || it.out_capacity_u32 < h.S * n))
                return fail(CI_E_INVAL, "item " + std::to_string(i) + ": out_capacity_u32 < n_streams * n");
        } else if (it.sink == CI_SINK_QC || it.sink == CI_SINK_DIGEST) {
            if (n > 0 && !it.aux_dev) return fail(CI_E_INVAL, "item " + std::to_string(i) + ": aux_dev is NULL");
            if (it.sink == CI_SINK_QC && (n & 1ull))
                return fail(CI_E_INVAL, "item " + std::to_string(i) + ": quarter-circle sink needs an even length");
        } else {
            return fail(CI_E_INVAL, "item " + std::to_string(i) + ": unknown sink");
        }
        if (n == 0) continue;
        b->tasks.push_back(make_task(h, n, it.sink, it.out_dev, it.aux_dev, n, 0));
    }
    const cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    return check_epilogue(cs, batch_launch_tasks(b, b->tasks.data(), (uint32_t)b->tasks.size(), cs));
}

ci_status ci_batch_destroy(ci_batch b) {
    if (!b) return CI_OK;
    if (b->magic != kBatchMagic) return fail(CI_E_STATE, "not a live ci_batch");
    batch_release(b);
    return CI_OK;
}

}  // extern "C"

// ------------------------------------------- allocation-free batched launch
// For callers that must not allocate device memory (see ci_batch_run_noalloc
// in ci_prng.h).  The work queue lives in a fixed, file-scope device array;
// the host stages it in fixed, file-scope host arrays.

namespace {

constexpr uint32_t kNoAllocMaxItems = CI_NOALLOC_MAX_ITEMS;
constexpr size_t kNoAllocBytes = sizeof(BatchHeader) + sizeof(BatchTask) * kNoAllocMaxItems;
constexpr int kNoAllocMaxDevices = 64;

// Per-device state of the set-up: the device address of the queue array and
// the launch geometry, found on the first call made with that device current.
struct NoAllocDevice {
    void *queue;
    BatchGeometry geo;
};

std::mutex g_noalloc_mu;                                   // serialises host-side staging
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];           // zero-initialised
alignas(64) unsigned char g_noalloc_host[kNoAllocBytes];    // header + tasks, staged here
BatchTask g_noalloc_tasks[kNoAllocMaxItems];
const void *g_noalloc_seen[kNoAllocMaxItems];

}  // namespace

// The queue: header (with the cursor) followed by up to kNoAllocMaxItems tasks.
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_queue[kNoAllocBytes];

extern "C" ci_status ci_batch_run_noalloc(const ci_batch_item *items, uint32_t n_items, void *cuda_stream) {
    if (n_items > kNoAllocMaxItems)
        return fail(CI_E_INVAL, "ci_batch_run_noalloc takes at most CI_NOALLOC_MAX_ITEMS (1024) items");
    if (n_items > 0 && !items) return fail(CI_E_INVAL, "items is NULL");
    cudaStream_t cs = static_cast<cudaStream_t>(cuda_stream);
    // The queue upload reads the library's host staging array, which the next
    // call overwrites: a captured upload would replay whatever was staged last.
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(cs, &capture);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (capture != cudaStreamCaptureStatusNone)
        return fail(CI_E_INVAL, "ci_batch_run_noalloc cannot run while its stream is being captured");
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(CI_E_INVAL, "device ordinal above 63");

    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.queue) {  // set-up, once per device, with that device current
        void *addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_noalloc_queue);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc queue");
        d.geo = batch_geometry(8);
        d.queue = addr;
    }

    uint32_t n_tasks = 0;
    for (uint32_t i = 0; i < n_items; ++i) {
        const ci_batch_item &it = items[i];
        if (!valid_handle(it.states)) return fail(CI_E_STATE, "an item's handle is not live");
        for (uint32_t j = 0; j < i; ++j)
            if (g_noalloc_seen[j] == it.states) return fail(CI_E_INVAL, "a handle may appear once per batch");
        g_noalloc_seen[i] = it.states;
        const ci_states_s &h = *it.states;
        const uint64_t n = it.n_per_stream;
        if (it.sink == CI_SINK_WRITTEN) {
            if (n > 0 && !it.out_dev) return fail(CI_E_INVAL, "an item's out_dev is NULL");
            if (n > 0 && (h.S > UINT64_MAX / n || it.out_capacity_u32 < h.S * n))
                return fail(CI_E_INVAL, "an item's out_capacity_u32 < n_streams * n");
        } else if (it.sink == CI_SINK_QC || it.sink == CI_SINK_DIGEST) {
            if (n > 0 && !it.aux_dev) return fail(CI_E_INVAL, "an item's aux_dev is NULL");
            if (it.sink == CI_SINK_QC && (n & 1ull)) return fail(CI_E_INVAL, "quarter-circle sink needs an even length");
        } else {
            return fail(CI_E_INVAL, "an item has an unknown sink");
        }
        if (n == 0) continue;
        g_noalloc_tasks[n_tasks++] = make_task(h, n, it.sink, it.out_dev, it.aux_dev, n, 0);
    }
    if (n_tasks == 0) return CI_OK;

    // Longest first (ties by position, so the order is deterministic); an
    // in-place sort, no temporary buffer.
    for (uint32_t i = 0; i < n_tasks; ++i) g_noalloc_tasks[i].prefix = i;
    std::sort(g_noalloc_tasks, g_noalloc_tasks + n_tasks, [](const BatchTask &a, const BatchTask &b) {
        const double ca = (double)a.n * kind_cost(a.kind), cb = (double)b.n * kind_cost(b.kind);
        return ca != cb ? ca > cb : a.prefix < b.prefix;
    });
    uint64_t units = 0;
    for (uint32_t i = 0; i < n_tasks; ++i) {
        g_noalloc_tasks[i].prefix = units;
        units += g_noalloc_tasks[i].ngroups;
    }
    BatchHeader hdr;
    std::memset(&hdr, 0, sizeof hdr);
    hdr.total_units = units;
    hdr.cursor = 0;  // the upload clears the cursor the previous call left behind
    hdr.n_tasks = n_tasks;
    std::memcpy(g_noalloc_host, &hdr, sizeof hdr);
    std::memcpy(g_noalloc_host + sizeof hdr, g_noalloc_tasks, sizeof(BatchTask) * n_tasks);
    const size_t bytes = sizeof hdr + sizeof(BatchTask) * n_tasks;

    // From pageable memory: returns once the bytes are staged, so the host
    // arrays may be reused by the next call.
    e = cudaMemcpyAsync(d.queue, g_noalloc_host, bytes, cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc queue upload");
    BatchHeader *dhdr = static_cast<BatchHeader *>(d.queue);
    const BatchTask *dtasks = reinterpret_cast<const BatchTask *>(static_cast<unsigned char *>(d.queue) + sizeof hdr);
    k_batched<8><<<d.geo.grid, d.geo.block, 0, cs>>>(dhdr, dtasks);
    e = cudaGetLastError();
    return check_epilogue(cs, e == cudaSuccess ? CI_OK : cuda_fail(e, "no-alloc batched kernel launch"));
}
