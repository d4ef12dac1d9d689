// ci_server.cu -- serving loop with continuous batching over the batched
// persistent kernel (ci_server_* in ci_prng.h).
//
// One worker thread per server owns a CUDA stream and an internal ci_batch
// (two CUDA-graph slots).  Each iteration it retires finished waves, admits
// pending requests (arrival order; slots and arena bytes permitting), and
// launches a wave holding the next time slice of every admitted request.
// Time slices continue each stream's state exactly, so a request's outputs
// do not depend on which other requests share its waves.
#include <cuda_runtime.h>
#include <time.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ci_arena.h"
#include "ci_batch.h"
#include "ci_split.h"
#include "ci_trace.h"

namespace ci {

static uint64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

enum ReqState { RQ_PENDING = 0, RQ_ACTIVE = 1, RQ_DONE = 2, RQ_FAILED = 3, RQ_RELEASED = 4 };

struct Req {
    ci_request r;
    uint8_t comb[16 * 32];
    bool has_comb;
    uint64_t S, L;
    int variant;
    int state;
    ci_status status;
    uint64_t root;  // ticket whose stream state this request advances
    ci_states h;
    uint64_t out_off, out_bytes;
    uint32_t *out;
    uint64_t enq;  // outputs per stream already queued on the GPU
    uint64_t t_submit, t_admit, t_done;
    uint64_t ticket;
    size_t active_idx;  // position in ci_server_s::active while admitted
    BatchTask tmpl;     // this request's queue entry; each wave sets col0 and n
    uint32_t waves;     // waves in flight holding a slice of it
    bool split;         // runs as one split job
    bool cancel;        // ci_cancel was called while it was admitted
    uint64_t handed_to; // the next request of its stream set, admitted before this one finished
    uint64_t early_of;  // while its predecessor runs: the request that handed it the stream set
};

// Requests of at most this many warp groups may run as split jobs, at most
// kSplitSlots of them at a time (measured on the serving mix: 16 slots against
// 4 and 8 cut p99 from 75 % load up, with the same saturation throughput).
constexpr uint64_t kSplitMaxGroups = 16;
constexpr int kSplitSlots = 16;

// A request run whole as one time-parallel split job (captured under the lock).
struct SplitJob {
    uint64_t ticket;
    ci_states h;
    uint32_t *out;
    uint64_t L, K;
};

// Requests of one stream set (a root request and its continuations) run one
// at a time, in submission order: the one queued or running is `busy`; later
// ones wait here and move to the ready queue when it finishes.
struct Chain {
    bool busy = false;
    std::deque<uint64_t> waiting;
};

struct StatesRec {
    ci_states h;
    uint64_t off, bytes;
    bool busy;
    bool released;
    bool poisoned;  // a request that advanced it failed or was cancelled part-way
};

// Host-side fault injection for tests (environment variable CI_FAULT, read
// when a server is created): "queue_full@N" makes the N-th submission return
// CI_E_BUSY, "reject_admit@N" fails the N-th admission with CI_E_NOMEM, and
// "launch_fail@N" treats the N-th wave launch as failed (nothing launched),
// several separated by commas.  Nothing reaches the GPU.
struct Faults {
    uint64_t queue_full = 0, reject_admit = 0, launch_fail = 0;
    uint64_t n_submit = 0, n_admit = 0, n_launch = 0;
};

Faults parse_faults(const char *spec) {
    Faults f;
    if (!spec) return f;
    std::string all(spec);
    size_t pos = 0;
    while (pos <= all.size()) {
        const size_t end = std::min(all.find(',', pos), all.size());
        const std::string item = all.substr(pos, end - pos);
        const size_t at = item.find('@');
        if (at != std::string::npos) {
            const std::string kind = item.substr(0, at);
            const uint64_t n = std::strtoull(item.c_str() + at + 1, nullptr, 10);
            if (kind == "queue_full") f.queue_full = n;
            if (kind == "reject_admit") f.reject_admit = n;
            if (kind == "launch_fail") f.launch_fail = n;
        }
        pos = end + 1;
    }
    return f;
}

struct Wave {
    cudaEvent_t ev;
    cudaEvent_t start;
    std::vector<uint64_t> finishing;
    std::vector<uint64_t> members;
};

}  // namespace ci

using namespace ci;

struct ci_server_s {
    uint32_t magic;
    int device;
    char *arena_base;
    Arena arena;
    ci_server_config cfg;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Req> reqs;
    std::unordered_map<uint64_t, StatesRec> states;
    std::deque<uint64_t> pending;    // new stream sets, arrival order
    std::deque<uint64_t> ready;      // continuations whose stream set is idle, arrival order
    std::unordered_map<uint64_t, Chain> chains;
    std::vector<Req *> active;       // element pointers of `reqs` stay valid across rehashing
    bool admit_dirty = true;         // something changed that may let a pending request in
    std::deque<uint64_t> completed;  // feed of ci_server_drive
    bool feed_completed = false;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    cudaStream_t stream = nullptr;       // waves
    cudaStream_t init_stream = nullptr;  // seeding of admitted stream sets, runs beside the waves
    // split jobs: up to kSplitSlots at once beside the waves, each slot with
    // its own stream (worker thread only, apart from creation)
    cudaStream_t split_stream[kSplitSlots] = {};
    bool split_busy[kSplitSlots] = {};
    Wave split_wave[kSplitSlots];
    cudaEvent_t init_last = nullptr;     // the latest seeding pass (split jobs wait for it)
    std::deque<SplitJob> split_queue;
    ci_batch batch = nullptr;
    std::deque<Wave> inflight;       // worker thread only
    std::vector<cudaEvent_t> spare;  // worker thread only
    // batched seeding of the stream sets admitted in one pass: two slots of
    // pinned staging + device task arrays, reused alternately
    InitTask *init_host[2] = {nullptr, nullptr};
    InitTask *init_dev[2] = {nullptr, nullptr};
    cudaEvent_t init_done[2] = {nullptr, nullptr};
    bool init_pending[2] = {false, false};
    int init_slot = 0;
    uint32_t init_n = 0;
    uint64_t init_lanes = 0;
    std::vector<uint64_t> init_tickets;
    ci_server_stats st;
    Faults faults;
};

static constexpr uint32_t kServerMagic = 0x5E2BE200u;

namespace {

bool valid_server(const ci_server s) { return s && s->magic == kServerMagic; }

void finish_request(ci_server_s *s, uint64_t t, ci_status status) {  // under lock
    Req &q = s->reqs[t];
    const bool held_states = q.state == RQ_ACTIVE;  // only an admitted request holds its streams
    const uint64_t next = held_states ? q.handed_to : 0;  // already admitted: the stream set passes to it
    // admitted early and finishing (cancelled) while its predecessor still
    // runs: the predecessor keeps the stream set's turn
    const uint64_t pred = held_states && q.early_of && s->reqs[q.early_of].state == RQ_ACTIVE ? q.early_of : 0;
    q.state = status == CI_OK ? RQ_DONE : RQ_FAILED;
    q.status = status;
    q.t_done = now_ns();
    auto sit = s->states.find(q.root);
    if (held_states && sit != s->states.end()) {
        if (!next && !pred) sit->second.busy = false;
        if (status != CI_OK) sit->second.poisoned = true;  // advanced part-way: continuations fail
    }
    if (status != CI_OK && q.out) {
        s->arena.release(q.out_off, q.out_bytes);
        q.out = nullptr;
    }
    if (held_states) {
        Req *last = s->active.back();
        s->active[q.active_idx] = last;
        last->active_idx = q.active_idx;
        s->active.pop_back();
    }
    if (s->feed_completed) s->completed.push_back(t);
    if (status == CI_OK) s->st.completed++;
    s->admit_dirty = true;
    if (next) {
        // Handed over: the next request holds the stream set's turn already
        // (behind q's own predecessor, if that one still runs).  q can only
        // fail here through its last wave's launch, and then the next request
        // has no slice queued yet: it fails as well.
        Req &n = s->reqs[next];
        n.early_of = pred;
        if (pred) s->reqs[pred].handed_to = next;
        if (status != CI_OK && n.state == RQ_ACTIVE && n.waves == 0) finish_request(s, next, CI_E_STATE);
        return;
    }
    if (pred) {
        s->reqs[pred].handed_to = 0;  // it passes the turn on itself when it finishes
        return;
    }
    Chain &ch = s->chains[q.root];
    if (!ch.waiting.empty()) {
        s->ready.push_back(ch.waiting.front());
        ch.waiting.pop_front();
    } else {
        ch.busy = false;
    }
}

void retire_front(ci_server_s *s) {
    Wave w = std::move(s->inflight.front());
    s->inflight.pop_front();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w.start, w.ev);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.gpu_ns += (uint64_t)(ms * 1e6);
        for (uint64_t t : w.members) {
            Req &q = s->reqs[t];
            if (q.waves) --q.waves;
        }
        for (uint64_t t : w.finishing)
            if (s->reqs[t].state == RQ_ACTIVE) finish_request(s, t, CI_OK);
        for (uint64_t t : w.members) {  // cancelled, and no slice of it left on the GPU
            Req &q = s->reqs[t];
            if (q.cancel && q.waves == 0 && q.state == RQ_ACTIVE) finish_request(s, t, CI_E_CANCELED);
        }
    }
    s->cv_done.notify_all();
    s->spare.push_back(w.ev);
    s->spare.push_back(w.start);
}

// Admission: first continuations whose stream set became idle, then new
// stream sets in arrival order; a request that does not fit the arena stops
// its queue (no overtaking by smaller requests).
bool admit_one(ci_server_s *s, uint64_t t) {  // under lock; false: no room now
    Req &q = s->reqs[t];
    if (s->faults.reject_admit && ++s->faults.n_admit == s->faults.reject_admit) {
        finish_request(s, t, fail(CI_E_NOMEM, "admission rejected (injected fault)"));
        return true;
    }
    const bool cont = q.r.continue_ticket != 0;
    StatesRec *sr = nullptr;
    if (cont) {
        auto sit = s->states.find(q.root);
        if (sit == s->states.end() || sit->second.released || sit->second.poisoned) {
            // its stream set failed, was cancelled part-way or was released
            finish_request(s, t, CI_E_STATE);
            return true;
        }
        sr = &sit->second;
    }
    uint64_t off_out = 0;
    if (!s->arena.alloc(q.out_bytes, &off_out)) return false;
    if (!cont) {
        uint64_t need = 0, off_st = 0;
        ci_params p = q.r.params;
        p.comb = q.has_comb ? q.comb : nullptr;
        ci_state_bytes(&p, q.S, &need);
        if (!s->arena.alloc_high(need, &off_st)) {
            s->arena.release(off_out, q.out_bytes);
            return false;
        }
        ci_states h = nullptr;
        const ci_status rc = prepare_handle(&p, q.S, s->arena_base + off_st, need, false, &h);
        if (rc != CI_OK) {
            s->arena.release(off_out, q.out_bytes);
            s->arena.release(off_st, need);
            finish_request(s, t, rc);
            return true;
        }
        fill_init_task(*h, p.seed, p.first_stream, s->init_lanes, &s->init_host[s->init_slot][s->init_n++]);
        s->init_lanes += h->P;
        s->init_tickets.push_back(t);
        StatesRec r;
        r.h = h;
        r.off = off_st;
        r.bytes = need;
        r.busy = true;
        r.released = false;
        r.poisoned = false;
        s->states[t] = r;
        q.h = h;
    } else {
        sr->busy = true;
        q.h = sr->h;
    }
    q.out_off = off_out;
    q.out = reinterpret_cast<uint32_t *>(s->arena_base + off_out);
    q.state = RQ_ACTIVE;
    q.t_admit = now_ns();
    q.enq = 0;
    q.tmpl = make_task(*q.h, 1, CI_SINK_WRITTEN, q.out, nullptr, q.L, 0);
    q.active_idx = s->active.size();
    s->active.push_back(&q);
    s->st.admitted++;
    return true;
}

void admit(ci_server_s *s) {  // under lock
    if (!s->admit_dirty) return;
    const int slot = s->init_slot;
    if (s->init_pending[slot]) {  // its staging may still be in an upload: try again later
        if (cudaEventQuery(s->init_done[slot]) != cudaSuccess) return;
        s->init_pending[slot] = false;
    }
    s->admit_dirty = false;
    s->init_n = 0;
    s->init_lanes = 0;
    s->init_tickets.clear();
    for (std::deque<uint64_t> *queue : {&s->ready, &s->pending}) {
        while (!queue->empty() && s->active.size() < s->cfg.max_slots) {
            if (!admit_one(s, queue->front())) break;
            queue->pop_front();
        }
    }
    if (s->init_n == 0) return;
    // one upload and one launch seed every stream set admitted in this pass,
    // on the seeding stream, concurrently with the waves in flight; the next
    // wave (the first to use them) waits for it
    cudaError_t e = cudaMemcpyAsync(s->init_dev[slot], s->init_host[slot], sizeof(InitTask) * s->init_n,
                                    cudaMemcpyHostToDevice, s->init_stream);
    if (e == cudaSuccess) e = launch_init_batched(s->init_dev[slot], s->init_n, s->init_lanes, s->init_stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->init_done[slot], s->init_stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->init_last, s->init_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->init_done[slot], 0);  // next wave waits
    if (e != cudaSuccess) {  // the new stream sets of this pass were not seeded: fail them
        cuda_fail(e, "batched state initialisation");
        for (uint64_t t : s->init_tickets) {
            auto sit = s->states.find(t);
            if (sit != s->states.end()) sit->second.released = true;  // continuations of it fail too
            finish_request(s, t, CI_E_CUDA);
        }
        return;
    }
    s->init_pending[slot] = true;
    s->init_slot ^= 1;
}

// Whether an admitted request would run as one split job (see build_wave).
bool split_candidate(const ci_server_s *s, const Req &q) {
    const uint64_t slice = q.variant == CI_VAR_BBS16 ? q.L
                           : q.variant == CI_VAR_BBS ? s->cfg.slice_bbs
                                                     : s->cfg.slice_xor;
    const uint64_t measure = q.variant == CI_VAR_BBS16 ? s->cfg.slice_bbs : slice;
    return (q.S + 31) / 32 <= kSplitMaxGroups && q.L / measure >= s->cfg.split_min_slices;
}

// Early admission of the next request of q's stream set (under lock): only
// for a request that runs in waves (a split job runs on its own stream, which
// would not wait for q's last wave), with a slot and arena room free now.
// Not when its admission could fail the request (a released or poisoned
// stream set, the injected admission fault): that would pass the stream
// set's turn on while q still runs.
void handover(ci_server_s *s, Req &q) {
    if (q.split || q.cancel || q.handed_to || s->faults.reject_admit) return;
    Chain &ch = s->chains[q.root];
    if (ch.waiting.empty() || s->active.size() >= s->cfg.max_slots) return;
    auto sit = s->states.find(q.root);
    if (sit == s->states.end() || sit->second.released || sit->second.poisoned) return;
    const uint64_t nt = ch.waiting.front();
    Req &n = s->reqs[nt];
    if (n.state != RQ_PENDING || split_candidate(s, n)) return;
    ch.waiting.pop_front();
    if (!admit_one(s, nt)) {  // no room now: it is admitted after q finishes, as before
        ch.waiting.push_front(nt);
        return;
    }
    q.handed_to = nt;
    n.early_of = q.ticket;
}

void build_wave(ci_server_s *s, std::vector<BatchTask> &tasks, Wave &w, std::vector<SplitJob> &splits) {
    // under lock
    for (Req *qp : s->active) {
        Req &q = *qp;
        if (q.enq >= q.L || q.cancel) continue;
        // CI_VAR_BBS16 outputs depend on call boundaries (per-call arrays and
        // rotation): such a request runs as a single slice, i.e. one call
        const uint64_t slice = q.variant == CI_VAR_BBS16 ? q.L
                               : q.variant == CI_VAR_BBS ? s->cfg.slice_bbs
                                                         : s->cfg.slice_xor;
        // long and narrow: the whole request as one split job on the split
        // stream (its serial chain would otherwise take L / slice waves)
        // (CI_VAR_BBS16 runs as one call anyway: its length counts in BBS slices)
        const uint64_t measure = q.variant == CI_VAR_BBS16 ? s->cfg.slice_bbs : slice;
        if (q.enq == 0 && q.tmpl.ngroups <= kSplitMaxGroups && q.L / measure >= s->cfg.split_min_slices) {
            const uint64_t K = split_segments(*q.h, q.L, 0);
            if (K > 1) {
                splits.push_back(SplitJob{q.ticket, q.h, q.out, q.L, K});
                q.enq = q.L;
                q.split = true;
                s->st.split_jobs++;
                continue;
            }
        }
        const uint64_t n = std::min(slice, q.L - q.enq);
        tasks.push_back(q.tmpl);
        BatchTask &tk = tasks.back();
        tk.col0 = q.enq;
        tk.n = n;
        s->st.units += tk.ngroups;
        q.enq += n;
        ++q.waves;
        w.members.push_back(q.ticket);
        if (q.enq == q.L) w.finishing.push_back(q.ticket);
    }
    // A request whose last slice is in this wave hands its stream set to the
    // next request of the set at once (after the loop: admission appends to
    // `active`).  Waves run in order on one stream, so the next request's
    // first slice, in the next wave, starts from the state this one leaves;
    // otherwise it would wait for this wave to finish and then for a wave
    // already queued behind it.
    for (uint64_t t : w.finishing) handover(s, s->reqs[t]);
}

// Split jobs run on their own streams, up to kSplitSlots at a time, so that
// waves keep running beside them (split calls share no queue or lock).  A job waits for the latest seeding pass
// (which covers the seeding of its own streams; a continuation's streams were
// last advanced by a request that had finished before it was admitted).
// Worker thread, no lock held.
bool split_idle(const ci_server_s *s) {
    for (int i = 0; i < kSplitSlots; ++i)
        if (s->split_busy[i]) return false;
    return s->split_queue.empty();
}

void start_split_jobs(ci_server_s *s) {
    for (int slot = 0; slot < kSplitSlots && !s->split_queue.empty(); ++slot) {
        if (s->split_busy[slot]) continue;
        const SplitJob j = s->split_queue.front();
        s->split_queue.pop_front();
        TraceRange trace("server split job");
        while (s->spare.size() < 2) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            s->spare.push_back(ev);
        }
        Wave w;
        w.start = s->spare.back();
        s->spare.pop_back();
        w.ev = s->spare.back();
        s->spare.pop_back();
        w.members.push_back(j.ticket);
        w.finishing.push_back(j.ticket);
        cudaStream_t st = s->split_stream[slot];
        ci_status rc = cudaStreamWaitEvent(st, s->init_last, 0) == cudaSuccess ? CI_OK : CI_E_CUDA;
        if (rc == CI_OK && cudaEventRecord(w.start, st) != cudaSuccess) rc = CI_E_CUDA;
        if (rc == CI_OK)
            rc = split_launch(*j.h, j.L, CI_SINK_WRITTEN, j.out, j.L, 0, nullptr, j.K, st);
        if (rc == CI_OK && cudaEventRecord(w.ev, st) != cudaSuccess) rc = CI_E_CUDA;
        if (rc != CI_OK) {
            std::lock_guard<std::mutex> lk(s->mu);
            finish_request(s, j.ticket, rc);
            s->spare.push_back(w.ev);
            s->spare.push_back(w.start);
            s->cv_done.notify_all();
            continue;
        }
        s->split_wave[slot] = std::move(w);
        s->split_busy[slot] = true;
    }
}

void poll_split_jobs(ci_server_s *s) {
    for (int slot = 0; slot < kSplitSlots; ++slot) {
        if (!s->split_busy[slot] || cudaEventQuery(s->split_wave[slot].ev) != cudaSuccess) continue;
        Wave &w = s->split_wave[slot];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, w.start, w.ev);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->st.gpu_ns += (uint64_t)(ms * 1e6);
            for (uint64_t t : w.finishing) finish_request(s, t, s->reqs[t].cancel ? CI_E_CANCELED : CI_OK);
        }
        s->cv_done.notify_all();
        s->spare.push_back(w.ev);
        s->spare.push_back(w.start);
        w = Wave();
        s->split_busy[slot] = false;
    }
}

void worker_main(ci_server_s *s) {
    cudaSetDevice(s->device);
    std::vector<BatchTask> tasks;
    std::vector<SplitJob> splits;
    for (;;) {
        while (!s->inflight.empty() && cudaEventQuery(s->inflight.front().ev) == cudaSuccess) retire_front(s);
        poll_split_jobs(s);
        start_split_jobs(s);
        tasks.clear();
        Wave w;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop) {  // requests never admitted will not run
                bool any = false;
                while (!s->pending.empty() || !s->ready.empty()) {
                    std::deque<uint64_t> &qq = s->ready.empty() ? s->pending : s->ready;
                    const uint64_t t = qq.front();
                    qq.pop_front();
                    finish_request(s, t, CI_E_STATE);  // may move a waiting continuation to ready
                    any = true;
                }
                if (any) s->cv_done.notify_all();
                if (s->active.empty() && s->inflight.empty() && split_idle(s)) break;
            }
            const uint64_t ta = now_ns();
            {
                TraceRange trace("server admit");
                admit(s);
            }
            const uint64_t tb = now_ns();
            s->st.host_admit_ns += tb - ta;
            if (s->inflight.size() < s->cfg.max_inflight) build_wave(s, tasks, w, splits);
            s->st.host_launch_ns += now_ns() - tb;
            if (tasks.empty() && splits.empty()) {
                if (s->inflight.empty() && split_idle(s))
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(1));
                else
                    s->cv_work.wait_for(lk, std::chrono::microseconds(20));
                continue;
            }
        }
        for (const SplitJob &j : splits) s->split_queue.push_back(j);
        splits.clear();
        start_split_jobs(s);
        if (tasks.empty()) continue;
        while (s->spare.size() < 2) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            s->spare.push_back(ev);
        }
        w.start = s->spare.back();
        s->spare.pop_back();
        w.ev = s->spare.back();
        s->spare.pop_back();
        cudaEventRecord(w.start, s->stream);
        uint64_t wave_units = 0;
        for (const BatchTask &tk : tasks) wave_units += tk.ngroups;
        const uint64_t tl = now_ns();
        ci_status rc;
        if (s->faults.launch_fail && ++s->faults.n_launch == s->faults.launch_fail) {
            rc = fail(CI_E_CUDA, "wave launch failed (injected fault)");
        } else {
            TraceRange trace("server wave");
            rc = batch_launch_tasks(s->batch, tasks.data(), (uint32_t)tasks.size(), s->stream, false);
        }
        const uint64_t tl_end = now_ns();
        if (rc == CI_OK && cudaEventRecord(w.ev, s->stream) != cudaSuccess) rc = CI_E_CUDA;
        if (rc != CI_OK) {
            // earlier waves may still write the members' outputs: let them
            // finish before the outputs' arena bytes are released
            cudaStreamSynchronize(s->stream);
            std::lock_guard<std::mutex> lk(s->mu);
            for (uint64_t t : w.members) {
                Req &q = s->reqs[t];
                q.waves = 0;
                if (q.state == RQ_ACTIVE) finish_request(s, t, rc);
            }
            s->spare.push_back(w.ev);
            s->spare.push_back(w.start);
            s->cv_done.notify_all();
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->st.host_launch_ns += tl_end - tl;
            s->st.waves++;
            s->st.max_wave_units = std::max(s->st.max_wave_units, wave_units);
        }
        s->inflight.push_back(std::move(w));
    }
}

void fill_result(const Req &q, ci_result *r) {
    std::memset(r, 0, sizeof *r);
    r->status = q.state == RQ_DONE || q.state == RQ_RELEASED ? CI_OK : q.status;
    r->out_dev = q.state == RQ_DONE ? q.out : nullptr;
    r->n_streams = q.S;
    r->n_per_stream = q.L;
    r->states = q.h;
    r->submit_ns = q.t_submit;
    r->admit_ns = q.t_admit;
    r->done_ns = q.t_done;
}

ci_status poll_locked(ci_server_s *s, uint64_t ticket, ci_result *result) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(CI_E_INVAL, "unknown ticket");
    const Req &q = it->second;
    if (result) fill_result(q, result);
    if (q.state == RQ_PENDING || q.state == RQ_ACTIVE) return CI_PENDING;
    if (q.state == RQ_FAILED) return q.status;
    return CI_OK;
}

ci_status release_locked(ci_server_s *s, uint64_t ticket) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(CI_E_INVAL, "unknown ticket");
    Req &q = it->second;
    if (q.state != RQ_DONE) return fail(CI_E_BUSY, "request not done (or already released)");
    s->arena.release(q.out_off, q.out_bytes);
    q.out = nullptr;
    q.state = RQ_RELEASED;
    s->st.released++;
    s->admit_dirty = true;
    return CI_OK;
}

ci_status submit_locked(ci_server_s *s, const ci_request *req, uint64_t *ticket) {
    if (s->faults.queue_full && ++s->faults.n_submit == s->faults.queue_full)
        return fail(CI_E_BUSY, "queue full (injected fault)");
    Req q;
    std::memset(&q, 0, sizeof q);
    q.r = *req;
    q.L = req->n_per_stream;
    if (q.L == 0) return fail(CI_E_INVAL, "n_per_stream must be >= 1");
    if (req->continue_ticket) {
        auto it = s->reqs.find(req->continue_ticket);
        if (it == s->reqs.end()) return fail(CI_E_INVAL, "unknown continue_ticket");
        const Req &base = it->second;
        if (base.state == RQ_FAILED) return fail(CI_E_STATE, "continue_ticket failed");
        auto sit = s->states.find(base.root);
        if (sit != s->states.end() && sit->second.released) return fail(CI_E_INVAL, "its streams were released");
        if (sit != s->states.end() && sit->second.poisoned)
            return fail(CI_E_STATE, "its streams were left part-way by a failed or cancelled request");
        q.root = base.root;
        q.S = base.S;
        q.variant = base.variant;
    } else {
        uint64_t need = 0;
        ci_status rc = ci_state_bytes(&req->params, req->n_streams, &need);
        if (rc != CI_OK) return rc;
        q.S = req->n_streams;
        q.variant = req->params.variant;
        if (req->params.comb) {
            const uint32_t n = (req->params.variant == CI_VAR_XOR ? 2u : 16u) * req->params.comb_size;
            std::memcpy(q.comb, req->params.comb, n);
            q.has_comb = true;
        }
    }
    if (q.S > UINT64_MAX / 4 / q.L) return fail(CI_E_INVAL, "n_streams * n_per_stream overflows");
    q.out_bytes = round256(q.S * q.L * 4ull);
    uint64_t st_bytes = 0;
    if (!req->continue_ticket) ci_state_bytes(&req->params, q.S, &st_bytes);
    if (q.out_bytes + round256(st_bytes) > s->arena.size())
        return fail(CI_E_NOMEM, "output plus state larger than the whole arena");
    const uint64_t t = s->next_ticket++;
    if (!req->continue_ticket) q.root = t;
    q.state = RQ_PENDING;
    q.status = CI_PENDING;
    q.t_submit = now_ns();
    q.h = nullptr;
    q.ticket = t;
    s->reqs.emplace(t, q);
    Chain &ch = s->chains[q.root];
    if (!req->continue_ticket) {
        ch.busy = true;
        s->pending.push_back(t);
    } else if (!ch.busy) {
        ch.busy = true;
        s->ready.push_back(t);
    } else {
        ch.waiting.push_back(t);
    }
    s->admit_dirty = true;
    s->st.submitted++;
    *ticket = t;
    return CI_OK;
}

}  // namespace

extern "C" {

ci_status ci_server_create(void *arena_dev, uint64_t arena_bytes, const ci_server_config *cfg, ci_server *out) {
    if (!out) return fail(CI_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!arena_dev || (reinterpret_cast<uintptr_t>(arena_dev) & 255u)) return fail(CI_E_INVAL, "arena_dev must be 256-byte aligned");
    if (arena_bytes < 4096) return fail(CI_E_INVAL, "arena too small");
    ci_server_s *s = new (std::nothrow) ci_server_s();
    if (!s) return fail(CI_E_NOMEM, "host allocation failed");
    s->magic = kServerMagic;
    cudaGetDevice(&s->device);
    s->arena_base = static_cast<char *>(arena_dev);
    s->arena.init(arena_bytes & ~255ull);
    ci_server_config c;
    std::memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    if (c.max_slots == 0) c.max_slots = 4096;
    if (c.max_inflight == 0 || c.max_inflight > 2) c.max_inflight = 2;
    if (c.slice_xor == 0) c.slice_xor = 16384;
    if (c.slice_bbs == 0) c.slice_bbs = 512;
    c.slice_xor = std::max<uint64_t>(4, c.slice_xor & ~3ull);  // keep 16-byte store alignment
    c.slice_bbs = std::max<uint64_t>(4, c.slice_bbs & ~3ull);
    if (c.split_min_slices == 0) c.split_min_slices = 16;  // swept over 4, 8, 16, 32: the lowest p99 at half load
    s->cfg = c;
    s->faults = parse_faults(std::getenv("CI_FAULT"));
    std::memset(&s->st, 0, sizeof s->st);
    s->st.arena_bytes = s->arena.size();
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->init_stream, cudaStreamNonBlocking);
    const bool splits = c.split_min_slices != UINT64_MAX;
    for (int i = 0; i < kSplitSlots && splits && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&s->split_stream[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->init_last, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(s->init_last, s->init_stream);
    if (e == cudaSuccess && splits) e = split_prepare(s->split_stream[0]);
    ci_status rc = e == cudaSuccess ? ci_batch_create(c.max_slots, &s->batch) : CI_E_CUDA;
    if (e != cudaSuccess || rc != CI_OK) {
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->init_stream) cudaStreamDestroy(s->init_stream);
        for (int i = 0; i < kSplitSlots; ++i)
            if (s->split_stream[i]) cudaStreamDestroy(s->split_stream[i]);
        if (s->init_last) cudaEventDestroy(s->init_last);
        delete s;
        return e != cudaSuccess ? cuda_fail(e, "server streams") : rc;
    }
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaHostAlloc(reinterpret_cast<void **>(&s->init_host[i]), sizeof(InitTask) * c.max_slots,
                          cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&s->init_dev[i]), sizeof(InitTask) * c.max_slots);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->init_done[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (int i = 0; i < 2; ++i) {
            if (s->init_host[i]) cudaFreeHost(s->init_host[i]);
            if (s->init_dev[i]) cudaFree(s->init_dev[i]);
            if (s->init_done[i]) cudaEventDestroy(s->init_done[i]);
        }
        ci_batch_destroy(s->batch);
        cudaStreamDestroy(s->stream);
        cudaStreamDestroy(s->init_stream);
        for (int i = 0; i < kSplitSlots; ++i)
            if (s->split_stream[i]) cudaStreamDestroy(s->split_stream[i]);
        cudaEventDestroy(s->init_last);
        delete s;
        return e == cudaErrorMemoryAllocation ? fail(CI_E_NOMEM, "server buffers") : cuda_fail(e, "server buffers");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return CI_OK;
}

ci_status ci_submit(ci_server s, const ci_request *req, uint64_t *ticket) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    if (!req || !ticket) return fail(CI_E_INVAL, "req or ticket is NULL");
    ci_status rc;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return fail(CI_E_STATE, "server is stopping");
        rc = submit_locked(s, req, ticket);
    }
    if (rc == CI_OK) s->cv_work.notify_one();
    return rc;
}

ci_status ci_poll(ci_server s, uint64_t ticket, ci_result *result) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    std::lock_guard<std::mutex> lk(s->mu);
    return poll_locked(s, ticket, result);
}

ci_status ci_wait(ci_server s, uint64_t ticket, uint32_t timeout_ms, ci_result *result) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(CI_E_INVAL, "unknown ticket");
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        const int st = s->reqs[ticket].state;
        return st != RQ_PENDING && st != RQ_ACTIVE;
    });
    if (!ok) return fail(CI_E_TIMEOUT, "request not done within timeout_ms");
    return poll_locked(s, ticket, result);
}

ci_status ci_release(ci_server s, uint64_t ticket) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    std::lock_guard<std::mutex> lk(s->mu);
    return release_locked(s, ticket);
}

ci_status ci_cancel(ci_server s, uint64_t ticket) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    ci_status rc = CI_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end() || it->second.state == RQ_RELEASED) return fail(CI_E_INVAL, "unknown ticket");
        Req &q = it->second;
        if (q.state == RQ_DONE || q.state == RQ_FAILED) return q.status;  // already finished
        if (q.state == RQ_PENDING) {
            Chain &ch = s->chains[q.root];
            auto wit = std::find(ch.waiting.begin(), ch.waiting.end(), ticket);
            if (wit != ch.waiting.end()) {  // behind another request of its stream set
                ch.waiting.erase(wit);
                q.state = RQ_FAILED;
                q.status = CI_E_CANCELED;
                q.t_done = now_ns();
                if (s->feed_completed) s->completed.push_back(ticket);
            } else {  // queued for admission: it holds its stream set's turn
                for (std::deque<uint64_t> *dq : {&s->pending, &s->ready}) {
                    auto qit = std::find(dq->begin(), dq->end(), ticket);
                    if (qit != dq->end()) dq->erase(qit);
                }
                finish_request(s, ticket, CI_E_CANCELED);
            }
        } else {  // admitted
            q.cancel = true;
            if (!q.split && q.waves == 0) finish_request(s, ticket, CI_E_CANCELED);
        }
        rc = CI_OK;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_one();
    return rc;
}

ci_status ci_release_states(ci_server s, uint64_t ticket) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->states.find(ticket);
    if (it == s->states.end() || it->second.released) return fail(CI_E_INVAL, "ticket owns no live stream state");
    if (it->second.busy) return fail(CI_E_BUSY, "stream state in use");
    auto ch = s->chains.find(ticket);
    if (ch != s->chains.end() && ch->second.busy)
        return fail(CI_E_BUSY, "a queued request continues these streams");
    s->arena.release(it->second.off, it->second.bytes);
    s->admit_dirty = true;
    ci_free_states(it->second.h);
    it->second.h = nullptr;
    it->second.released = true;
    return CI_OK;
}

ci_status ci_server_get_stats(ci_server s, ci_server_stats *out) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    if (!out) return fail(CI_E_INVAL, "out is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->arena_used = s->arena.used();
    out->arena_peak = s->arena.peak();
    uint64_t waiting = 0;
    for (const auto &kv : s->chains) waiting += kv.second.waiting.size();
    out->pending = s->pending.size() + s->ready.size() + waiting;
    out->active = s->active.size();
    return CI_OK;
}

ci_status ci_server_drive(ci_server s, const ci_request *reqs, const double *arrival_s, const int64_t *continues,
                          const uint8_t *hold, uint32_t n, ci_result *results, uint64_t *tickets) {
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    if (n > 0 && (!reqs || !arrival_s || !results || !tickets)) return fail(CI_E_INVAL, "NULL argument");
    std::unordered_map<uint64_t, uint32_t> index;
    index.reserve(n * 2 + 1);
    uint32_t done = 0;
    ci_status first_err = CI_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->feed_completed = true;
        s->completed.clear();
    }
    auto drain = [&](std::unique_lock<std::mutex> &lk) {
        while (!s->completed.empty()) {
            const uint64_t t = s->completed.front();
            s->completed.pop_front();
            auto ix = index.find(t);
            if (ix == index.end()) continue;
            Req &q = s->reqs[t];
            fill_result(q, &results[ix->second]);
            if (q.state == RQ_DONE && !(hold && hold[ix->second])) release_locked(s, t);
            ++done;
        }
        (void)lk;
    };
    const uint64_t t0 = now_ns();
    for (uint32_t i = 0; i < n; ++i) {
        const uint64_t due = t0 + (uint64_t)(arrival_s[i] * 1e9);
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(s->mu);
                drain(lk);
            }
            if (now_ns() >= due) break;
            std::this_thread::yield();
        }
        ci_request r = reqs[i];
        if (continues && continues[i] >= 0) {
            if ((uint64_t)continues[i] >= i) return fail(CI_E_INVAL, "continues[i] must refer to an earlier request");
            r.continue_ticket = tickets[continues[i]];
        }
        uint64_t t = 0;
        ci_status rc;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            rc = submit_locked(s, &r, &t);
            if (rc == CI_OK) index[t] = i;
        }
        if (rc != CI_OK) {
            tickets[i] = 0;
            std::memset(&results[i], 0, sizeof results[i]);
            results[i].status = rc;
            if (first_err == CI_OK) first_err = rc;
            ++done;
            continue;
        }
        tickets[i] = t;
        s->cv_work.notify_one();
    }
    {
        std::unique_lock<std::mutex> lk(s->mu);
        while (done < n) {
            drain(lk);
            if (done < n) s->cv_done.wait_for(lk, std::chrono::milliseconds(1));
        }
        s->feed_completed = false;
    }
    return first_err;
}

ci_status ci_server_destroy(ci_server s) {
    if (!s) return CI_OK;
    if (!valid_server(s)) return fail(CI_E_STATE, "not a live server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->init_stream);
    cudaStreamSynchronize(s->stream);
    for (int i = 0; i < kSplitSlots; ++i)
        if (s->split_stream[i]) cudaStreamSynchronize(s->split_stream[i]);
    for (auto &kv : s->states)
        if (!kv.second.released && kv.second.h) ci_free_states(kv.second.h);
    for (cudaEvent_t ev : s->spare) cudaEventDestroy(ev);
    for (int i = 0; i < 2; ++i) {
        cudaFreeHost(s->init_host[i]);
        cudaFree(s->init_dev[i]);
        cudaEventDestroy(s->init_done[i]);
    }
    ci_batch_destroy(s->batch);
    cudaStreamDestroy(s->init_stream);
    cudaStreamDestroy(s->stream);
    for (int i = 0; i < kSplitSlots; ++i)
        if (s->split_stream[i]) cudaStreamDestroy(s->split_stream[i]);
    cudaEventDestroy(s->init_last);
    s->magic = 0;
    delete s;
    return CI_OK;
}

}  // extern "C"
