/*
 * ci_prng.h -- C ABI of the GB300 chaotic-iterations PRNG library
 * (libci_prng.so).
 *
 * The generator is the one of Bahi, Couturier, Guyeux & Heam, arXiv 1112.5239:
 *   - Eq. (Oplus): x^n = x^{n-1} XOR S^n -- bit k of the 32-bit state x flips
 *     iff bit k of the strategy word S^n is 1 (Sec. 4.2);
 *   - Algorithm 4 (Sec. 6.2): each stream ("thread") draws one word from its
 *     own xor-like generator and XORs in the previous strategies of two
 *     partner streams of its group, chosen through two combination arrays of
 *     size combination_size; the result is the strategy S^n;
 *   - Algorithm 5 (Sec. 9.1): the secure variant, whose own word is assembled
 *     from the low bits of a Blum Blum Shub generator x_{k+1} = x_k^2 mod M,
 *     with sixteen combination arrays of which each stream uses two;
 *   - Sec. 9.2: the chaotic Blum-Goldwasser cryptosystem built on the same
 *     BBS iteration and Eq. (Oplus) (ci_bg_encrypt / ci_bg_decrypt);
 *   - Listing 1 / Algorithm 3: the naive generator the paper starts from
 *     (ci_naive_*).
 *
 * Conventions shared by every call:
 *   - Every function returns a ci_status; nothing throws across the ABI.
 *     On failure ci_last_error() returns a message (per calling thread).
 *   - Device pointers ("_dev") are CUDA global-memory addresses on the current
 *     device; host pointers are ordinary process memory.
 *   - cuda_stream is a cudaStream_t passed as void* (NULL: the legacy default
 *     stream).  Generation calls are asynchronous on that stream: they return
 *     after enqueueing, and the caller synchronises before reading outputs.
 *   - Output layout is stream-major: out[s * n_per_stream + i] is stream s's
 *     (i + 1)-th output of the call, i.e. the state x after its (i + 1)-th
 *     update, for s < n_streams.
 *   - Results depend only on (parameters, stream index, position in the
 *     stream): not on launch shape, batching, or how a stream's length is split
 *     over calls (a call continues exactly where the previous one stopped).
 *     The one exception is CI_VAR_BBS16, Algorithm 5 as printed, whose array
 *     choice and rotation happen per call (see ci_params.variant).
 */
#ifndef CI_PRNG_H
#define CI_PRNG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef int32_t ci_status;
enum {
    CI_OK = 0,          /* success                                          */
    CI_PENDING = 1,     /* ci_poll: request not finished yet                */
    CI_E_INVAL = -1,    /* bad argument (null pointer, size, capacity)      */
    CI_E_NOMEM = -2,    /* device or arena memory exhausted                 */
    CI_E_CUDA = -3,     /* a CUDA runtime call failed                       */
    CI_E_BUSY = -4,     /* server queue full / admission refused            */
    CI_E_TIMEOUT = -5,  /* a bounded wait gave up                           */
    CI_E_STATE = -6,    /* handle of the wrong variant, or freed            */
    CI_E_CANCELED = -7  /* the request was cancelled (ci_cancel)            */
};

/* --------------------------------------------------------------- params */
enum { CI_VAR_XOR = 0, CI_VAR_BBS = 1, CI_VAR_BBS16 = 2 };  /* Alg. 4 / Alg. 5 / Alg. 5 as printed */
enum { CI_XL_XOR128 = 0, CI_XL_XORSHIFT32 = 1, CI_XL_XOR64 = 2 };   /* xor-like of Alg. 4 */

typedef struct {
    int32_t variant;      /* CI_VAR_XOR, CI_VAR_BBS (one 62-bit-modulus BBS per
                             stream, w = 5) or CI_VAR_BBS16 (Algorithm 5 as
                             printed: eight BBS per stream with 16-bit moduli,
                             4 bits per squaring, combination arrays chosen per
                             call, generators rotated at the end of a call --
                             so its outputs depend on how a stream's length is
                             split into calls)                                */
    int32_t xl;           /* xor variant: CI_XL_XOR128 (the 32-bit xor128 the
                             paper uses for Alg. 4, Sec. 6.2), CI_XL_XORSHIFT32
                             (Alg. 2) or CI_XL_XOR64 (the 64-bit xorshift of the
                             Sec. 7 measurements; strategy = low 32 bits of each
                             step); ignored for BBS                           */
    uint32_t comb_size;   /* combination_size C of Alg. 4/5: 1, 2, 4, 8, 16 or
                             32; a group of C streams mixes within itself     */
    uint32_t flags;       /* reserved, must be 0                               */
    uint64_t seed;        /* per-stream state seed (counter-based splitmix64) */
    uint64_t comb_seed;   /* seed of the combination arrays                    */
    uint64_t first_stream;/* global index of this handle's stream 0, a multiple
                             of 32 (0 for a standalone handle): stream s is
                             seeded as global stream first_stream + s, so
                             handles holding consecutive slices of one stream
                             range (e.g. one per GPU) reproduce it exactly   */
    const uint8_t *comb;  /* NULL: derive the arrays from comb_seed.  Else
                             host array of 2*C bytes (xor: comb1 then comb2) or
                             16*C bytes (BBS: array a at comb[a*C]); every
                             entry must be < C.  Copied during the call.      */
} ci_params;

/* Opaque per-parameter-set stream state (the paper's InternalVar...Array,
 * x and the shared-memory slots), resident in device memory between calls. */
typedef struct ci_states_s *ci_states;

/* What a handle holds (filled by ci_states_query). */
typedef struct {
    int32_t variant, xl;
    uint32_t comb_size;
    uint32_t reserved;
    uint64_t n_streams;     /* streams requested                               */
    uint64_t n_lanes;       /* lanes computed: n_streams rounded up to 32      */
    uint64_t state_bytes;   /* size of the device state (export/import size)   */
    void *state_dev;        /* device address of the state                     */
    uint8_t comb[16 * 32];  /* the combination arrays in use (2*C or 16*C)     */
} ci_states_desc;

/* Bytes of device memory a state of n_streams streams needs (layout in
 * ci_export_state).  For callers that place states in their own memory. */
ci_status ci_state_bytes(const ci_params *params, uint64_t n_streams, uint64_t *bytes);

/* Creates a state for n_streams independent streams
 * (1 <= n_streams, first_stream + n_streams <= 2^32)
 * and seeds it on cuda_stream (Sec. 6.1: the paper seeds every thread's
 * xor-like parameters on the host with ISAAC; here lane s takes draws
 * s*2^32 + k of a counter-based splitmix64 of params->seed, k = 0, 1, 2:
 * xor128 words (lo, hi of draw 0, lo, hi of draw 1; all-zero -> first word 1),
 * XORshift word (lo of draw 0, 0 -> 1), x (lo of draw 2) and the shared-memory
 * slot (hi of draw 2).  BBS lanes draw Blum primes p, q in [2^30, 2^31),
 * p = q = 3 mod 4, p != q, by rejection, a seed coprime to M = p q in
 * [2, M), then x and the slot).  Streams are padded to a multiple of 32 lanes;
 * padding lanes are computed but never returned.
 * The library allocates the device memory (cudaMalloc); ci_free_states frees it.
 * Errors: CI_E_INVAL (bad params, n_streams out of range), CI_E_NOMEM,
 * CI_E_CUDA.
 * Fault injection (tests of the error paths; host only): with the environment
 * variable CI_FAULT holding "alloc_fail@N", the N-th state allocation of
 * ci_init_states / ci_init_states_many since CI_FAULT took its current value
 * fails with CI_E_NOMEM before any device call.  The serving loop reads
 * "queue_full@N", "reject_admit@N" and "launch_fail@N" from the same variable
 * (comma-separated) when a server is created (ci_server_create). */
ci_status ci_init_states(const ci_params *params, uint64_t n_streams, void *cuda_stream,
                         ci_states *out);

/* As ci_init_states, but the state lives in caller-owned device memory
 * state_dev (state_bytes >= ci_state_bytes(), 256-byte aligned), which must
 * outlive the handle; ci_free_states then frees only the handle. */
ci_status ci_init_states_at(const ci_params *params, uint64_t n_streams, void *state_dev,
                            uint64_t state_bytes, void *cuda_stream, ci_states *out);

/* Creates n states at once (params[i], n_streams[i]; library-allocated as in
 * ci_init_states) and seeds all of them in ONE kernel launch on cuda_stream:
 * results equal n separate ci_init_states calls.  Worth it for many small
 * states, whose separate seeding launches would run one after another.  On
 * failure no handle is left allocated (out[i] = NULL).  Errors: CI_E_INVAL
 * (with the failing item's index in ci_last_error), CI_E_NOMEM, CI_E_CUDA. */
ci_status ci_init_states_many(const ci_params *params, const uint64_t *n_streams, uint32_t n, void *cuda_stream,
                              ci_states *out);

/* Frees the handle (and its device memory if the library allocated it).
 * The caller must ensure no enqueued call still uses it.  NULL is a no-op. */
ci_status ci_free_states(ci_states states);

/* Fills *out with what the handle holds: parameters, stream and lane counts,
 * the state's size and device address, and the combination arrays in use.
 * Host only; no device call.  Errors: CI_E_STATE (dead handle), CI_E_INVAL
 * (out NULL). */
ci_status ci_states_query(ci_states states, ci_states_desc *out);

/* ---------------------------------------------------------- generation */

/* Algorithm 4 (Sec. 6.2) with Eq. (Oplus): advances every stream of a
 * CI_VAR_XOR state by n_per_stream iterations and writes the outputs to
 * out_dev[s * n_per_stream + i] (uint32, stream-major, caller-owned device
 * memory of out_capacity_u32 elements).  Per iteration and stream:
 * t = xorlike() ^ slot[o1] ^ slot[o2] (partners' previous strategies,
 * o = group base + comb[s % C]); slot[s] = t; x ^= t; output x.
 * Errors: CI_E_STATE (BBS handle), CI_E_INVAL (null output, or
 * out_capacity_u32 < n_streams * n_per_stream), CI_E_CUDA.
 * n_per_stream == 0 is a no-op.  A state of at most one warp group (32
 * streams) per SM is run as time segments, as ci_generate_split does, with
 * identical results; that form allocates a stream-ordered workspace. */
ci_status ci_generate(ci_states states, uint64_t n_per_stream, uint32_t *out_dev,
                      uint64_t out_capacity_u32, void *cuda_stream);

/* Algorithm 5 (Sec. 9.1): the same for a CI_VAR_BBS or CI_VAR_BBS16 state.
 * CI_VAR_BBS16 follows the printed listing: BBS1..BBS8 give one 4-bit chunk
 * each (x <- x^2 mod M_k, M_k = p q of Blum primes in [128, 256)), then
 * shift = BBS3 & 3, t <<= shift, t |= BBS1 & {0,1,3,7}[shift] and the same
 * with BBS7 and BBS2 (12 squarings per output); the arrays are comb[BBS1 & 7]
 * and comb[8 + (BBS2 & 7)] taken when the call starts, and at its end
 * generator k (state and modulus) moves to place k + 1.
 * For CI_VAR_BBS, each strategy word takes ceil(32/w) BBS outputs' low w bits (w = floor(log2 log2 M) = 5
 * for these 62-bit moduli), then twice: shift = BBS & 3; t <<= shift;
 * t |= BBS & {0,1,3,7}[shift] -- 11 modular squarings per output, done with
 * 64x64->128-bit multiplies and Barrett reduction.  The stream's two
 * combination arrays are comb[sel1] and comb[8 + sel2] with sel1 = v & 7,
 * sel2 = (v >> 3) & 7 of its BBS seed v.  A CI_VAR_BBS state is run as
 * time segments, as ci_generate_split does, with identical results, unless
 * its streams alone fill about ten waves of resident warps; so is a
 * CI_VAR_BBS16 state of at most one warp group (32 streams) per SM, within
 * the one call.  That form allocates a stream-ordered workspace.  Errors as ci_generate
 * (CI_E_STATE for an xor handle). */
ci_status ci_generate_bbs(ci_states states, uint64_t n_per_stream, uint32_t *out_dev,
                          uint64_t out_capacity_u32, void *cuda_stream);

/* Generation fused with its consumer (Sec. 7: numbers consumed right after
 * generation, without storage): the call's outputs of each stream are taken
 * in pairs (o0, o1) = (out[2k], out[2k+1]) and mapped to the point
 * (a, b) = (o0 >> 8, o1 >> 8) / 2^24 in [0,1)^2; counts_dev[s] (uint64,
 * caller-owned, n_streams elements) is INCREMENTED by the number of points
 * with a^2 + b^2 < 1 (exact integer test (o0>>8)^2 + (o1>>8)^2 < 2^48).
 * Works for both variants; the state advances exactly as in the written
 * form.  n_per_stream must be even (CI_E_INVAL otherwise).  Narrow states run
 * as time segments (identical counts): xor-like and CI_VAR_BBS16 states as
 * in ci_generate / ci_generate_bbs; CI_VAR_BBS states as in ci_generate_bbs
 * while n_streams * n_per_stream <= 2^29 (the outputs then pass through a
 * stream-ordered scratch and are counted from there), otherwise under about
 * two waves of resident warps. */
ci_status ci_generate_fused_qc(ci_states states, uint64_t n_per_stream, uint64_t *counts_dev,
                               void *cuda_stream);

/* Generation fused with a verification consumer: digest_dev[s] (uint64,
 * caller-owned, n_streams elements) is SET to the Horner digest of stream s's
 * outputs o_0 .. o_{n-1} of this call, D = sum_i o_i K^(n-1-i) mod 2^64 with
 * K = 0xD1342543DE82EF95 (D <- D * K + o_i from D = 0).  No outputs are
 * stored; the state advances as in the written form.  Not a construct of the
 * paper: it lets very large runs be compared without holding their outputs.
 * n_per_stream == 0 is a no-op.  Narrow states run as time segments as in
 * ci_generate_fused_qc (identical digests).
 * Errors: CI_E_STATE, CI_E_INVAL (digest_dev NULL with n > 0), CI_E_CUDA. */
ci_status ci_generate_digest(ci_states states, uint64_t n_per_stream, uint64_t *digest_dev,
                             void *cuda_stream);

/* --------------------------------------------------- batched launches */

/* Where a batch item's outputs go. */
enum {
    CI_SINK_WRITTEN = 0,  /* out_dev[s * n_per_stream + i], as ci_generate        */
    CI_SINK_QC = 1,       /* aux_dev[s] += quarter-circle hits, as the fused call  */
    CI_SINK_DIGEST = 2    /* aux_dev[s] = digest, as ci_generate_digest            */
};

typedef struct {
    ci_states states;           /* handle to advance (xor or BBS: its own variant) */
    uint64_t n_per_stream;      /* outputs per stream (0: item skipped)            */
    int32_t sink;               /* CI_SINK_*                                        */
    int32_t reserved;           /* must be 0                                        */
    uint32_t *out_dev;          /* CI_SINK_WRITTEN: caller-owned device output      */
    uint64_t out_capacity_u32;  /* elements available at out_dev                   */
    uint64_t *aux_dev;          /* CI_SINK_QC / CI_SINK_DIGEST: n_streams uint64    */
} ci_batch_item;

/* A reusable batch launcher: a device work queue with room for max_items
 * requests, pinned host staging, and two instantiated CUDA graphs (queue
 * upload -> one persistent kernel) used alternately, so the host can prepare
 * one batch while the previous one runs.  Allocates device and pinned host
 * memory (cudaMalloc, cudaHostAlloc).  Errors: CI_E_INVAL, CI_E_NOMEM,
 * CI_E_CUDA. */
typedef struct ci_batch_s *ci_batch;
ci_status ci_batch_create(uint32_t max_items, ci_batch *out);

/* Runs every item in ONE launch of the persistent kernel, asynchronously on
 * cuda_stream: each item is the same computation as the single-request call
 * for its variant and sink (identical outputs and final state), requests of
 * uneven stream counts, lengths and variants sharing the GPU.  The work queue
 * holds one entry per item; a unit is (item, warp group of 32 streams, whole
 * length); warps claim units through an atomic cursor, longest-first.
 * A handle may appear at most once per batch.  The call may wait for the
 * batch-before-last on this ci_batch to finish (its staging buffer is reused).
 * Errors: CI_E_STATE (dead batch or handle), CI_E_INVAL (item checks as for
 * the single-request calls, duplicate handle, n_items > max_items),
 * CI_E_CUDA. */
ci_status ci_batch_run(ci_batch batch, const ci_batch_item *items, uint32_t n_items, void *cuda_stream);

/* Waits for the batch's launches to finish and frees it.  NULL is a no-op. */
ci_status ci_batch_destroy(ci_batch batch);

/* Allocation-free batched launch.  The paper has no counterpart: this is a
 * library convenience.  Some callers may not allocate device memory: code
 * that runs while its host framework owns all device memory through its own
 * allocator, real-time paths where an allocation's latency or failure is not
 * acceptable, or code that must not touch the allocator (e.g. inside callbacks
 * of another library).  With their states placed in their own memory
 * (ci_init_states_at) they can run a batch through this call, which calls no
 * cudaMalloc, cudaFree, cudaHostAlloc or any other allocating routine.
 *
 * Same computation and results as ci_batch_run on the same items, in one
 * launch of the same persistent kernel on cuda_stream.  Its work queue (header
 * with the claim cursor, then up to CI_NOALLOC_MAX_ITEMS task entries, about
 * 112 KiB) is a fixed device array inside the library: every GPU that loads
 * the library holds it until the process exits.  Every call shares that
 * array and overwrites it (the upload also resets the cursor the previous call
 * left), so calls that overlap on the GPU race: order them, e.g. issue them on
 * one stream.  The queue is copied from the library's own host memory, so the
 * call waits until work already queued on cuda_stream has started the copy;
 * host-side calls are serialised by a lock.  The first call on a device, made
 * with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and the launch size for that device's SM count.
 * Because each call stages its queue in one host array that the next call
 * overwrites, the call refuses to run on a stream that is being captured into
 * a CUDA graph (a replay would read whatever the latest call staged).
 * Errors: CI_E_INVAL (n_items > CI_NOALLOC_MAX_ITEMS, the stream is being
 * captured, or the item checks of ci_batch_run), CI_E_STATE, CI_E_CUDA. */
#define CI_NOALLOC_MAX_ITEMS 1024
ci_status ci_batch_run_noalloc(const ci_batch_item *items, uint32_t n_items, void *cuda_stream);

/* ------------------------------------------------------------ serving */

/* A serving loop with continuous batching.  A worker thread owns the
 * server's CUDA streams.  Requests queue on submission; at every wave the
 * worker:
 *  - admits pending requests in arrival order while a slot and arena memory
 *    for the request's output (and, for new streams, its state) are free;
 *  - takes the next time slice of every admitted request (slice_xor or
 *    slice_bbs outputs per stream) into one launch of the batched persistent
 *    kernel (a CUDA graph replay);
 *  - keeps up to two waves in flight, so requests that arrive while others
 *    are on the GPU join the next wave;
 *  - admits the next request of a stream set as soon as the request before
 *    it has its last slice queued, so that its first slice runs in the next
 *    wave (waves run in order, so it starts from the state the earlier
 *    request leaves).
 * Slicing a stream over waves is exact: each result equals the one-call
 * result whether the request runs alone or in any mix.  (CI_VAR_BBS16, whose
 * outputs depend on call boundaries, runs each request as one slice: one
 * call.)  Long requests over few streams run instead as one time-parallel
 * split job (see ci_generate_split), up to sixteen at a time, each on its own
 * side stream beside the waves, with the same results.  New stream sets are
 * seeded in one launch per admission pass on another side stream.  Stream
 * state stays resident in the arena between requests; a request may continue
 * the streams of an earlier request. */
typedef struct ci_server_s *ci_server;

typedef struct {
    uint32_t max_slots;     /* requests admitted at once (0: 4096)               */
    uint32_t max_inflight;  /* waves queued on the GPU at once, 1 or 2 (0: 2)    */
    uint64_t slice_xor;     /* outputs per stream per wave, xor (0: 16384)       */
    uint64_t slice_bbs;     /* outputs per stream per wave, BBS (0: 512)         */
    uint64_t split_min_slices;  /* a new request of at most 16 warp groups (512
                               streams) and at least this many slices runs as
                               one time-parallel job (ci_generate_split) instead
                               of slices in waves (0: 16; UINT64_MAX: never;
                               CI_VAR_BBS16 lengths count in BBS slices)          */
} ci_server_config;

typedef struct {
    ci_params params;          /* parameters of NEW streams (ignored when continuing) */
    uint64_t n_streams;        /* new streams (ignored when continuing)               */
    uint64_t n_per_stream;     /* outputs per stream, >= 1                             */
    uint64_t continue_ticket;  /* 0: new streams; else continue the streams of that
                                  earlier ticket (they must not be released)         */
} ci_request;

typedef struct {
    ci_status status;         /* CI_OK once done; an error status if it failed      */
    int32_t reserved;
    uint32_t *out_dev;        /* [n_streams][n_per_stream] uint32 in the arena, valid
                                 until ci_release                                    */
    uint64_t n_streams;
    uint64_t n_per_stream;
    ci_states states;         /* server-owned state of the streams (query/export)   */
    uint64_t submit_ns;       /* CLOCK_MONOTONIC times: submission,                 */
    uint64_t admit_ns;        /*   admission,                                        */
    uint64_t done_ns;         /*   last wave observed complete                       */
} ci_result;

typedef struct {
    uint64_t submitted, admitted, completed, released;
    uint64_t waves, units;            /* launches of the batched kernel, work units  */
    uint64_t arena_bytes, arena_used, arena_peak;
    uint64_t pending, active;
    uint64_t gpu_ns;                  /* summed GPU time of retired waves            */
    uint64_t max_wave_units;          /* largest wave, in work units                 */
    uint64_t host_admit_ns;           /* worker time admitting and seeding           */
    uint64_t host_launch_ns;          /* worker time building and launching waves    */
    uint64_t split_jobs;              /* requests run as time-parallel split jobs    */
} ci_server_stats;

/* Creates a server over caller-owned device memory `arena_dev` of arena_bytes
 * bytes (outputs and stream states are sub-allocated from it; it must outlive
 * the server), on the current device.  cfg may be NULL (defaults).  Starts the
 * worker thread.  Fault injection (host only, read here from the environment
 * variable CI_FAULT, comma-separated): "queue_full@N" makes the N-th
 * submission return CI_E_BUSY, "reject_admit@N" fails the N-th admission with
 * CI_E_NOMEM, "launch_fail@N" treats the N-th wave as not launched (its
 * requests end with CI_E_CUDA once the earlier waves have completed).
 * Errors: CI_E_INVAL, CI_E_NOMEM, CI_E_CUDA. */
ci_status ci_server_create(void *arena_dev, uint64_t arena_bytes, const ci_server_config *cfg, ci_server *out);

/* Queues a request (thread-safe) and returns its ticket (> 0).  Errors:
 * CI_E_INVAL (bad parameters, sizes, unknown or released continue_ticket),
 * CI_E_NOMEM (output plus state can never fit the arena), CI_E_STATE. */
ci_status ci_submit(ci_server server, const ci_request *req, uint64_t *ticket);

/* Cancels a request (thread-safe).  A queued request is dropped.  An
 * admitted one gets no further slices and finishes with CI_E_CANCELED once its
 * slices on the GPU have completed (a request running as one split job, or
 * whose last slice is already queued, completes first; the split job then
 * reports CI_E_CANCELED, the other CI_OK).  A request cancelled or failed
 * after admission leaves its stream set part-way, so later continuations of
 * it fail with CI_E_STATE (the set can still be released).  Cancelling a
 * finished request returns its status.  Errors: CI_E_INVAL (unknown ticket). */
ci_status ci_cancel(ci_server server, uint64_t ticket);

/* Non-blocking: CI_PENDING while queued or running; CI_OK and *result once
 * done; the request's error status if it failed; CI_E_INVAL for an unknown
 * ticket. */
ci_status ci_poll(ci_server server, uint64_t ticket, ci_result *result);

/* Blocks until the ticket is done (or timeout_ms passes: CI_E_TIMEOUT), then
 * behaves as ci_poll. */
ci_status ci_wait(ci_server server, uint64_t ticket, uint32_t timeout_ms, ci_result *result);

/* Frees a done request's output bytes in the arena. */
ci_status ci_release(ci_server server, uint64_t ticket);

/* Frees the stream state created by `ticket` (a request that did not
 * continue another); later continuations of it are rejected.  The state must
 * not be in use by a queued or running request (CI_E_BUSY). */
ci_status ci_release_states(ci_server server, uint64_t ticket);

/* Copies the server's counters (a consistent snapshot taken under its lock)
 * into *out.  Errors: CI_E_STATE (dead server), CI_E_INVAL (out NULL). */
ci_status ci_server_get_stats(ci_server server, ci_server_stats *out);

/* Load generator for measurement: submits reqs[i] when arrival_s[i] seconds
 * have passed since the call started (continues[i] >= 0: continue the streams
 * of request continues[i] of this list, which must come earlier), collects
 * every result into results[i] (tickets[i] gets the ticket) and releases each
 * output as soon as it is done unless hold[i] != 0 (hold may be NULL).
 * Returns when all are done or failed.  Errors: as ci_submit. */
ci_status ci_server_drive(ci_server server, const ci_request *reqs, const double *arrival_s,
                          const int64_t *continues, const uint8_t *hold, uint32_t n, ci_result *results,
                          uint64_t *tickets);

/* Stops the server: requests already admitted finish, requests still queued
 * fail with CI_E_STATE; then frees every stream state and the server.
 * Outputs not yet released are abandoned (the arena is the caller's). */
ci_status ci_server_destroy(ci_server server);

/* -------------------------------------------------- checkpoint / resume */

/* Copies the whole device state (bytes == state_bytes) to host_buf /
 * from host_buf, ordered on cuda_stream (the call waits for the copy).
 * Layout for P = n_lanes lanes:
 *   [0, 512)            partner table u8[16][32]: lane j of a warp mixes with
 *                       lanes table[a][j] (xor: a = 0, 1; BBS: a = sel1, 8+sel2)
 *   then 9 uint32 fields of P lanes each (field f at 512 + 4*f*P):
 *     0..3 xor-like words (xor128 a, b, c, d; XORshift z in field 0; xor64
 *       low word in field 0, high word in field 1),
 *     4 x, 5 slot (last strategy), 6 sel1 | sel2 << 8, 7 p, 8 q
 *   then (CI_VAR_BBS16 only) 16 more uint32 fields: 9..16 the states of
 *     BBS1..BBS8 (each < its modulus), 17..24 their moduli (>= 2, < 2^16);
 *   then (CI_VAR_BBS only) 3 uint64 fields of P lanes: 0 y (canonical
 *     residue, BBS state), 1 M (odd, bit length n <= 62), 2 the Barrett
 *     reciprocal floor(2^(2n+1) / M), shifted left by 61 - n when n <= 61.
 * Importing replaces the state of a handle with the same parameters and
 * n_streams.  Every lane of an imported CI_VAR_BBS state must hold M = p q of
 * 33 to 62 bits (the lengths for which Algorithm 5 takes w = 5 bits per
 * squaring, as the kernels do), y < M and the reciprocal of M; every
 * generator of a CI_VAR_BBS16 state a modulus in [3, 2^16) and a state below
 * it.  The host checks this before copying anything.
 * Errors: CI_E_INVAL (size mismatch, or a lane that breaks those rules; the
 * handle's state is then unchanged), CI_E_CUDA. */
ci_status ci_export_state(ci_states states, void *host_buf, uint64_t bytes, void *cuda_stream);
ci_status ci_import_state(ci_states states, const void *host_buf, uint64_t bytes,
                          void *cuda_stream);

/* ----------------------------------------------------------- autotuning */

/* Launch shape of one generation kernel class.  Shapes change speed only,
 * never results. */
typedef struct {
    uint32_t warps_per_block;  /* 4, 8 or 16 (block of 128, 256 or 512 threads)     */
    uint32_t tile_depth;       /* written outputs: outputs per stream staged in
                                  shared memory per flush, 32 or 64 (64 only for
                                  16-byte-aligned xor-variant outputs)             */
    uint32_t cache_policy;     /* 16-byte-aligned written outputs: 0 streaming
                                  (evict-first) 16-byte stores, 1 write-back
                                  16-byte stores, 2 TMA bulk tensor stores of the
                                  staging tile (xor sources, tile depth 32; falls
                                  back to 0 where TMA's alignment rules fail)     */
    float ms;                  /* time of the tuning problem with this shape (0:
                                  not measured)                                    */
} ci_tune_choice;

/* choice[source][sink]: source 0 xor128, 1 XORshift32, 2 BBS, 3 BBS16, 4 xor64; sink 0 written
 * 16-byte-aligned, 1 written unaligned, 2 quarter-circle, 3 digest. */
typedef struct {
    ci_tune_choice choice[5][4];
    uint32_t batch_warps_per_block;  /* batched persistent kernel (read when a
                                        ci_batch or ci_server is created)        */
    float batch_ms;
} ci_tune_table;

/* Times every allowed shape of every class on representative problems (xor:
 * 2^20 streams x 256 written / x 1024 consumed; BBS: 2^16 streams x 128; a
 * 64-request mixed batch; median of 5 launches each) on cuda_stream, installs
 * the fastest for this process and returns the table.  Allocates and frees its
 * own test states and buffers (about 1.2 GB); takes about a second.  flags
 * must be 0.  Errors: CI_E_INVAL,
 * CI_E_NOMEM, CI_E_CUDA. */
ci_status ci_autotune(uint32_t flags, void *cuda_stream, ci_tune_table *out);

/* Reads / installs the table (e.g. to cache tuning results across runs).
 * ci_tune_set rejects shapes not allowed for their class (CI_E_INVAL). */
ci_status ci_tune_get(ci_tune_table *out);
ci_status ci_tune_set(const ci_tune_table *in);

/* ------------------------------------------------- naive generator */

/* The paper's naive generator (Listing 1 and Algorithm 3, Sec. 5 and
 * Sec. 6.1): every stream (thread) runs Listing 1 on its own state, with no
 * exchange between streams.  One output: x ^= the low and high 32-bit halves
 * of t1, t2, t3, one step each of three xor-likes with 64-bit words, which
 * the paper cites to Marsaglia without printing them: xorshift with five
 * words (t = a ^ a >> 7; shift the words; e = (e ^ e << 6) ^ (t ^ t << 13);
 * output (b + b + 1) e, b the new second word), xor128 (t = a ^ a << 11;
 * shift; d = (d ^ d >> 19) ^ (t ^ t >> 8); output d) and xorwow (t = a ^ a >> 2;
 * shift; e = (e ^ e << 4) ^ (t ^ t << 1); w += 362437; output w + e).
 * The state is caller-owned device memory of ci_naive_state_bytes() bytes
 * (8-byte aligned; P = n_streams rounded up to 32: fifteen uint64 fields of P
 * lanes -- xorshift words 0-4, xor128 words 5-8, xorwow words 9-13, the Weyl
 * counter 14 -- then the uint32 field x).  ci_naive_init seeds stream s from
 * the counter-based draws of stream first_stream + s (the paper uses ISAAC on
 * the host): draws 0-4 xorshift, 5-8 xor128, 9-13 xorwow, 14 the counter, the
 * low half of 15 x.  ci_naive_generate advances every stream by n_per_stream
 * outputs into out_dev[s * n_per_stream + i] (uint32, caller-owned, at least
 * n_streams * n_per_stream elements); a call continues where the last one
 * stopped.  Both are asynchronous on cuda_stream.
 * Errors: CI_E_INVAL (n_streams outside [1, 2^32], first_stream + n_streams
 * above 2^32, NULL or short buffers, unaligned state), CI_E_CUDA. */
ci_status ci_naive_state_bytes(uint64_t n_streams, uint64_t *bytes);
ci_status ci_naive_init(uint64_t n_streams, uint64_t seed, uint64_t first_stream, void *state_dev,
                        uint64_t state_bytes, void *cuda_stream);
ci_status ci_naive_generate(void *state_dev, uint64_t n_streams, uint64_t n_per_stream, uint32_t *out_dev,
                            uint64_t out_capacity_u32, void *cuda_stream);

/* ---------------------------------------------- time-parallel generation */

/* Not a construct of the paper: one call of n_per_stream iterations cut into
 * n_segments time segments that run concurrently, with outputs, sink results
 * and the final state IDENTICAL to the sequential call (ci_generate /
 * ci_generate_bbs for CI_SINK_WRITTEN, ci_generate_fused_qc for CI_SINK_QC,
 * ci_generate_digest for CI_SINK_DIGEST).  For states with few streams and
 * long lengths, whose sequential chains leave most of the GPU idle.  (Those
 * single-call entry points split states on their own: written CI_VAR_BBS
 * outputs unless the state fills about ten waves of resident warps, BBS
 * consumer sinks likewise up to 2^29 outputs per call and under about two
 * waves above that, xor-like states of at most one warp
 * group per SM, with segments of at least 1024 iterations, and CI_VAR_BBS16
 * states of at most one warp group per SM.)
 * Method: each segment's own generator is jumped ahead (xor-likes: GF(2)
 * matrix powers of their step; BBS: x <- x^(2^(11 k len) mod lcm(p-1, q-1))
 * mod M), the segments run from a zero mixing state, a per-warp scan restores
 * their true starts from the linearity of Algorithm 4/5's mixing and Eq.
 * (Oplus) over the lanes, and the segments run again from those starts into
 * the sink (written BBS-source outputs are corrected in place instead: the
 * homogeneous part is XORed in, two shuffles per output; their consumer sinks
 * take the same written form into a scratch of up to 2^29 outputs, then count
 * or digest it, so the squarings run once; from 12 warp groups
 * per SM on, inside the generation launch, each segment's correction run by
 * the warp that completes the last of its two inputs, the segment's own
 * outputs and its predecessor's true end).  Cost: about twice the generator
 * work (once for BBS-source outputs written, or counted through the
 * scratch), spread over up to n_segments times more warps.
 * out_dev: uint32 outputs (CI_SINK_WRITTEN, out_capacity elements, layout as
 * ci_generate) or uint64[n_streams] (counts INCREMENTED for CI_SINK_QC,
 * digests SET for CI_SINK_DIGEST; out_capacity ignored).  n_segments == 0
 * picks the count from the GPU size; the count is capped at 8192 and
 * segments hold a multiple of 32 iterations, so small calls run unsplit.
 * n_segments == 1 runs the call unsplit, as ONE launch of the single-call
 * kernel (without the automatic split of the single-call entry points).
 * Allocates a stream-ordered workspace of about n_segments state copies.
 * CI_VAR_BBS16, whose outputs depend on call boundaries, is split within the
 * one call: every segment uses the arrays the call chose at its start, each of
 * the eight generators jumps by its own squaring count (x <- x^(2^(c k len)
 * mod lambda(M)) mod M, lambda from the factors of the 16-bit modulus), and
 * the generators rotate once, at the end.
 * Errors: CI_E_STATE (invalid handle), CI_E_INVAL (unknown sink, NULL output,
 * capacity, odd length for CI_SINK_QC), CI_E_NOMEM, CI_E_CUDA. */
ci_status ci_generate_split(ci_states states, uint64_t n_per_stream, int32_t sink, void *out_dev,
                           uint64_t out_capacity, uint32_t n_segments, void *cuda_stream);

/* ------------------------------------------- chaotic Blum-Goldwasser */

/* The chaotic Blum-Goldwasser cryptosystem of Sec. 9.2: Blum-Goldwasser
 * whose keystream is Eq. (Oplus) iterated on the BBS bits.  n_msgs messages of
 * n_chunks chunks each, every message under its own key; per message i:
 *   x_0 = r^2 mod N;  for k = 0 .. n_chunks-1:
 *     b_k = x_k & (2^w - 1), w = floor(log2 floor(log2 N)) (w = 5 for
 *     2^32 <= N < 2^62),
 *     key_k = S0 ^ b_0 ^ ... ^ b_k,  c_k = m_k ^ key_k,  x_{k+1} = x_k^2 mod N;
 *   y = x_{n_chunks}.
 * Layout (device memory, caller-owned): msg_dev / cipher_dev are uint8,
 * message-major: chunk k of message i at [i * n_chunks + k]; one chunk per
 * byte, its low w bits carrying the message (higher bits pass through the XOR
 * unchanged, as do S0's).  N_dev, r_dev, y_dev: uint64[n_msgs]; S0_dev:
 * uint8[n_msgs] (the paper's S^0, normally < 2^w).  cipher_dev may equal
 * msg_dev (in place).  Requirements: N odd with 3 <= N < 2^62 (else the
 * message is REJECTED: its ciphertext row and y are written as zeros), N the
 * product of two primes = 3 mod 4 and gcd(r, N) = 1 for the ciphertext to be
 * decryptable (not checkable without the factors).  n_rejected_dev (uint32,
 * may be NULL) is INCREMENTED by the number of rejected messages.
 * Asynchronous on cuda_stream.  n_msgs == 0 is a no-op; n_chunks == 0 still
 * writes y = r^2 mod N.  Fastest when n_chunks is a multiple of 32 and both
 * chunk buffers are 16-byte aligned (each thread then moves its message's
 * chunks 32 at a time); any other size or alignment gives the same result.
 * Errors: CI_E_INVAL (a null array, n_msgs * n_chunks overflowing), CI_E_CUDA. */
ci_status ci_bg_encrypt(uint64_t n_msgs, uint64_t n_chunks, const uint64_t *N_dev, const uint8_t *S0_dev,
                        const uint64_t *r_dev, const uint8_t *msg_dev, uint8_t *cipher_dev, uint64_t *y_dev,
                        uint32_t *n_rejected_dev, void *cuda_stream);

/* Decryption (Sec. 9.2) with the private key (p, q), N = p q: x_0 is the
 * square root of y taken n_chunks times, by y^(((p+1)/4)^n_chunks) mod p and
 * likewise mod q, joined by the Chinese remainder theorem; then the keystream
 * of ci_bg_encrypt is regenerated and m_k = c_k ^ key_k.  p_dev, q_dev, y_dev:
 * uint64[n_msgs]; S0_dev, cipher_dev, msg_dev as for encryption (msg_dev may
 * equal cipher_dev).  A key is REJECTED (message row written as zeros,
 * n_rejected_dev incremented) unless p != q are primes = 3 mod 4 below 2^32
 * with p q < 2^62 (primality by Miller-Rabin with bases 2, 7, 61, exact there).
 * n_msgs == 0 or n_chunks == 0 is a no-op.  Errors as ci_bg_encrypt. */
ci_status ci_bg_decrypt(uint64_t n_msgs, uint64_t n_chunks, const uint64_t *p_dev, const uint64_t *q_dev,
                        const uint8_t *S0_dev, const uint64_t *y_dev, const uint8_t *cipher_dev, uint8_t *msg_dev,
                        uint32_t *n_rejected_dev, void *cuda_stream);

/* --------------------------------------------------------------- misc */

/* Bounds-checked debugging build.  The paper has no counterpart: this stands
 * in for a memory checker.  Built with -DCI_CHECKED (build.py --checked,
 * libci_prng_checked.so), the generation, batched and split kernels check, at
 * the start of each warp's work, that the warp group lies within the state's
 * lanes, that the columns it writes lie within a row of the output, that
 * 16-byte and TMA stores start on aligned columns, that a batched unit lies
 * within its task, and that a split segment index lies within the call's
 * segments.  A failed check records (check id << 56) | index in a status word
 * of the device (allocated on first use; the first failure wins) and the warp
 * skips the guarded work: nothing traps and no out-of-range access is made.
 * Every synchronous entry point that launches those kernels (ci_generate*,
 * ci_generate_split, ci_batch_run, ci_batch_run_noalloc) then waits for its
 * stream, reads and clears the word, and returns CI_E_INVAL naming the check.
 *
 * ci_check_status: waits for cuda_stream, stores the status word in *word
 * (0: no check failed) and clears it.  ci_check_probe: launches one warp whose
 * check fails on purpose (no memory is touched) and returns what the
 * epilogue reports, CI_E_INVAL, so the reporting path can be tested.
 * Errors: CI_E_STATE in the ordinary build (the checks are compiled out
 * there), CI_E_INVAL (word NULL), CI_E_CUDA. */
ci_status ci_check_status(uint64_t *word, void *cuda_stream);
ci_status ci_check_probe(void *cuda_stream);

/* Message for the last failing call on this thread ("" if none). */
const char *ci_last_error(void);

/* Library version, as major * 10000 + minor * 100 + patch. */
uint32_t ci_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CI_PRNG_H */
