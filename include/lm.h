/*
 * lm.h -- C ABI of the GB300 local-max matching library (liblm.so).
 *
 * Computes maximal matchings with the local max algorithm of Birn, Osipov,
 * Sanders, Schulz and Sitchinava, "Efficient Parallel and External Matching"
 * (Sec. 1 defines the algorithm; Sec. 2 the data-parallel phase: candidate
 * selection by a segmented maximum over each vertex's edges, mutual-choice
 * matching, deletion and compaction of the edge set, repeated until no edge
 * is left).
 *
 * Edge order.  Edges are compared by the 64-bit key
 *     K(e) = ord(w_e) << 32 | perm_seed(e)
 * where ord() maps a non-NaN float32 monotonically to uint32 (-0.0 == +0.0)
 * and perm_seed() is a seeded bijection of the 32-bit edge index e (the index
 * of the edge in the caller's edge list).  This total order stands in for the
 * paper's "ties broken by random perturbation" (Sec. 1); it is fixed for the
 * whole call.  With a strict order fixed for the run, local max selects
 * exactly the greedy matching of Sec. 3 under the same order, so the result
 * is unique for a given (graph, seed).
 *     perm_seed(e) = fmix32(fmix32(e ^ k0) ^ k1),
 *     (k0, k1) = low and high 32 bits of SplitMix64(seed) (its first output),
 *     fmix32 = the MurmurHash3 32-bit finaliser.
 *
 * Conventions.
 *   - All functions return LM_OK (0) or an LM_E* code; lm_strerror() names it.
 *   - Vertex ids and edge indices are uint32; n >= 1 unless m == 0 as well;
 *     2*m must fit in 32 bits (m <= 2^31 - 1).
 *   - Pointers are host or device (GPU global memory of the context's
 *     device); where both are accepted the kind is detected with
 *     cudaPointerGetAttributes, and `mem` arguments say which explicitly.
 *   - Calls on one context are ordered on the context's stream and are not
 *     thread-safe with respect to each other, except lm_submit / lm_poll /
 *     lm_wait, which may be called from any thread.
 *   - After an LM_ECUDA error the context is poisoned: every later call on it
 *     returns LM_ECUDA.  LM_ETIMEOUT means a bounded device-side wait gave up;
 *     the result of that call is undefined but the context stays usable.
 */
#ifndef LM_H
#define LM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LM_OK        0
#define LM_EINVAL    1   /* bad argument: null pointer, id >= n, self loop, NaN weight, sizes */
#define LM_ENOMEM    2   /* device or pinned allocation failed, or HBM budget exceeded */
#define LM_EAGAIN    3   /* serving: no admission slot / budget right now (retry later) */
#define LM_ETIMEOUT  4   /* a bounded device wait or lm_wait's timeout expired */
#define LM_ECUDA     5   /* CUDA runtime error; the context is poisoned */
#define LM_ENOTFOUND 6   /* unknown ticket */

#define LM_NIL  0xFFFFFFFFu  /* mate[v] of an unmatched vertex */

#define LM_HOST    0
#define LM_DEVICE  1

/* lm_config.flags */
#define LM_F_PROFILE   1u   /* record CUDA events around every kernel (fills lm_stats timings) */
#define LM_F_EDGE_CENTRIC 2u /* lm_match takes the edge-centric path: every live edge offers its key
                                to both ends with an atomic maximum (the Combining CRCW formulation
                                of Sec. 2) instead of the row-wise segmented maximum; same result */
#define LM_F_RENEW     4u   /* lm_match / lm_batch_match renew the perturbation every round, as the
                                proof of Lemma 1 assumes (Sec. 2, its footnote): round r orders edges
                                by (weight, perm_seed with the halves of the r-th SplitMix64 output of
                                the seed); round 0 is the default order.  The result can differ from
                                the default's when weights tie.  Not with LM_F_EDGE_CENTRIC, and
                                lm_submit refuses it (LM_EINVAL) */
#define LM_F_ASYNC     8u   /* lm_match returns once the match is queued on the context's stream
                                instead of after it completes: mate must be device memory and stats
                                NULL (else LM_EINVAL), and the result is ready when the stream reaches
                                that point (lm_sync, or any later work on the stream).  Device-side
                                errors of queued matches are reported by lm_sync.  Not with
                                LM_F_PROFILE or LM_F_EDGE_CENTRIC; lm_batch_match, lm_submit and
                                lm_autotune stay synchronous */

typedef struct lm_ctx lm_ctx;
typedef struct lm_graph lm_graph;

typedef struct {
    int      device;            /* CUDA device ordinal */
    void*    stream;            /* cudaStream_t the context works on; NULL = the legacy default stream */
    uint64_t hbm_budget_bytes;  /* serving admission budget; 0 = 40 GiB */
    uint32_t max_slots;         /* serving: maximum requests in flight; 0 = 4096 */
    uint32_t flags;             /* LM_F_* */
} lm_config;

#define LM_STATS_ROUNDS 64
/* kernel kinds (index into the per-kind arrays of lm_stats) */
#define LM_K_INIT    0   /* reset of mate / candidate / deletion state */
#define LM_K_SWEEP   1   /* k_sweep: deletion + compaction + next candidates over live rows */
#define LM_K_VERTEX  2   /* k_vertex: mutual-choice match over live rows + task lists */
#define LM_K_CAND    3   /* k_round0: round-0 candidates over the input arrays in tiles */
#define LM_K_OTHER   4   /* cut rows of round 0, loop checks, result conversion, batch set-up */
#define LM_K_TAIL    5   /* k_tail: the last rounds (few live entries) in one CTA, no launch per round */
#define LM_K_COUNT   6

typedef struct {
    uint32_t rounds;                        /* local-max iterations performed */
    uint32_t launches;                      /* kernels launched by the call */
    uint64_t matched;                       /* |M| */
    uint64_t round_m[LM_STATS_ROUNDS];      /* live edges at the start of round r (r < 64) */
    uint64_t round_n[LM_STATS_ROUNDS];      /* live vertices at the start of round r (r < 64) */
    /* filled only with LM_F_PROFILE: */
    double   kernel_ms[LM_K_COUNT];         /* summed device time per kernel kind */
    uint32_t kernel_launches[LM_K_COUNT];   /* launches per kernel kind */
    double   total_ms;                      /* device time from first to last kernel of the call */
} lm_stats;

/* Create a context on cfg->device working on cfg->stream.  *out receives the
 * handle, owned by the caller until lm_destroy.  Errors: LM_EINVAL (null
 * argument, bad device, or flags that cannot go together: LM_F_RENEW or
 * LM_F_ASYNC with LM_F_EDGE_CENTRIC, LM_F_ASYNC with LM_F_PROFILE), LM_ECUDA. */
int  lm_create(const lm_config* cfg, lm_ctx** out);

/* Destroy a context: waits for its stream, stops the serving thread, frees
 * every device / pinned buffer it owns.  Graphs created on it must be
 * destroyed first.  NULL is ignored. */
void lm_destroy(lm_ctx* ctx);

/* Build a device graph from an undirected edge list (Sec. 2.1, "graph
 * representation": offsets V over the vertices, the adjacency array A of
 * (vertex, edge) entries, and per-edge records).  Edge i joins eu[i] and ev[i]
 * with weight w[i]; its index i is the edge id used by perm_seed.  Parallel
 * edges are allowed.
 *   n, m    : vertex and edge counts (m may be 0; 2*m < 2^32)
 *   eu, ev  : uint32[m] endpoints, each < n, eu[i] != ev[i]
 *   w       : float32[m] weights, any non-NaN value (+-inf and -0.0 allowed)
 *   mem     : LM_HOST or LM_DEVICE, where eu / ev / w live
 * The arrays are copied; the caller keeps ownership.  The graph is immutable
 * and may be matched any number of times, also concurrently through
 * different contexts on the same device.  Errors: LM_EINVAL (null pointer
 * with m > 0, n == 0 with m > 0, endpoint >= n, self loop, NaN weight,
 * m > 2^31 - 1), LM_ENOMEM, LM_ECUDA. */
int  lm_graph_create(lm_ctx* ctx, uint32_t n, uint32_t m, const uint32_t* eu, const uint32_t* ev,
                     const float* w, int mem, lm_graph** out);

/* Free a graph's device memory (waits for the context's stream).  NULL ok. */
void lm_graph_destroy(lm_graph* g);

/* Vertex count, edge count and device bytes held by a graph. */
int  lm_graph_info(const lm_graph* g, uint32_t* n, uint32_t* m, uint64_t* device_bytes);

/* Maximal matching of g by local max under the order K (Sec. 1, Sec. 2):
 *   mate : uint32[n], caller-owned, host or device memory; on success
 *          mate[v] is v's partner or LM_NIL.
 *   stats: optional (NULL ok).
 * Returns when mate is complete.  Scratch memory is the context's
 * (allocated on first use, reused).  Errors: LM_EINVAL, LM_ENOMEM, LM_ECUDA,
 * LM_ETIMEOUT. */
int  lm_match(lm_ctx* ctx, const lm_graph* g, uint64_t seed, uint32_t* mate, lm_stats* stats);

/* Match `count` independent graphs together: their rounds run in the same
 * kernel launches over the disjoint union of the graphs (each graph keeps its
 * own seed and edge ids, so every result equals lm_match of that graph alone).
 *   g[i], seeds[i], mates[i] (uint32[n_i], host or device), stats[i] (optional
 *   array of `count`, or NULL).  stats[i].rounds is graph i's own round count.
 * Errors: as lm_match. */
int  lm_batch_match(lm_ctx* ctx, const lm_graph* const* g, uint32_t count, const uint64_t* seeds,
                    uint32_t* const* mates, lm_stats* stats);

/* Serving: queue a matching request and return at once with a ticket.  A
 * scheduler thread of the context admits requests while their device
 * footprint fits the HBM budget and a slot is free, and runs rounds of all
 * admitted requests together (a request joins between rounds).  mate
 * (uint32[n], host or device) must stay valid until the request completes;
 * the graph must outlive it.  Errors: LM_EINVAL, LM_EAGAIN (queue full),
 * LM_ENOMEM (the request alone exceeds the budget), LM_ECUDA. */
int  lm_submit(lm_ctx* ctx, const lm_graph* g, uint64_t seed, uint32_t* mate, uint64_t* ticket);

/* *done = 1 once the request's mate is complete (then stats, if non-NULL, is
 * filled and the ticket is released), else 0.  Errors: LM_ENOTFOUND, or the
 * request's own error code. */
int  lm_poll(lm_ctx* ctx, uint64_t ticket, int* done, lm_stats* stats);

/* Block until the request completes or timeout_ms passes (LM_ETIMEOUT; the
 * ticket stays valid).  Does not release the ticket: call lm_poll after. */
int  lm_wait(lm_ctx* ctx, uint64_t ticket, uint32_t timeout_ms);

/* Limits of every later lm_match / lm_batch_match on the context (and of served
 * requests that run alone).  Sec. 2 bounds the rounds of local max by O(log m)
 * only in expectation; with a fixed order a graph can need Theta(n) rounds (a
 * path with monotone weights), so a caller who must bound how long the GPU is
 * held sets either limit:
 *   max_rounds     the match gives up with LM_ETIMEOUT once it has run more than
 *                  this many rounds without emptying the edge set (0 = no cap
 *                  beyond m + 2, which a match never reaches: every round matches
 *                  the heaviest live edge).  Checked after every second round,
 *                  so up to one round more may run.
 *   time_limit_ms  the match gives up with LM_ETIMEOUT once its rounds have run
 *                  longer than this (0 = 120 s).  Checked with the cap.
 * A match that gives up leaves mate undefined; the context stays usable.
 * Errors: LM_EINVAL (null ctx). */
int  lm_set_limits(lm_ctx* ctx, uint32_t max_rounds, uint32_t time_limit_ms);

/* Fault injection for tests of the error paths (read by lm_create from the
 * environment; nothing on the GPU is made to fail):
 *   LM_FAULT=alloc      every device allocation the new context makes after
 *                       lm_create fails as out of memory (calls return LM_ENOMEM)
 *   LM_FAULT=alloc:N    only the next N of them fail. */

/* Launch parameters of a context's matching and contraction paths (the paper
 * has no counterpart; they only affect speed, never the result):
 *   rmax               rows with at most this many live entries are swept in
 *                      batches, one batch to a warp; longer rows are split into
 *                      chunks (1 .. 2^20)
 *   chunk              entries per chunk of a long row (a power of two, 2^8 .. 2^20)
 *   batch              a batch ends after 32 rows, or where its entries cross a
 *                      multiple of `batch` (so it holds at most rmax + batch
 *                      entries); a power of two, 2^6 .. 2^20, or 0 = 32 rows only
 *   sweep_ctas_per_sm  CTAs per SM of the sweep kernel (0 = as many as fit, at most 16)
 *   vertex_ctas_per_sm CTAs per SM of the vertex pass (0 = 4, at most 4)
 *   contract_bits      lm_contract: the low bits of each edge's pair hash that its
 *                      sort orders by (8, 16, 24 or 32), the buckets of equal low bits
 *                      then searched for repeated hashes in shared memory; 0 = by
 *                      size (as few bytes as leave about 2048 edges to a bucket)
 *   ms                 lm_autotune only: median time of one call with these parameters
 * Defaults: rmax 1024, chunk 1024, sweep 0, vertex 4, batch 512, contract_bits 0.
 * The serving thread takes the context's parameters when it starts (first lm_submit). */
typedef struct lm_tuning {
    uint32_t rmax;
    uint32_t chunk;
    uint32_t sweep_ctas_per_sm;
    uint32_t vertex_ctas_per_sm;
    uint32_t batch;
    uint32_t contract_bits;
    double   ms;
} lm_tuning;

/* Current launch parameters of the context (ms = 0). */
int  lm_get_tuning(const lm_ctx* ctx, lm_tuning* out);

/* Set the launch parameters (ms is ignored).  Errors: LM_EINVAL (out of range). */
int  lm_set_tuning(lm_ctx* ctx, const lm_tuning* t);

/* Autotuner: times a fixed set of candidate launch parameters on the caller's
 * own workload -- lm_match of g[0] when count == 1, lm_batch_match of the
 * `count` graphs otherwise (one warm-up call and three timed calls each) --
 * keeps the fastest in the context and returns it in *best (best may be NULL).
 * mates receive the results as in lm_batch_match.  Errors: as lm_batch_match. */
int  lm_autotune(lm_ctx* ctx, const lm_graph* const* g, uint32_t count, const uint64_t* seeds,
                 uint32_t* const* mates, lm_tuning* best);

/* Small graphs without allocation.  The paper has no counterpart: this is a
 * service for callers that must not allocate device memory while they run,
 * for example a host loop that keeps a fixed device footprint or hands all
 * free memory to another allocator, and so cannot let lm_create /
 * lm_graph_create reserve buffers.  It matches one graph of at most
 * LM_NOALLOC_MAX_N vertices and LM_NOALLOC_MAX_M edges by local max under the
 * same order K as lm_match (same seed, same edge ids: the result equals
 * lm_match's on that graph), in one kernel launch on `stream`, and returns
 * once the launch is queued.  Its only scratch is one static device array of
 * LM_NOALLOC_SCRATCH_BYTES in the library itself; nothing is allocated or
 * freed, on the device or on the host.
 *   n, m      : vertex and edge counts, n <= LM_NOALLOC_MAX_N, m <= LM_NOALLOC_MAX_M
 *   eu, ev, w : device arrays uint32[m], uint32[m], float32[m] as in lm_graph_create
 *   mate      : device uint32[n]; when the kernel ends, v's partner or LM_NIL
 *   status    : device uint32[1]; when the kernel ends, 0 = ok, 1 = an edge had an
 *               endpoint >= n, a self loop or a NaN weight, 2 = round cap exceeded
 *               (not expected: every round matches an edge); in both error cases
 *               every mate[v] is LM_NIL
 *   stream    : cudaStream_t, NULL = the default stream
 * Nothing needs to start at zero: each call initialises the scratch it reads.
 * There is one scratch per device, so two calls on one device whose kernels
 * can overlap (different streams, or threads without ordering) race on it and
 * corrupt each other's results: order them, e.g. issue them on one stream.
 * The first call on a device resolves the scratch's address there (with that
 * device current); make that first call before any stream capture on it.  The
 * address is kept for the life of the process: after cudaDeviceReset (or any
 * other teardown of the device's primary context) it is stale and further
 * calls on that device are invalid.
 * All five arrays must be global memory of the current device (checked with
 * cudaPointerGetAttributes; eu, ev, w may be NULL when m = 0, mate when n = 0).
 * Errors (returned at once): LM_EINVAL (n or m beyond the limits, a null
 * pointer, an array that is not memory of the current device, current device
 * index >= 64), LM_ECUDA (the address lookup or the launch failed). */
#define LM_NOALLOC_MAX_N 65536u
#define LM_NOALLOC_MAX_M 262144u
#define LM_NOALLOC_SCRATCH_BYTES (9ull * LM_NOALLOC_MAX_N + 8ull * LM_NOALLOC_MAX_M)
int  lm_match_small_noalloc(uint32_t n, uint32_t m, const uint32_t* eu, const uint32_t* ev, const float* w,
                            uint64_t seed, uint32_t* mate, uint32_t* status, void* stream);

/* Contraction of a matching: the step multilevel graph partitioning repeats on
 * maximal matchings (Sec. 1 names it as the matching's main use; the exact
 * operation is this library's reading).  A matched pair becomes one coarse
 * vertex and an unmatched vertex stays alone; coarse ids number the
 * representatives (unmatched vertices and the smaller end of each pair) in
 * vertex order; a coarse vertex weighs the sum of its members; edges inside a
 * pair vanish; the original edges between two coarse vertices become one
 * coarse edge, placed and oriented as the first of them in input order,
 * weighing their sum (accumulated in double in input order, rounded once to
 * float32).  The output is itself an edge list in lm_graph_create's form, so
 * levels chain.
 *   n, m          vertices and edges; eu, ev, w: device uint32[m], uint32[m], float32[m]
 *   vw            device uint32[n] vertex weights, or NULL (1 each)
 *   mate          device uint32[n]: a matching of the vertex set (partner or LM_NIL)
 *   cmap          device uint32[n] out: coarse id of every vertex
 *   cvw           device uint32[n] out: coarse vertex weights (the first *n_out)
 *   ceu, cev, cw  device uint32[m], uint32[m], float32[m] out: coarse edges (the first *m_out)
 *   n_out, m_out  host out: coarse vertex and edge counts
 * Runs on the context's stream and returns when the outputs are complete; the
 * caller owns every array.  Errors: LM_EINVAL (null or host pointer; mate not
 * a matching of the vertex set; an endpoint >= n; m >= 2^31; n = 2^32 - 1),
 * LM_ENOMEM, LM_ECUDA. */
int  lm_contract(lm_ctx* ctx, uint32_t n, uint32_t m, const uint32_t* eu, const uint32_t* ev, const float* w,
                 const uint32_t* vw, const uint32_t* mate, uint32_t* cmap, uint32_t* cvw, uint32_t* ceu,
                 uint32_t* cev, float* cw, uint32_t* n_out, uint32_t* m_out);

/* Wait for every match queued on the context (LM_F_ASYNC) and report the first
 * device-side error any of them met since the previous lm_sync (LM_ECUDA for a
 * failed index check, LM_ETIMEOUT for a bounded wait that gave up), else LM_OK. */
int  lm_sync(lm_ctx* ctx);

/* Static description of an error code. */
const char* lm_strerror(int code);

/* Last detailed error message of the context (empty if none). */
const char* lm_last_error(const lm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LM_H */
