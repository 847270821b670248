// Host-side structures shared by lm_api.cpp (plain and batched matching) and
// lm_serve.cpp (the serving loop).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lm.h"
#include "lm_internal.h"

namespace lm {

constexpr int MAX_PROFILE_EVENTS = 1024;

// Scratch arrays of one engine (one allocation, carved).
struct Workspace {
    void* block = nullptr;
    size_t bytes = 0;
    uint32_t cap_v = 0, cap_e = 0, cap_c = 0, cap_g = 0;
    // per-vertex arrays (union ids)
    uint32_t* start = nullptr;       // [cap_v] row start (batches; a single graph uses its own offsets)
    uint32_t* gid = nullptr;         // [cap_v] graph of each vertex (batches)
    uint32_t* len[2] = {nullptr, nullptr};   // [cap_v] live row lengths by round parity
    uint32_t* cnbr = nullptr;        // [cap_v] chosen neighbour
    uint32_t* dead = nullptr;        // [cap_v / 32 + 2] matched bit per vertex
    uint32_t* mate = nullptr;        // [cap_v] union result / staging
    uint32_t* bcnt = nullptr;        // [cap_v] finished chunks of long rows
    unsigned long long* bkey = nullptr;  // [cap_v] heaviest surviving key of long rows
    // task lists: four sets, each R [cap_v] and C [cap_c]
    uint2* R[4] = {nullptr, nullptr, nullptr, nullptr};
    uint2* C[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t* B[4] = {nullptr, nullptr, nullptr, nullptr};   // [cap_v] first row of each batch of R
    // live entries (ping-pong), union entry space
    uint64_t* key[2] = {nullptr, nullptr};   // [cap_e]
    uint32_t* nbr[2] = {nullptr, nullptr};   // [cap_e]
    // per-graph tables (batches / serving)
    SegIn* segs = nullptr;           // [cap_g]
    uint32_t* gvbase = nullptr;      // [cap_g + 1] first union vertex of each graph
    uint32_t* gebase = nullptr;      // [cap_g] first union entry of each graph
    const uint32_t** goff = nullptr; // [cap_g] each graph's row offsets
    uint32_t* grounds = nullptr;     // [cap_g] rounds per graph
    uint32_t* glive = nullptr;       // [cap_g] live rows per graph
    uint32_t** gdst = nullptr;       // [cap_g] result destination per graph
    unsigned long long* gmatched = nullptr;  // [cap_g] matched vertices per graph
};

// Device state + workspace + the stream they are used on.
constexpr size_t ARG_AREA = 1 << 16;  // bytes of kernel arguments uploaded per call / step
struct Engine {
    int device = 0;
    cudaStream_t stream = nullptr;
    DevState* st = nullptr;          // device control block
    DevState* st_host = nullptr;     // pinned mirror
    void* pinned = nullptr;          // pinned staging for tables
    size_t pinned_bytes = 0;
    char* dargs = nullptr;           // [ARG_AREA] kernel arguments (device)
    char* hargs = nullptr;           // [ARG_AREA] their pinned staging
    void* graph = nullptr;           // executable job graph (device-driven round loop)
    void* cblock = nullptr;          // contraction scratch (grown on demand)
    size_t cbytes = 0;
    cudaEvent_t staged = nullptr;    // recorded after a queued job's uploads from pinned staging
    bool staged_pending = false;
    void* egraph = nullptr;          // the same for the edge-centric path
    LaunchCfg cfg;                   // launch parameters of the next jobs
    LaunchCfg graph_cfg;             // the ones `graph` was built with
    Workspace ws;
    int sweep_grid = 0, vertex_grid = 0;
};

struct ServeState;

}  // namespace lm

struct lm_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint32_t max_slots = 0;
    uint32_t flags = 0;
    bool poisoned = false;
    std::string last_error;
    lm::Engine eng;
    cudaEvent_t ev[lm::MAX_PROFILE_EVENTS];
    int nev = 0;
    bool ev_ready = false;
    std::mutex call_mu;              // serialises calls on the context's engine
    std::mutex err_mu;
    lm::ServeState* serve = nullptr;
    // the context's own stream-ordered memory pool (graph arrays, graph-build
    // staging): memory a destroyed graph frees stays mapped for the next one
    cudaMemPool_t pool = nullptr;
    // upload of a host edge list in chunks on its own stream, each chunk's degree
    // count on the context's stream while the next chunk is in flight
    cudaStream_t up = nullptr;
    cudaEvent_t up_ev = nullptr;
    // limits of every match (lm_set_limits): a round cap (0 = none beyond m + 2)
    // and a time limit in ns (0 = LOOP_LIMIT_NS)
    uint32_t lim_rounds = 0;
    uint64_t lim_ns = 0;
    // host-side fault injection read from LM_FAULT at lm_create: the next
    // fault_alloc device allocations fail as out of memory (-1: all of them)
    std::atomic<int64_t> fault_alloc{0};
};

// A device graph (Sec. 2.1 representation): per-vertex offsets V into the
// adjacency array A, whose entries carry the neighbour and a word with the
// order-preserving image of the edge weight and the edge index, plus the
// edge records E (both endpoints of every edge).
struct lm_graph {
    lm_ctx* ctx = nullptr;
    uint32_t n = 0, m = 0, nrows = 0, nent = 0, ntiles = 0;
    void* block = nullptr;
    size_t bytes = 0;
    uint32_t* off = nullptr;         // [n + 1] row offsets of all vertices
    uint32_t* vid = nullptr;         // [nrows] vertices with at least one edge (the rows)
    uint32_t* rdeg = nullptr;        // [nrows] their degrees
    uint32_t* roff = nullptr;        // [nrows + 1] entry offset of each row
    uint32_t* tmap = nullptr;        // [ntiles + 1] row holding entry t * TILE0 (round-0 tiles)
    uint32_t* rbits = nullptr;       // [ntiles * TILE0 / 32 + 8] row-start bit per entry
    uint4* tdesc = nullptr;          // [ntiles] round-0 tile descriptors
    uint32_t* nbr = nullptr;         // [2m] neighbour of each entry
    uint64_t* pk = nullptr;          // [2m] ord(weight) << 32 | edge index, per entry
    uint64_t* edges = nullptr;       // [m] edge records eu | ev << 32
    uint32_t* eword = nullptr;       // [m] ord(weight) of each edge (edge-centric path)
};

namespace lm {

int fail(lm_ctx* ctx, int code, const char* fmt, ...);
// true when fault injection (LM_FAULT=alloc[:N]) makes the next device allocation fail
bool fault_alloc(lm_ctx* ctx);
// round cap and time limit (ns) of a job over `nedges` edges on this context
void job_limits(const lm_ctx* ctx, uint32_t nedges, uint32_t* max_rounds, unsigned long long* limit_ns);
int cuda_fail(lm_ctx* ctx, cudaError_t e, const char* where);
bool is_device_ptr(const void* p);
uint64_t splitmix64_first(uint64_t seed);
SegIn seg_of(const lm_graph* g, uint64_t seed, uint32_t vbase, uint32_t ebase, uint32_t tile_begin);
// chunk-list capacity for a union entry space of `ne` entries: every row longer
// than RMAX adds at most one partial chunk to its ne / CHUNK full ones
inline uint32_t chunks_cap(uint64_t ne, const LaunchCfg& c) {
    return (uint32_t)(ne / (1u << c.chunk_shift) + ne / (c.rmax + 1) + 64);
}

int engine_init(lm_ctx* ctx, Engine& e, cudaStream_t stream);
void engine_free(Engine& e);
int ensure_ws(lm_ctx* ctx, Engine& e, uint32_t nv, uint32_t ne, uint32_t ng);
int ensure_pinned(lm_ctx* ctx, Engine& e, size_t bytes);

// list set `k` of an engine (device counters in DevState::lcnt[k])
Lists lists_of(Engine& e, int k);
// per-vertex arrays of a job whose rows start at `start` (NULL: the workspace's)
VertexArrays vertex_arrays(Engine& e, uint32_t nvert, const uint32_t* start, bool with_gid, uint32_t* mate);

// The local-max loop over prepared union arrays (see lm_api.cpp).
struct Job {
    VertexArrays va;
    uint32_t nedges = 0;             // total edges (the device loop's round cap)
    uint32_t nseg = 0;               // graphs with edges (segment table already on the device)
    uint32_t ecap = 0;               // union entries
    const uint32_t* vlist = nullptr; // rows: explicit list (single graph) ...
    const uint32_t* rdeg = nullptr;
    uint32_t nvlist = 0;             // ... or, with vlist == NULL, the dense range [0, nvlist)
    uint32_t ntiles = 0;             // round-0 tiles of all graphs
    uint32_t* grounds = nullptr;
    bool async = false;              // return once queued (LM_F_ASYNC): no final state read
};
// Per-kernel CUDA-event timing of one call (LM_F_PROFILE); NULL-safe helpers.
struct Prof {
    lm_ctx* ctx;
    cudaStream_t s;
    bool on;
    int kind[MAX_PROFILE_EVENTS / 2];
    int n = 0;
    uint32_t launches[LM_K_COUNT] = {};
    Prof(lm_ctx* c, cudaStream_t st);
    void begin(int k);
    void end();
    void fill(lm_stats* st);
};
int run_job(lm_ctx* ctx, Engine& e, Job& job, Prof& prof);
// count graphs in the same launches (see lm_api.cpp); rounds[i], matched2[i] per graph
int match_batch(lm_ctx* ctx, Engine& e, const lm_graph* const* gs, uint32_t count, const uint64_t* seeds,
                uint32_t* const* mates, uint32_t* rounds, unsigned long long* matched2, Prof& prof);
int match_one(lm_ctx* ctx, Engine& e, const lm_graph* g, uint64_t seed, uint32_t* mate, bool dev_out, Prof& prof,
              bool async = false);
// the pinned staging (arguments, tables) is free again: the copies a queued
// (asynchronous) job made from it have run
int staging_ready(lm_ctx* ctx, Engine& e);

}  // namespace lm

#define LM_CK(ctx, call)                                               \
    do {                                                               \
        cudaError_t e__ = (cudaError_t)(call);                         \
        if (e__ != cudaSuccess) return lm::cuda_fail(ctx, e__, #call); \
    } while (0)
