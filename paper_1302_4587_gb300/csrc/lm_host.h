// Host-side structures shared by lm_api.cpp (plain and batched matching) and
// lm_serve.cpp (the serving loop).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

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
    uint32_t cap_v = 0, cap_e = 0, cap_r = 0, cap_t = 0, cap_g = 0;
    uint32_t* cnbr = nullptr;        // [cap_v] chosen neighbour per vertex
    uint8_t* dead = nullptr;         // [cap_v] matched flag per vertex
    uint32_t* mate = nullptr;        // [cap_v] union result / staging
    uint64_t* key[2] = {nullptr, nullptr};   // [cap_e] live keys (ping-pong)
    uint32_t* nbr[2] = {nullptr, nullptr};   // [cap_e] live neighbours
    uint32_t* off[2] = {nullptr, nullptr};   // [cap_r + 1] live row offsets
    uint32_t* vid[2] = {nullptr, nullptr};   // [cap_r] live row vertex ids
    uint32_t* tilemap = nullptr;     // [cap_t + 1] first row of each tile of the live entries
    uint32_t* lb_desc = nullptr;     // [4 * cap_t] look-back descriptors
    Part* lb_part = nullptr;         // [cap_t] partial row maxima per tile
    SegDesc* segs = nullptr;         // [cap_g] input segments of a sweep
    uint32_t* gvbase = nullptr;      // [cap_g + 1] first union vertex of each graph
    uint32_t* grounds = nullptr;     // [cap_g] rounds per graph
    uint32_t** gdst = nullptr;       // [cap_g] result destination per graph
    unsigned long long* gmatched = nullptr;  // [cap_g] matched vertices per graph
    uint32_t* rows_per = nullptr;    // [cap_g] live rows per graph
};

// Device state + workspace + the stream they are used on.
struct Engine {
    int device = 0;
    cudaStream_t stream = nullptr;
    DevState* st = nullptr;          // device control block
    DevState* st_host = nullptr;     // pinned mirror
    void* pinned = nullptr;          // pinned staging for tables
    size_t pinned_bytes = 0;
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
};

struct lm_graph {
    lm_ctx* ctx = nullptr;
    uint32_t n = 0, m = 0, nrows = 0, nent = 0, ntiles = 0;
    void* block = nullptr;
    size_t bytes = 0;
    uint32_t* off = nullptr;         // [nrows + 1]
    uint32_t* vid = nullptr;         // [nrows]
    uint32_t* nbr = nullptr;         // [2m]
    uint32_t* eid = nullptr;         // [2m]
    uint32_t* ordw = nullptr;        // [2m]
    uint32_t* tilemap = nullptr;     // [ntiles + 1]
};

namespace lm {

int fail(lm_ctx* ctx, int code, const char* fmt, ...);
int cuda_fail(lm_ctx* ctx, cudaError_t e, const char* where);
bool is_device_ptr(const void* p);
uint64_t splitmix64_first(uint64_t seed);
SegDesc seg_of(const lm_graph* g, uint64_t seed, uint32_t vbase, uint32_t tile_begin);
inline uint32_t tiles_of(uint32_t nent) { return (nent + SWEEP_T - 1) / SWEEP_T; }

int engine_init(lm_ctx* ctx, Engine& e, cudaStream_t stream);
void engine_free(Engine& e);
int ensure_ws(lm_ctx* ctx, Engine& e, uint32_t nv, uint32_t ne, uint32_t nr, uint32_t nt, uint32_t ng);
int ensure_pinned(lm_ctx* ctx, Engine& e, size_t bytes);

SweepArgs base_sweep_args(Engine& e, uint32_t nvert);
VertexArgs base_vertex_args(Engine& e, uint32_t nvert, uint32_t* mate);

}  // namespace lm

#define LM_CK(ctx, call)                                               \
    do {                                                               \
        cudaError_t e__ = (cudaError_t)(call);                         \
        if (e__ != cudaSuccess) return lm::cuda_fail(ctx, e__, #call); \
    } while (0)
