// Host side of liblm: context, graphs, plain and batched matching (include/lm.h).
//
// Everything on the result path runs on the GPU (lm_kernels.cu); this file
// validates arguments, owns device memory, builds launch arguments, drives
// the round loop and moves results between host and device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "lm_host.h"

using namespace lm;

namespace {

struct DevGuard {  // make the context's device current for a call, restore the caller's afterwards
    int prev = -1;
    bool ok = true;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DevGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One device allocation carved into 256-byte aligned pieces.
struct Carver {
    size_t total = 0;
    struct Item { void** out; size_t bytes; };
    std::vector<Item> items;
    template <class T> void add(T** out, size_t count) {
        const size_t b = align_up(std::max<size_t>(count, 1) * sizeof(T), 256);
        items.push_back({reinterpret_cast<void**>(out), b});
        total += b;
    }
    void assign(void* base) {
        char* p = static_cast<char*>(base);
        for (auto& it : items) { *it.out = p; p += it.bytes; }
    }
};

}  // namespace

// ============================================================ shared helpers
namespace lm {

int fail(lm_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->last_error = buf;
        if (code == LM_ECUDA) ctx->poisoned = true;
    }
    return code;
}

bool fault_alloc(lm_ctx* ctx) {
    if (!ctx) return false;
    int64_t left = ctx->fault_alloc.load();
    while (left != 0) {
        if (left < 0 || ctx->fault_alloc.compare_exchange_weak(left, left - 1)) return true;
    }
    return false;
}

void job_limits(const lm_ctx* ctx, uint32_t nedges, uint32_t* max_rounds, unsigned long long* limit_ns) {
    // every round matches at least the heaviest live edge, so m + 2 rounds never run out
    uint32_t r = nedges + 2;
    if (ctx && ctx->lim_rounds && ctx->lim_rounds < r) r = ctx->lim_rounds;
    *max_rounds = r;
    *limit_ns = (ctx && ctx->lim_ns) ? ctx->lim_ns : LOOP_LIMIT_NS;
}

int cuda_fail(lm_ctx* ctx, cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, LM_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    }
    return fail(ctx, LM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

uint64_t splitmix64_first(uint64_t seed) {
    // SplitMix64 (Steele, Lea, Flood 2014): first output for state `seed`
    uint64_t z = seed + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

SegIn seg_of(const lm_graph* g, uint64_t seed, uint32_t vbase, uint32_t ebase, uint32_t tile_begin) {
    SegIn d;
    memset(&d, 0, sizeof d);
    const uint64_t z = splitmix64_first(seed);
    d.nbr = g->nbr;
    d.pk = g->pk;
    d.edges = g->edges;
    d.roff = g->roff;
    d.rvid = g->vid;
    d.tmap = g->tmap;
    d.rbits = g->rbits;
    d.tdesc = g->tdesc;
    d.m = g->m;
    d.nrows = g->nrows;
    d.nent = g->nent;
    d.ntiles = g->ntiles;
    d.tile_begin = tile_begin;
    d.ebase = ebase;
    d.vbase = vbase;
    d.k0 = (uint32_t)z;
    d.k1 = (uint32_t)(z >> 32);
    d.seed = seed;
    return d;
}

int engine_init(lm_ctx* ctx, Engine& e, cudaStream_t stream) {
    e.device = ctx->device;
    e.stream = stream;
    LM_CK(ctx, cudaMalloc(&e.st, sizeof(DevState)));
    LM_CK(ctx, cudaMallocHost(&e.st_host, sizeof(DevState)));
    memset(e.st_host, 0, sizeof(DevState));
    LM_CK(ctx, cudaMemcpy(e.st, e.st_host, sizeof(DevState), cudaMemcpyHostToDevice));
    LM_CK(ctx, cudaMalloc(&e.dargs, ARG_AREA));
    LM_CK(ctx, cudaMallocHost(&e.hargs, ARG_AREA));
    e.sweep_grid = 0;
    e.vertex_grid = 0;
    return LM_OK;
}

void engine_free(Engine& e) {
    if (e.stream) cudaStreamSynchronize(e.stream);
    else cudaDeviceSynchronize();
    if (e.ws.block) cudaFree(e.ws.block);
    if (e.pinned) cudaFreeHost(e.pinned);
    if (e.st) cudaFree(e.st);
    if (e.st_host) cudaFreeHost(e.st_host);
    if (e.dargs) cudaFree(e.dargs);
    if (e.hargs) cudaFreeHost(e.hargs);
    destroy_job_graph(e.graph);
    destroy_job_graph(e.egraph);
    if (e.staged) cudaEventDestroy(e.staged);
    if (e.cblock) cudaFree(e.cblock);
    cudaGetLastError();
    e = Engine();
}

int ensure_ws(lm_ctx* ctx, Engine& e, uint32_t nv, uint32_t ne, uint32_t ng) {
    Workspace& w = e.ws;
    const uint32_t nc = chunks_cap(ne, e.cfg);
    if (w.block && nv <= w.cap_v && ne <= w.cap_e && nc <= w.cap_c && ng <= w.cap_g) return LM_OK;
    LM_CK(ctx, cudaStreamSynchronize(e.stream));
    Workspace nw;
    nw.cap_v = std::max(nv, w.cap_v);
    nw.cap_e = std::max(ne, w.cap_e);
    nw.cap_c = std::max(nc, w.cap_c);
    nw.cap_g = std::max(std::max(ng, w.cap_g), 1u);
    const size_t V = (size_t)nw.cap_v + 1, E = (size_t)nw.cap_e + 4, C = nw.cap_c, G = nw.cap_g;
    Carver c;
    c.add(&nw.start, V);
    c.add(&nw.gid, V);
    c.add(&nw.len[0], V);
    c.add(&nw.len[1], V);
    c.add(&nw.cnbr, V);
    c.add(&nw.dead, V / 32 + 2);
    c.add(&nw.mate, V);
    c.add(&nw.bcnt, V);
    c.add(&nw.bkey, V);
    for (int k = 0; k < 4; k++) {
        c.add(&nw.R[k], V);
        c.add(&nw.C[k], C);
        c.add(&nw.B[k], V);
    }
    for (int b = 0; b < 2; b++) {
        c.add(&nw.key[b], E);
        c.add(&nw.nbr[b], E);
    }
    c.add(&nw.segs, G);
    c.add(&nw.gvbase, G + 1);
    c.add(&nw.gebase, G);
    c.add(&nw.goff, G);
    c.add(&nw.grounds, G);
    c.add(&nw.glive, G);
    c.add(&nw.gdst, G);
    c.add(&nw.gmatched, G);
    if (w.block) {
        cudaFree(w.block);
        w.block = nullptr;
    }
    void* p = nullptr;
    cudaError_t err = fault_alloc(ctx) ? cudaErrorMemoryAllocation : cudaMalloc(&p, c.total);
    if (err != cudaSuccess) {
        cudaGetLastError();
        e.ws = Workspace();
        return fail(ctx, LM_ENOMEM, "workspace of %zu bytes: %s", c.total, cudaGetErrorString(err));
    }
    c.assign(p);
    nw.block = p;
    nw.bytes = c.total;
    e.ws = nw;
    // long-row slots start at zero (every sweep leaves them at zero)
    LM_CK(ctx, cudaMemsetAsync(e.ws.bcnt, 0, V * sizeof(uint32_t), e.stream));
    LM_CK(ctx, cudaMemsetAsync(e.ws.bkey, 0, V * sizeof(unsigned long long), e.stream));
    return LM_OK;
}

int ensure_pinned(lm_ctx* ctx, Engine& e, size_t bytes) {
    if (e.pinned_bytes >= bytes) return LM_OK;
    LM_CK(ctx, cudaStreamSynchronize(e.stream));
    if (e.pinned) cudaFreeHost(e.pinned);
    e.pinned = nullptr;
    e.pinned_bytes = 0;
    const size_t want = std::max(bytes, (size_t)1 << 16);
    LM_CK(ctx, cudaMallocHost(&e.pinned, want));
    e.pinned_bytes = want;
    return LM_OK;
}

Lists lists_of(Engine& e, int k) {
    Lists l;
    l.R = e.ws.R[k];
    l.C = e.ws.C[k];
    l.B = e.ws.B[k];
    l.capR = e.ws.cap_v;
    l.capC = e.ws.cap_c;
    l.cnt = &e.st->lcnt[k][0];
    return l;
}

VertexArrays vertex_arrays(Engine& e, uint32_t nvert, const uint32_t* start, bool with_gid, uint32_t* mate) {
    VertexArrays va;
    va.start = start ? start : e.ws.start;
    va.len[0] = e.ws.len[0];
    va.len[1] = e.ws.len[1];
    va.cnbr = e.ws.cnbr;
    va.dead = e.ws.dead;
    va.mate = mate;
    va.bcnt = e.ws.bcnt;
    va.bkey = e.ws.bkey;
    va.gid = with_gid ? e.ws.gid : nullptr;
    va.nvert = nvert;
    return va;
}

Prof::Prof(lm_ctx* c, cudaStream_t st) : ctx(c), s(st), on(c && (c->flags & LM_F_PROFILE) && c->ev_ready) {}
void Prof::begin(int k) {
    launches[k]++;
    if (!on || n >= MAX_PROFILE_EVENTS / 2) return;
    kind[n] = k;
    cudaEventRecord(ctx->ev[2 * n], s);
}
void Prof::end() {
    if (!on || n >= MAX_PROFILE_EVENTS / 2) return;
    cudaEventRecord(ctx->ev[2 * n + 1], s);
    n++;
}
void Prof::fill(lm_stats* st) {
    uint32_t tot = 0;
    for (int k = 0; k < LM_K_COUNT; k++) {
        st->kernel_launches[k] = launches[k];
        tot += launches[k];
    }
    st->launches = tot;
    if (!on || n == 0) return;
    for (int i = 0; i < n; i++) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]) == cudaSuccess) st->kernel_ms[kind[i]] += ms;
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[2 * n - 1]) == cudaSuccess) st->total_ms = ms;
    cudaGetLastError();
}

static int check_err(lm_ctx* ctx, Engine& e) {
    const uint32_t err = e.st_host->err;
    if (err & ERR_BOUNDS) return fail(ctx, LM_ECUDA, "device index check failed (index %u)", e.st_host->err_info);
    if (err & ERR_TIMEOUT) return fail(ctx, LM_ETIMEOUT, "a bounded device wait gave up (%u)", e.st_host->err_info);
    return LM_OK;
}

// The local-max loop of one job.  Expects the segment table in e.ws.segs
// and, for batches, the union arrays (start, gid, len[0]) set up.  Round r's
// vertex pass reads list set r & 1 and fills set (r + 1) & 1, which round
// r's sweep consumes; live entries alternate between buffers 1 and 0 (round 0
// reads the graphs' own arrays).  All kernel arguments are uploaded in one
// block; by default an executable graph runs the whole job, its round loop a
// conditional node that repeats while the device has not flagged the edge set
// empty.  With profiling the same launches are issued one by one on the
// stream, with events around each, and the host polls between rounds.
int staging_ready(lm_ctx* ctx, Engine& e) {
    if (!e.staged_pending) return LM_OK;
    LM_CK(ctx, cudaEventSynchronize(e.staged));
    e.staged_pending = false;
    return LM_OK;
}

int run_job(lm_ctx* ctx, Engine& e, Job& job, Prof& prof) {
    Workspace& w = e.ws;
    cudaStream_t s = e.stream;
    if (int rc = staging_ready(ctx, e)) return rc;
    static_assert(sizeof(JobArgs) <= ARG_AREA, "argument area too small");
    JobArgs& A = *reinterpret_cast<JobArgs*>(e.hargs);
    memset(&A, 0, sizeof A);
    A.init.mate = job.va.mate;
    A.init.dead = job.va.dead;
    A.init.dbase = 0;
    A.init.bcnt = job.va.bcnt;
    A.init.bkey = job.va.bkey;
    A.init.n = job.va.nvert;
    job_limits(ctx, job.nedges, &A.init.max_rounds, &A.init.limit_ns);
    A.init.st = e.st;
    auto vargs = [&](VertexArgs& v, int in_set, int out_set, uint32_t par, uint32_t match) {
        v.va = job.va;
        v.in = lists_of(e, in_set < 4 ? in_set : 0);
        if (in_set >= 4) v.in.cnt = nullptr;
        v.in_set = (uint32_t)in_set;
        v.out = lists_of(e, out_set);
        v.out_set = (uint32_t)out_set;
        v.par = par;
        v.match = match;
        v.grounds = match ? job.grounds : nullptr;
        v.rmax = e.cfg.rmax;
        v.chunk_shift = e.cfg.chunk_shift;
        v.batch_shift = e.cfg.batch_shift;
        v.st = e.st;
    };
    auto sargs = [&](SweepArgs& c, int in_set, uint32_t par, bool input) {
        c.va = job.va;
        c.in = lists_of(e, in_set);
        c.in_set = (uint32_t)in_set;
        c.par = par;
        c.segs = w.segs;
        c.nsegs = job.nseg;
        c.task_ctr = &e.st->task[0];
        if (!input) { c.in_key = w.key[par]; c.in_nbr = w.nbr[par]; }
        c.out_key = w.key[par ^ 1u];
        c.out_nbr = w.nbr[par ^ 1u];
        c.ecap = job.ecap;
        c.rmax = e.cfg.rmax;
        c.chunk_shift = e.cfg.chunk_shift;
        c.st = e.st;
    };
    // round 0: candidates over the graphs' own arrays in tiles; match, open rows
    // filed in set 1; compaction from the input arrays into buffer 1
    A.r0.va = job.va;
    A.r0.segs = w.segs;
    A.r0.nsegs = job.nseg;
    A.r0.ntiles = job.ntiles;
    A.r0.st = e.st;
    vargs(A.v[0], 4, 1, 0, 1);
    A.v[0].vlist = job.vlist;
    A.v[0].nvlist = job.nvlist;
    A.v[0].deg0 = job.rdeg;
    A.v[0].round = 0;
    sargs(A.s[0], 1, 0, true);
    // round 1: set 1 -> 0, buffer 1 -> 0
    vargs(A.v[1], 1, 0, 1, 1);
    A.v[1].round_from_state = 1;
    sargs(A.s[1], 0, 1, false);
    // rounds of parity 0 (set 0 -> 1, buffer 0 -> 1) and 1 (set 1 -> 0, buffer 1 -> 0)
    vargs(A.v[2], 0, 1, 0, 1);
    A.v[2].round_from_state = 1;
    sargs(A.s[2], 1, 0, false);
    vargs(A.v[3], 1, 0, 1, 1);
    A.v[3].round_from_state = 1;
    sargs(A.s[3], 0, 1, false);
    JobArgs* D = reinterpret_cast<JobArgs*>(e.dargs);
    LM_CK(ctx, cudaMemcpyAsync(D, &A, sizeof A, cudaMemcpyHostToDevice, s));
    if (job.async) {
        // the next job may rewrite the staging only after these uploads ran
        if (!e.staged) LM_CK(ctx, cudaEventCreateWithFlags(&e.staged, cudaEventDisableTiming));
        LM_CK(ctx, cudaEventRecord(e.staged, s));
        e.staged_pending = true;
    }

    if (job.nseg == 0) {
        prof.begin(LM_K_INIT);
        LM_CK(ctx, launch_init(s, &D->init));
        prof.end();
    } else if (!prof.on) {
        if (e.graph && e.graph_cfg != e.cfg) {
            destroy_job_graph(e.graph);
            e.graph = nullptr;
        }
        if (!e.graph) {
            LM_CK(ctx, build_job_graph(D, e.st, e.cfg, &e.graph));
            e.graph_cfg = e.cfg;
        }
        LM_CK(ctx, launch_job_graph(e.graph, s));
        // launches of one job: init, 4 for round 0, then 5 per pair of rounds
        prof.launches[LM_K_INIT] += 1;
    } else {
        prof.begin(LM_K_INIT);
        LM_CK(ctx, launch_init(s, &D->init));
        prof.end();
        prof.begin(LM_K_CAND);
        LM_CK(ctx, launch_round0(s, &D->r0));
        prof.end();
        prof.begin(LM_K_OTHER);
        LM_CK(ctx, launch_round0_cut(s, &D->r0));
        prof.end();
        prof.begin(LM_K_VERTEX);
        LM_CK(ctx, launch_vertex(s, &D->v[0], e.cfg));
        prof.end();
        prof.begin(LM_K_SWEEP);
        LM_CK(ctx, launch_sweep_input(s, &D->s[0], e.cfg));
        prof.end();
        prof.begin(LM_K_VERTEX);
        LM_CK(ctx, launch_vertex(s, &D->v[1], e.cfg));
        prof.end();
        prof.begin(LM_K_SWEEP);
        LM_CK(ctx, launch_sweep_live(s, &D->s[1], e.cfg));
        prof.end();
        // the same limits as the device-driven loop: the round cap and the time limit
        const auto t_start = std::chrono::steady_clock::now();
        for (uint32_t pair = 0;; pair++) {
            for (int k = 2; k < 4; k++) {
                prof.begin(LM_K_VERTEX);
                LM_CK(ctx, launch_vertex(s, &D->v[k], e.cfg));
                prof.end();
                prof.begin(LM_K_SWEEP);
                LM_CK(ctx, launch_sweep_live(s, &D->s[k], e.cfg));
                prof.end();
            }
            LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            LM_CK(ctx, cudaStreamSynchronize(s));
            if (e.st_host->err || e.st_host->done) break;
            if (e.st_host->round > A.init.max_rounds) return fail(ctx, LM_ETIMEOUT, "round cap reached");
            if (e.st_host->last_ent < TAIL_ENT) {  // as the loop check: the tail finishes the job
                prof.begin(LM_K_TAIL);
                LM_CK(ctx, launch_tail(s, D, e.cfg));
                prof.end();
                break;
            }
            const auto waited = std::chrono::steady_clock::now() - t_start;
            if (std::chrono::duration_cast<std::chrono::nanoseconds>(waited).count() > (long long)A.init.limit_ns)
                return fail(ctx, LM_ETIMEOUT, "round loop exceeded its time limit");
        }
    }
    if (job.async) return LM_OK;  // queued; lm_sync reports device errors
    LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (job.nseg && !prof.on) {
        // kernels the graph ran: rounds 0 and 1 (tile candidates + cut rows, 2 vertex passes,
        // 2 sweeps), then per pair of rounds 2 vertex passes + 2 sweeps + 1 check, then the
        // tail kernel; round 1 leaves DevState::round at 2 and every later vertex pass
        // advances it (the loop's last round is the one the tail took over at, if it did)
        const uint32_t last = e.st_host->tail ? e.st_host->tail_round : e.st_host->round;
        const uint32_t pairs = (last >= 2) ? (last - 2) / 2 : 0;
        prof.launches[LM_K_CAND] += 1;
        prof.launches[LM_K_VERTEX] += 2 + 2 * pairs;
        prof.launches[LM_K_SWEEP] += 2 + 2 * pairs;
        prof.launches[LM_K_OTHER] += 1 + pairs;
        prof.launches[LM_K_TAIL] += 1;
    }
    return check_err(ctx, e);
}

// The edge-centric path of one graph (LM_F_EDGE_CENTRIC).  Its arguments sit
// in the second half of the argument area; the live edge lists reuse the
// workspace's neighbour buffers, the offers its long-row maxima, the stamps its
// long-row counters (all of which it leaves at zero).
constexpr size_t EDGE_ARGS_OFF = ARG_AREA / 2;
struct EdgeJobArgs {
    InitArgs init;
    EdgeArgs ea;
};
int match_edges(lm_ctx* ctx, Engine& e, const lm_graph* g, uint64_t seed, uint32_t* mate, bool dev_out, Prof& prof) {
    cudaStream_t s = e.stream;
    int rc = ensure_ws(ctx, e, g->n, g->nent, 1);
    if (rc) return rc;
    Workspace& w = e.ws;
    uint32_t* mate_d = dev_out ? mate : w.mate;
    static_assert(EDGE_ARGS_OFF + sizeof(EdgeJobArgs) <= ARG_AREA, "argument area too small");
    EdgeJobArgs& A = *reinterpret_cast<EdgeJobArgs*>(e.hargs + EDGE_ARGS_OFF);
    EdgeJobArgs* D = reinterpret_cast<EdgeJobArgs*>(e.dargs + EDGE_ARGS_OFF);
    memset(&A, 0, sizeof A);
    A.init.mate = mate_d;
    A.init.dead = w.dead;
    A.init.dbase = 0;
    A.init.bcnt = w.bcnt;
    A.init.bkey = w.bkey;
    A.init.n = g->n;
    job_limits(ctx, g->m, &A.init.max_rounds, &A.init.limit_ns);
    A.init.st = e.st;
    const uint64_t z = splitmix64_first(seed);
    EdgeArgs& a = A.ea;
    a.edges = g->edges;
    a.eword = g->eword;
    a.m = g->m;
    a.k0 = (uint32_t)z;
    a.k1 = (uint32_t)(z >> 32);
    a.nvert = g->n;
    a.live[0] = w.nbr[0];
    a.live[1] = w.nbr[1];
    a.cap = w.cap_e;
    a.best = w.bkey;
    a.stamp = w.bcnt;
    a.dead = w.dead;
    a.mate = mate_d;
    a.st = e.st;
    LM_CK(ctx, cudaMemcpyAsync(D, &A, sizeof A, cudaMemcpyHostToDevice, s));
    if (g->m == 0) {
        prof.begin(LM_K_INIT);
        LM_CK(ctx, launch_init(s, &D->init));
        prof.end();
    } else if (!prof.on) {
        if (!e.egraph) LM_CK(ctx, build_edge_graph(&D->init, &D->ea, e.st, &e.egraph));
        LM_CK(ctx, launch_job_graph(e.egraph, s));
        prof.launches[LM_K_INIT] += 1;
    } else {
        prof.begin(LM_K_INIT);
        LM_CK(ctx, launch_init(s, &D->init));
        prof.end();
        static const int kinds[4] = {LM_K_CAND, LM_K_VERTEX, LM_K_SWEEP, LM_K_OTHER};
        const auto t_start = std::chrono::steady_clock::now();
        for (;;) {
            for (int ph = 0; ph < 4; ph++) {
                prof.begin(kinds[ph]);
                LM_CK(ctx, launch_edge_round(s, &D->ea, ph));
                prof.end();
            }
            LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            LM_CK(ctx, cudaStreamSynchronize(s));
            if (e.st_host->err || e.st_host->done) break;
            if (e.st_host->round > A.init.max_rounds) return fail(ctx, LM_ETIMEOUT, "round cap reached");
            const auto waited = std::chrono::steady_clock::now() - t_start;
            if (std::chrono::duration_cast<std::chrono::nanoseconds>(waited).count() > (long long)A.init.limit_ns)
                return fail(ctx, LM_ETIMEOUT, "round loop exceeded its time limit");
        }
    }
    LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (g->m && !prof.on) {
        const uint32_t rounds = e.st_host->round >= 1 ? e.st_host->round - 1 : 0;  // rounds the loop ran
        prof.launches[LM_K_CAND] += rounds;
        prof.launches[LM_K_VERTEX] += rounds;
        prof.launches[LM_K_SWEEP] += rounds;
        prof.launches[LM_K_OTHER] += rounds;
    }
    rc = check_err(ctx, e);
    if (rc) return rc;
    if (!dev_out && g->n > 0) {
        LM_CK(ctx, cudaMemcpyAsync(mate, mate_d, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
        LM_CK(ctx, cudaStreamSynchronize(s));
    }
    return LM_OK;
}

// One graph on engine e, results to mate (device memory when dev_out, else host
// memory staged through the workspace); the engine's DevState holds its statistics.
int match_one(lm_ctx* ctx, Engine& e, const lm_graph* g, uint64_t seed, uint32_t* mate, bool dev_out, Prof& prof,
              bool async) {
    cudaStream_t s = e.stream;
    int rc = staging_ready(ctx, e);
    if (rc) return rc;
    rc = ensure_ws(ctx, e, g->n, g->nent, 1);
    if (rc) return rc;
    rc = ensure_pinned(ctx, e, sizeof(SegIn));
    if (rc) return rc;
    Job job;
    uint32_t* mate_d = dev_out ? mate : e.ws.mate;
    job.va = vertex_arrays(e, g->n, g->off, false, mate_d);
    job.nedges = g->m;
    job.ecap = g->nent;
    job.vlist = g->vid;
    job.rdeg = g->rdeg;
    job.nvlist = g->nrows;
    job.nseg = g->nent > 0 ? 1 : 0;
    job.ntiles = g->ntiles;
    job.async = async && dev_out && !prof.on;
    if (job.nseg) {
        const SegIn sg = seg_of(g, seed, 0, 0, 0);
        memcpy(e.pinned, &sg, sizeof sg);
        LM_CK(ctx, cudaMemcpyAsync(e.ws.segs, e.pinned, sizeof sg, cudaMemcpyHostToDevice, s));
    }
    rc = run_job(ctx, e, job, prof);
    if (rc) return rc;
    if (!dev_out && g->n > 0) {
        LM_CK(ctx, cudaMemcpyAsync(mate, mate_d, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
        LM_CK(ctx, cudaStreamSynchronize(s));
    }
    return LM_OK;
}

// Many graphs on engine e in the same launches (lm_batch_match, and groups of
// served requests): their vertex and entry ranges are laid side by side in one
// union id space, each graph keeping its own seed and edge ids.  mates[i] is
// device or host memory; rounds[i] and matched2[i] receive graph i's round count
// and matched vertices.
int match_batch(lm_ctx* ctx, Engine& e, const lm_graph* const* gs, uint32_t count, const uint64_t* seeds,
                uint32_t* const* mates, uint32_t* rounds, unsigned long long* matched2, Prof& prof) {
    uint64_t nv = 0, ne = 0;
    for (uint32_t i = 0; i < count; i++) {
        nv += gs[i]->n;
        ne += gs[i]->nent;
    }
    if (nv > 0xFFFFFFF0ull || ne > 0xFFFFFFF0ull) return fail(ctx, LM_EINVAL, "batch too large for 32-bit union ids");
    cudaStream_t s = e.stream;
    int rc = ensure_ws(ctx, e, (uint32_t)nv, (uint32_t)ne, count);
    if (rc) return rc;
    Workspace& w = e.ws;
    // host tables: graph vertex / entry bases, offsets, segments, destinations
    std::vector<uint32_t> gvb(count + 1), geb(count);
    std::vector<const uint32_t*> goff(count);
    std::vector<SegIn> segs(count);
    std::vector<uint32_t*> dst(count);
    std::vector<char> host_dst(count);
    uint32_t vb = 0, eb = 0, tb = 0;
    for (uint32_t i = 0; i < count; i++) {
        gvb[i] = vb;
        geb[i] = eb;
        goff[i] = gs[i]->off;
        segs[i] = seg_of(gs[i], seeds[i], vb, eb, tb);
        tb += gs[i]->ntiles;
        host_dst[i] = !is_device_ptr(mates[i]);
        dst[i] = host_dst[i] ? w.cnbr + vb : mates[i];  // host results are staged in the cnbr array
        vb += gs[i]->n;
        eb += gs[i]->nent;
    }
    gvb[count] = vb;
    const size_t b_gvb = (count + 1) * sizeof(uint32_t), b_geb = count * sizeof(uint32_t);
    const size_t b_off = count * sizeof(void*), b_seg = count * sizeof(SegIn), b_dst = count * sizeof(void*);
    rc = staging_ready(ctx, e);
    if (rc) return rc;
    rc = ensure_pinned(ctx, e, b_gvb + b_geb + b_off + b_seg + b_dst + 256);
    if (rc) return rc;
    char* pin = static_cast<char*>(e.pinned);
    size_t o = 0;
    auto stage = [&](void* dev, const void* src, size_t bytes) -> cudaError_t {
        memcpy(pin + o, src, bytes);
        cudaError_t r = cudaMemcpyAsync(dev, pin + o, bytes, cudaMemcpyHostToDevice, s);
        o = align_up(o + bytes, 16);
        return r;
    };
    LM_CK(ctx, stage(w.gvbase, gvb.data(), b_gvb));
    LM_CK(ctx, stage(w.gebase, geb.data(), b_geb));
    LM_CK(ctx, stage(w.goff, goff.data(), b_off));
    LM_CK(ctx, stage(w.segs, segs.data(), b_seg));
    LM_CK(ctx, stage(w.gdst, dst.data(), b_dst));
    LM_CK(ctx, cudaMemsetAsync(w.grounds, 0, count * sizeof(uint32_t), s));
    LM_CK(ctx, cudaMemsetAsync(w.gmatched, 0, count * sizeof(unsigned long long), s));
    prof.begin(LM_K_OTHER);
    LM_CK(ctx, launch_union_setup(s, w.gvbase, w.gebase, w.goff, count, (uint32_t)nv, w.start, w.gid, w.len[0]));
    prof.end();
    Job job;
    job.va = vertex_arrays(e, (uint32_t)nv, nullptr, true, w.mate);
    job.nedges = (uint32_t)(ne / 2);
    job.ecap = (uint32_t)ne;
    job.vlist = nullptr;
    job.rdeg = nullptr;
    job.nvlist = (uint32_t)nv;
    job.nseg = ne > 0 ? count : 0;
    job.ntiles = tb;
    job.grounds = w.grounds;
    rc = run_job(ctx, e, job, prof);
    if (rc) return rc;
    prof.begin(LM_K_OTHER);
    LM_CK(ctx, launch_to_local_batch(s, w.mate, w.gvbase, w.gid, count, w.gdst, w.gmatched, (uint32_t)nv));
    prof.end();
    bool any_host = false;
    for (uint32_t i = 0; i < count; i++) any_host |= host_dst[i] != 0;
    std::vector<uint32_t> hmate;
    if (any_host) {
        hmate.resize(nv);
        LM_CK(ctx, cudaMemcpyAsync(hmate.data(), w.cnbr, nv * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    }
    LM_CK(ctx, cudaMemcpyAsync(rounds, w.grounds, count * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaMemcpyAsync(matched2, w.gmatched, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (any_host)
        for (uint32_t i = 0; i < count; i++)
            if (host_dst[i] && gs[i]->n) memcpy(mates[i], hmate.data() + gvb[i], (size_t)gs[i]->n * sizeof(uint32_t));
    return LM_OK;
}

}  // namespace lm

namespace {

void fill_round_stats(const DevState& d, lm_stats* st) {
    st->rounds = d.rounds;
    st->matched = d.matched2 / 2;
    for (int i = 0; i < LM_STATS_ROUNDS; i++) {
        st->round_m[i] = d.ring_m[i];
        st->round_n[i] = d.ring_n[i];
    }
}

}  // namespace

// ============================================================ C ABI
extern "C" {

const char* lm_strerror(int code) {
    switch (code) {
        case LM_OK: return "ok";
        case LM_EINVAL: return "invalid argument";
        case LM_ENOMEM: return "out of memory or HBM budget";
        case LM_EAGAIN: return "no admission slot available, retry";
        case LM_ETIMEOUT: return "timed out";
        case LM_ECUDA: return "CUDA error (context poisoned)";
        case LM_ENOTFOUND: return "unknown ticket";
        default: return "unknown error";
    }
}

const char* lm_last_error(const lm_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

int lm_create(const lm_config* cfg, lm_ctx** out) {
    if (!cfg || !out) return LM_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return LM_EINVAL;
    }
    DevGuard g(cfg->device);
    if (!g.ok) return LM_ECUDA;
    if ((cfg->flags & LM_F_EDGE_CENTRIC) && (cfg->flags & LM_F_RENEW)) return LM_EINVAL;
    if ((cfg->flags & LM_F_ASYNC) && (cfg->flags & (LM_F_PROFILE | LM_F_EDGE_CENTRIC))) return LM_EINVAL;
    std::unique_ptr<lm_ctx> ctx(new lm_ctx());
    ctx->device = cfg->device;
    ctx->budget = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : (40ull << 30);
    ctx->max_slots = cfg->max_slots ? cfg->max_slots : 4096;
    ctx->flags = cfg->flags;
    ctx->eng.cfg.renew = (cfg->flags & LM_F_RENEW) != 0;
    // host-side fault injection for tests of the error paths: LM_FAULT=alloc makes
    // every later device allocation of this context fail, alloc:N the next N
    if (const char* f = getenv("LM_FAULT")) {
        if (!strncmp(f, "alloc", 5)) {
            long long k = -1;
            if (f[5] == ':') k = strtoll(f + 6, nullptr, 10);
            ctx->fault_alloc = k;
        }
    }
    {
        cudaMemPoolProps pp;
        memset(&pp, 0, sizeof pp);
        pp.allocType = cudaMemAllocationTypePinned;
        pp.handleTypes = cudaMemHandleTypeNone;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = cfg->device;
        if (cudaMemPoolCreate(&ctx->pool, &pp) != cudaSuccess) {
            cudaGetLastError();
            return LM_ECUDA;
        }
        uint64_t keep = ~0ull;  // never trim on synchronisation
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    int rc = engine_init(ctx.get(), ctx->eng, (cudaStream_t)cfg->stream);
    if (rc) {
        engine_free(ctx->eng);
        cudaMemPoolDestroy(ctx->pool);
        return rc;
    }
    if (cfg->flags & LM_F_PROFILE) {
        bool ok = true;
        for (int i = 0; i < MAX_PROFILE_EVENTS && ok; i++) {
            ok = cudaEventCreate(&ctx->ev[i]) == cudaSuccess;
            if (ok) ctx->nev = i + 1;
        }
        ctx->ev_ready = ok;
        cudaGetLastError();
    }
    *out = ctx.release();
    return LM_OK;
}

__attribute__((visibility("hidden"))) void lm_serve_shutdown(lm_ctx* ctx);  // lm_serve.cpp

void lm_destroy(lm_ctx* ctx) {
    if (!ctx) return;
    lm_serve_shutdown(ctx);
    DevGuard g(ctx->device);
    engine_free(ctx->eng);
    for (int i = 0; i < ctx->nev; i++) cudaEventDestroy(ctx->ev[i]);
    if (ctx->up) cudaStreamDestroy(ctx->up);
    if (ctx->up_ev) cudaEventDestroy(ctx->up_ev);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);  // released once no allocation is left
    cudaGetLastError();
    delete ctx;
}

int lm_graph_create(lm_ctx* ctx, uint32_t n, uint32_t m, const uint32_t* eu, const uint32_t* ev, const float* w,
                    int mem, lm_graph** out) {
    if (!ctx || !out) return LM_EINVAL;
    *out = nullptr;
    if (ctx->poisoned) return LM_ECUDA;
    if (mem != LM_HOST && mem != LM_DEVICE) return fail(ctx, LM_EINVAL, "mem must be LM_HOST or LM_DEVICE");
    if (m > 0x7FFFFFFFu) return fail(ctx, LM_EINVAL, "m = %u exceeds 2^31 - 1", m);
    if (m > 0 && (!eu || !ev || !w)) return fail(ctx, LM_EINVAL, "null edge array");
    if (m > 0 && n == 0) return fail(ctx, LM_EINVAL, "edges on an empty vertex set");
    if (n == 0xFFFFFFFFu) return fail(ctx, LM_EINVAL, "n must be below 2^32 - 1");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DevGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, LM_ECUDA, "cudaSetDevice failed");
    Engine& e = ctx->eng;
    cudaStream_t s = e.stream;
    std::unique_ptr<lm_graph> g(new lm_graph());
    g->ctx = ctx;
    g->n = n;
    g->m = m;
    g->nent = 2 * m;

    const uint32_t* d_eu = eu;
    const uint32_t* d_ev = ev;
    const float* d_w = w;
    const size_t nn = (size_t)n + 1;
    const size_t scan_words = std::max(exclusive_scan_tmp_words(n + 1), exclusive_scan_tmp_words(build_fill_scan_count(n, m)));
    Carver tc;
    uint32_t *t_eu = nullptr, *t_ev = nullptr, *deg = nullptr, *cursor = nullptr;
    uint32_t *flags = nullptr, *rowidx = nullptr, *scan_tmp = nullptr, *err = nullptr, *fill_tmp = nullptr;
    float* t_w = nullptr;
    if (mem == LM_HOST && m > 0) {
        tc.add(&t_eu, m);
        tc.add(&t_ev, m);
        tc.add(&t_w, m);
    }
    tc.add(&deg, nn);
    tc.add(&cursor, nn);
    tc.add(&flags, nn);
    tc.add(&rowidx, nn);
    tc.add(&scan_tmp, scan_words);
    tc.add(&err, 4);
    if (m > 0) tc.add(&fill_tmp, build_fill_tmp_words(n, m));
    void* tmp = nullptr;
    cudaError_t ce = fault_alloc(ctx) ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync(&tmp, tc.total, ctx->pool, s);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "graph staging");
    tc.assign(tmp);
    struct TmpFree {
        void* p;
        cudaStream_t s;
        ~TmpFree() { if (p) cudaFreeAsync(p, s); }
    } tf{tmp, s};
    LM_CK(ctx, cudaMemsetAsync(deg, 0, nn * 4, s));
    LM_CK(ctx, cudaMemsetAsync(err, 0, 16, s));
    // validation rides on the degree count: endpoint < n, no self loop, no NaN
    if (mem == LM_HOST && m > 0) {
        // chunks of the host arrays go up on the upload stream; the context's stream
        // counts a chunk's degrees while the next chunk is copied
        if (!ctx->up) {
            LM_CK(ctx, cudaStreamCreateWithFlags(&ctx->up, cudaStreamNonBlocking));
            LM_CK(ctx, cudaEventCreateWithFlags(&ctx->up_ev, cudaEventDisableTiming));
        }
        LM_CK(ctx, cudaEventRecord(ctx->up_ev, s));  // after the memsets (and earlier work)
        LM_CK(ctx, cudaStreamWaitEvent(ctx->up, ctx->up_ev, 0));
        constexpr uint32_t NCHUNK = 8;
        const uint32_t step = ((m + NCHUNK - 1) / NCHUNK + 31) & ~31u;
        for (uint32_t off = 0; off < m; off += step) {
            const uint32_t cnt = std::min(step, m - off);
            LM_CK(ctx, cudaMemcpyAsync(t_eu + off, eu + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, ctx->up));
            LM_CK(ctx, cudaMemcpyAsync(t_ev + off, ev + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, ctx->up));
            LM_CK(ctx, cudaMemcpyAsync(t_w + off, w + off, (size_t)cnt * 4, cudaMemcpyHostToDevice, ctx->up));
            LM_CK(ctx, cudaEventRecord(ctx->up_ev, ctx->up));
            LM_CK(ctx, cudaStreamWaitEvent(s, ctx->up_ev, 0));
            LM_CK(ctx, launch_build_degrees(s, t_eu + off, t_ev + off, t_w + off, n, cnt, deg, err));
        }
        d_eu = t_eu;
        d_ev = t_ev;
        d_w = t_w;
    } else if (m > 0) {
        LM_CK(ctx, launch_build_degrees(s, d_eu, d_ev, d_w, n, m, deg, err));
    }
    int rc = ensure_pinned(ctx, e, 64);
    if (rc) return rc;
    uint32_t* hp = static_cast<uint32_t*>(e.pinned);
    LM_CK(ctx, cudaMemcpyAsync(&hp[1], err, 4, cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, launch_nonzero_flags(s, deg, n + 1, flags));
    LM_CK(ctx, launch_exclusive_scan(s, flags, rowidx, n + 1, scan_tmp, scan_words));
    LM_CK(ctx, cudaMemcpyAsync(&hp[0], rowidx + n, 4, cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (hp[1]) return fail(ctx, LM_EINVAL, "edge list: endpoint >= n, self loop or NaN weight");
    g->nrows = hp[0];

    Carver gc;
    gc.add(&g->off, nn);
    // round-0 tiles copy rows [r & ~3, ...) of vid / roff in whole 16-byte words: pad both
    g->ntiles = (g->nent + TILE0 - 1) / TILE0;
    gc.add(&g->vid, (size_t)g->nrows + 8);
    gc.add(&g->rdeg, (size_t)g->nrows + 1);
    gc.add(&g->roff, (size_t)g->nrows + 8);
    gc.add(&g->tmap, (size_t)g->ntiles + 1);
    gc.add(&g->rbits, (size_t)g->ntiles * (TILE0 / 32) + 8);
    gc.add(&g->tdesc, (size_t)g->ntiles + 1);
    gc.add(&g->nbr, (size_t)g->nent + 4);
    gc.add(&g->pk, (size_t)g->nent + 4);
    gc.add(&g->edges, (size_t)g->m + 2);
    gc.add(&g->eword, (size_t)g->m + 4);
    ce = fault_alloc(ctx) ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync(&g->block, gc.total, ctx->pool, s);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "graph arrays");
    // every return before the graph is handed out gives the block back
    struct BlockFree {
        std::unique_ptr<lm_graph>& g;
        cudaStream_t s;
        ~BlockFree() { if (g && g->block) cudaFreeAsync(g->block, s); }
    } bf{g, s};
    gc.assign(g->block);
    g->bytes = gc.total;
    LM_CK(ctx, launch_exclusive_scan(s, deg, g->off, n + 1, scan_tmp, scan_words));
    if (m > 0) {
        LM_CK(ctx, cudaMemcpyAsync(cursor, g->off, nn * 4, cudaMemcpyDeviceToDevice, s));
        LM_CK(ctx, launch_build_fill(s, d_eu, d_ev, d_w, n, m, cursor, g->nbr, g->pk, g->edges, g->eword, fill_tmp,
                                     scan_tmp, scan_words, err));
        LM_CK(ctx, cudaMemcpyAsync(&hp[2], err, 4, cudaMemcpyDeviceToHost, s));
    }
    LM_CK(ctx, launch_build_rows(s, deg, rowidx, g->off, n, g->nrows, g->nent, g->vid, g->rdeg, g->roff));
    if (g->nrows) {
        LM_CK(ctx, cudaMemsetAsync(g->rbits, 0, ((size_t)g->ntiles * (TILE0 / 32) + 8) * 4, s));
        LM_CK(ctx, launch_build_tilemap(s, g->roff, g->nrows, g->nent, g->tmap, g->rbits, g->tdesc));
    }
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (m > 0 && (hp[2] & 2u)) return fail(ctx, LM_ECUDA, "graph build: a fill slot fell outside the edge arrays");
    *out = g.release();
    return LM_OK;
}

void lm_graph_destroy(lm_graph* g) {
    if (!g) return;
    DevGuard dg(g->ctx->device);
    // the graph may still be read by work on the context's stream or the serving
    // engine's: wait for the device, then return the block to the context's pool
    cudaDeviceSynchronize();
    if (g->block) cudaFreeAsync(g->block, g->ctx->eng.stream);
    cudaGetLastError();
    delete g;
}

int lm_graph_info(const lm_graph* g, uint32_t* n, uint32_t* m, uint64_t* device_bytes) {
    if (!g) return LM_EINVAL;
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (device_bytes) *device_bytes = g->bytes;
    return LM_OK;
}

int lm_match(lm_ctx* ctx, const lm_graph* g, uint64_t seed, uint32_t* mate, lm_stats* stats) {
    if (!ctx) return LM_EINVAL;
    if (ctx->poisoned) return LM_ECUDA;
    if (!g || !mate) return fail(ctx, LM_EINVAL, "null graph or mate");
    if (g->ctx->device != ctx->device) return fail(ctx, LM_EINVAL, "graph lives on another device");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DevGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, LM_ECUDA, "cudaSetDevice failed");
    if (stats) memset(stats, 0, sizeof *stats);
    Prof prof(ctx, ctx->eng.stream);
    const bool dev_out = is_device_ptr(mate);
    const bool async = (ctx->flags & LM_F_ASYNC) != 0;
    if (async && (!dev_out || stats))
        return fail(ctx, LM_EINVAL, "an asynchronous match writes device memory and returns no statistics");
    const int rc = (ctx->flags & LM_F_EDGE_CENTRIC) ? match_edges(ctx, ctx->eng, g, seed, mate, dev_out, prof)
                                                    : match_one(ctx, ctx->eng, g, seed, mate, dev_out, prof, async);
    if (rc) return rc;
    if (stats) {
        fill_round_stats(*ctx->eng.st_host, stats);
        prof.fill(stats);
    }
    return LM_OK;
}

int lm_contract(lm_ctx* ctx, uint32_t n, uint32_t m, const uint32_t* eu, const uint32_t* ev, const float* w,
                const uint32_t* vw, const uint32_t* mate, uint32_t* cmap, uint32_t* cvw, uint32_t* ceu,
                uint32_t* cev, float* cw, uint32_t* n_out, uint32_t* m_out) {
    if (!ctx) return LM_EINVAL;
    if (ctx->poisoned) return LM_ECUDA;
    if (!n_out || !m_out) return fail(ctx, LM_EINVAL, "null count output");
    *n_out = 0;
    *m_out = 0;
    if (n == 0 && m == 0) return LM_OK;
    const void* dev_in[] = {mate, cmap, cvw};
    for (const void* p : dev_in)
        if (!is_device_ptr(p)) return fail(ctx, LM_EINVAL, "contraction arrays must be device memory");
    if (m > 0) {
        const void* dev_e[] = {eu, ev, w, ceu, cev, cw};
        for (const void* p : dev_e)
            if (!is_device_ptr(p)) return fail(ctx, LM_EINVAL, "contraction arrays must be device memory");
    }
    if (vw && !is_device_ptr(vw)) return fail(ctx, LM_EINVAL, "vertex weights must be device memory");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DevGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, LM_ECUDA, "cudaSetDevice failed");
    Engine& e = ctx->eng;
    cudaStream_t s = e.stream;
    ContractArgs c;
    memset(&c, 0, sizeof c);
    c.n = n;
    c.m = m;
    c.eu = eu;
    c.ev = ev;
    c.w = w;
    c.vw = vw;
    c.mate = mate;
    c.cmap = cmap;
    c.cvw = cvw;
    c.ceu = ceu;
    c.cev = cev;
    c.cw = cw;
    c.sort_bits = e.cfg.contract_bits;
    if (m >= (1u << 31)) return fail(ctx, LM_EINVAL, "too many edges");
    if (n == 0xFFFFFFFFu) return fail(ctx, LM_EINVAL, "n must be below 2^32 - 1");
    const uint32_t scan_count = (n > m ? n : m) + 1;
    c.scan_words = exclusive_scan_tmp_words(scan_count);
    const size_t M = (size_t)m + 1;
    Carver cv;
    cv.add(&c.flag, (size_t)n + 1);
    cv.add(&c.rank, (size_t)n + 1);
    const size_t W = (size_t)m / 32 + 2;
    cv.add(&c.cross, W);
    cv.add(&c.counts, 8);
    cv.add(&c.cpair, 2 * (size_t)m + 8);
    cv.add(&c.key[0], M);
    cv.add(&c.key[1], M);
    cv.add(&c.val[0], M);
    cv.add(&c.val[1], M);
    cv.add(&c.shist, contract_sort_words(m));
    cv.add(&c.multi, (size_t)m / 32 + 2);
    cv.add(&c.wlead, W);
    cv.add(&c.wpos, W);
    cv.add(&c.tsum, 2 * ((size_t)m / 4096 + 2));
    cv.add(&c.gref, M);
    cv.add(&c.scan_tmp, c.scan_words);
    cv.add(&c.err, 4);
    if (e.cbytes < cv.total) {
        // grow-only scratch kept by the context (no allocation per call)
        LM_CK(ctx, cudaStreamSynchronize(s));
        if (e.cblock) cudaFree(e.cblock);
        e.cblock = nullptr;
        e.cbytes = 0;
        if (fault_alloc(ctx) || cudaMalloc(&e.cblock, cv.total) != cudaSuccess) {
            cudaGetLastError();
            e.cblock = nullptr;
            return fail(ctx, LM_ENOMEM, "contraction scratch of %zu bytes", cv.total);
        }
        e.cbytes = cv.total;
    }
    cv.assign(e.cblock);
    int rc = staging_ready(ctx, e);
    if (!rc) rc = ensure_pinned(ctx, e, 32);
    if (rc) return rc;
    uint32_t* hp = static_cast<uint32_t*>(e.pinned);
    cudaError_t ce = (cudaError_t)launch_contract(s, c, &hp[4]);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hp[0], c.err, 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hp[1], c.rank + n, 4, cudaMemcpyDeviceToHost, s);
    hp[2] = 0;
    if (ce == cudaSuccess && m > 0) ce = cudaMemcpyAsync(&hp[2], c.counts + 2, 4, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return fail(ctx, LM_ECUDA, "contraction: %s", cudaGetErrorString(ce));
    if (hp[0] & 1u) return fail(ctx, LM_EINVAL, "mate is not a matching of the vertex set");
    if (hp[0] & 2u) return fail(ctx, LM_EINVAL, "an edge endpoint is >= n");
    *n_out = hp[1];
    *m_out = hp[2];
    return LM_OK;
}

int lm_sync(lm_ctx* ctx) {
    if (!ctx) return LM_EINVAL;
    if (ctx->poisoned) return LM_ECUDA;
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DevGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, LM_ECUDA, "cudaSetDevice failed");
    Engine& e = ctx->eng;
    if (!e.st) return LM_OK;
    uint32_t* any = &reinterpret_cast<DevState*>(e.st_host)->err_any;
    LM_CK(ctx, cudaMemcpyAsync(any, &e.st->err_any, sizeof(uint32_t), cudaMemcpyDeviceToHost, e.stream));
    LM_CK(ctx, cudaStreamSynchronize(e.stream));
    e.staged_pending = false;
    const uint32_t bits = *any;
    if (!bits) return LM_OK;
    LM_CK(ctx, cudaMemsetAsync(&e.st->err_any, 0, sizeof(uint32_t), e.stream));
    LM_CK(ctx, cudaStreamSynchronize(e.stream));
    if (bits & ERR_BOUNDS) return fail(ctx, LM_ECUDA, "a queued match failed a device index check");
    return fail(ctx, LM_ETIMEOUT, "a queued match gave up a bounded device wait");
}

int lm_batch_match(lm_ctx* ctx, const lm_graph* const* gs, uint32_t count, const uint64_t* seeds,
                   uint32_t* const* mates, lm_stats* stats) {
    if (!ctx) return LM_EINVAL;
    if (ctx->poisoned) return LM_ECUDA;
    if (count == 0) return LM_OK;
    if (!gs || !seeds || !mates) return fail(ctx, LM_EINVAL, "null array");
    for (uint32_t i = 0; i < count; i++) {
        if (!gs[i] || !mates[i]) return fail(ctx, LM_EINVAL, "null graph or mate at %u", i);
        if (gs[i]->ctx->device != ctx->device) return fail(ctx, LM_EINVAL, "graph %u lives on another device", i);
    }
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DevGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, LM_ECUDA, "cudaSetDevice failed");
    if (stats) memset(stats, 0, sizeof(lm_stats) * count);
    Prof prof(ctx, ctx->eng.stream);
    std::vector<uint32_t> grounds(count);
    std::vector<unsigned long long> gm(count);
    const int rc = match_batch(ctx, ctx->eng, gs, count, seeds, mates, grounds.data(), gm.data(), prof);
    if (rc) return rc;
    if (stats) {
        // per graph: rounds, |M|, initial sizes; per call (copied into every entry): launches and timings
        lm_stats whole;
        memset(&whole, 0, sizeof whole);
        prof.fill(&whole);
        for (uint32_t i = 0; i < count; i++) {
            stats[i] = whole;
            stats[i].rounds = grounds[i];
            stats[i].matched = gm[i] / 2;
            stats[i].round_m[0] = gs[i]->m;
            stats[i].round_n[0] = gs[i]->nrows;
        }
    }
    return LM_OK;
}

namespace {
bool cfg_from(const lm_tuning* t, LaunchCfg* c) {
    if (!t || t->rmax < 1 || t->rmax > (1u << 20)) return false;
    if (t->chunk < 256 || t->chunk > (1u << 20) || (t->chunk & (t->chunk - 1))) return false;
    if (t->sweep_ctas_per_sm > 16 || t->vertex_ctas_per_sm > 4) return false;
    if (t->batch && (t->batch < 64 || t->batch > (1u << 20) || (t->batch & (t->batch - 1)))) return false;
    if (t->contract_bits % 8 || t->contract_bits > 32) return false;
    c->batch_shift = 32;
    if (t->batch)
        for (c->batch_shift = 0; (1u << c->batch_shift) < t->batch;) c->batch_shift++;
    c->rmax = t->rmax;
    c->chunk_shift = 0;
    while ((1u << c->chunk_shift) < t->chunk) c->chunk_shift++;
    c->sweep_ctas_per_sm = t->sweep_ctas_per_sm;
    c->vertex_ctas_per_sm = t->vertex_ctas_per_sm;
    c->contract_bits = t->contract_bits;
    return true;
}
void tuning_of(const LaunchCfg& c, lm_tuning* t) {
    t->rmax = c.rmax;
    t->chunk = 1u << c.chunk_shift;
    t->sweep_ctas_per_sm = c.sweep_ctas_per_sm;
    t->vertex_ctas_per_sm = c.vertex_ctas_per_sm;
    t->batch = c.batch_shift >= 32 ? 0u : 1u << c.batch_shift;
    t->contract_bits = c.contract_bits;
    t->ms = 0.0;
}
}  // namespace

int lm_set_limits(lm_ctx* ctx, uint32_t max_rounds, uint32_t time_limit_ms) {
    if (!ctx) return LM_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    ctx->lim_rounds = max_rounds;
    ctx->lim_ns = (uint64_t)time_limit_ms * 1000000ull;
    return LM_OK;
}

int lm_get_tuning(const lm_ctx* ctx, lm_tuning* out) {
    if (!ctx || !out) return LM_EINVAL;
    tuning_of(ctx->eng.cfg, out);
    return LM_OK;
}

int lm_set_tuning(lm_ctx* ctx, const lm_tuning* t) {
    if (!ctx) return LM_EINVAL;
    LaunchCfg c;
    if (!cfg_from(t, &c)) return fail(ctx, LM_EINVAL, "tuning out of range");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    c.renew = ctx->eng.cfg.renew;  // the order is the context's, not a tuning knob
    ctx->eng.cfg = c;
    return LM_OK;
}

int lm_autotune(lm_ctx* ctx, const lm_graph* const* g, uint32_t count, const uint64_t* seeds,
                uint32_t* const* mates, lm_tuning* best) {
    if (!ctx) return LM_EINVAL;
    if (count == 0 || !g || !seeds || !mates) return fail(ctx, LM_EINVAL, "nothing to tune on");
    // candidates (rmax, chunk, batch): task sizes from many short tasks to few long
    // ones, sweep at full or three-quarter occupancy
    static const uint32_t sizes[][3] = {{256, 1024, 256}, {512, 1024, 256}, {1024, 1024, 512}, {2048, 4096, 1024}};
    static const uint32_t sweeps[] = {0, 3};
    lm_tuning keep;
    lm_get_tuning(ctx, &keep);
    lm_tuning top = keep;
    top.ms = -1.0;
    for (const auto& sz : sizes) {
        for (uint32_t sw : sweeps) {
            lm_tuning t = {sz[0], sz[1], sw, keep.vertex_ctas_per_sm, sz[2], keep.contract_bits, 0.0};
            int rc = lm_set_tuning(ctx, &t);
            if (rc) return rc;
            std::vector<double> ms;
            for (int it = 0; it < 4; it++) {
                const auto t0 = std::chrono::steady_clock::now();
                rc = count == 1 ? lm_match(ctx, g[0], seeds[0], mates[0], nullptr)
                                : lm_batch_match(ctx, g, count, seeds, mates, nullptr);
                if (rc) {
                    lm_set_tuning(ctx, &keep);
                    return rc;
                }
                if (it > 0) ms.push_back(std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
            }
            std::sort(ms.begin(), ms.end());
            t.ms = ms[ms.size() / 2];
            if (top.ms < 0 || t.ms < top.ms) top = t;
        }
    }
    lm_set_tuning(ctx, &top);
    if (best) *best = top;
    return LM_OK;
}

}  // extern "C"
