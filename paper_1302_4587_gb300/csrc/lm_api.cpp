// Host side of liblm: context, graphs, plain and batched matching (include/lm.h).
//
// Everything on the result path runs on the GPU (lm_kernels.cu); this file
// validates arguments, owns device memory, builds launch arguments, drives
// the round loop and moves results between host and device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
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

SegDesc seg_of(const lm_graph* g, uint64_t seed, uint32_t vbase, uint32_t tile_begin) {
    SegDesc d;
    memset(&d, 0, sizeof d);
    const uint64_t z = splitmix64_first(seed);
    d.off = g->off;
    d.vid = g->vid;
    d.nbr = g->nbr;
    d.eid = g->eid;
    d.ordw = g->ordw;
    d.tilemap = g->tilemap;
    d.nrows = g->nrows;
    d.nent = g->nent;
    d.vbase = vbase;
    d.k0 = (uint32_t)z;
    d.k1 = (uint32_t)(z >> 32);
    d.tile_begin = tile_begin;
    d.ntiles = g->ntiles;
    return d;
}

int engine_init(lm_ctx* ctx, Engine& e, cudaStream_t stream) {
    e.device = ctx->device;
    e.stream = stream;
    LM_CK(ctx, cudaMalloc(&e.st, sizeof(DevState)));
    LM_CK(ctx, cudaMallocHost(&e.st_host, sizeof(DevState)));
    memset(e.st_host, 0, sizeof(DevState));
    e.st_host->epoch = 1;  // look-back records of generation 0 never count
    LM_CK(ctx, cudaMemcpy(e.st, e.st_host, sizeof(DevState), cudaMemcpyHostToDevice));
    e.sweep_grid = sweep_grid(ctx->device);
    e.vertex_grid = vertex_grid(ctx->device);
    return LM_OK;
}

void engine_free(Engine& e) {
    if (e.stream) cudaStreamSynchronize(e.stream);
    else cudaDeviceSynchronize();
    if (e.ws.block) cudaFree(e.ws.block);
    if (e.pinned) cudaFreeHost(e.pinned);
    if (e.st) cudaFree(e.st);
    if (e.st_host) cudaFreeHost(e.st_host);
    cudaGetLastError();
    e = Engine();
}

int ensure_ws(lm_ctx* ctx, Engine& e, uint32_t nv, uint32_t ne, uint32_t nr, uint32_t nt, uint32_t ng) {
    Workspace& w = e.ws;
    if (w.block && nv <= w.cap_v && ne <= w.cap_e && nr <= w.cap_r && nt <= w.cap_t && ng <= w.cap_g) return LM_OK;
    LM_CK(ctx, cudaStreamSynchronize(e.stream));
    Workspace nw;
    nw.cap_v = std::max(nv, w.cap_v);
    nw.cap_e = std::max(ne, w.cap_e);
    nw.cap_r = std::max(nr, w.cap_r);
    nw.cap_t = std::max(nt, w.cap_t);
    nw.cap_g = std::max(std::max(ng, w.cap_g), 1u);
    Carver c;
    c.add(&nw.cnbr, (size_t)nw.cap_v + 1);
    c.add(&nw.dead, (size_t)nw.cap_v + 1);
    c.add(&nw.mate, (size_t)nw.cap_v + 1);
    for (int b = 0; b < 2; b++) {
        c.add(&nw.key[b], (size_t)nw.cap_e + 4);
        c.add(&nw.nbr[b], (size_t)nw.cap_e + 4);
        c.add(&nw.off[b], (size_t)nw.cap_r + 2);
        c.add(&nw.vid[b], (size_t)nw.cap_r + 1);
    }
    c.add(&nw.tilemap, (size_t)nw.cap_t + 2);
    c.add(&nw.lb_desc, 4 * ((size_t)nw.cap_t + 1));
    c.add(&nw.lb_part, (size_t)nw.cap_t + 1);
    c.add(&nw.segs, (size_t)nw.cap_g);
    c.add(&nw.gvbase, (size_t)nw.cap_g + 1);
    c.add(&nw.grounds, (size_t)nw.cap_g);
    c.add(&nw.gdst, (size_t)nw.cap_g);
    c.add(&nw.gmatched, (size_t)nw.cap_g);
    c.add(&nw.rows_per, (size_t)nw.cap_g);
    if (w.block) {
        cudaFree(w.block);
        w.block = nullptr;
    }
    void* p = nullptr;
    cudaError_t err = cudaMalloc(&p, c.total);
    if (err != cudaSuccess) {
        cudaGetLastError();
        e.ws = Workspace();
        return fail(ctx, LM_ENOMEM, "workspace of %zu bytes: %s", c.total, cudaGetErrorString(err));
    }
    c.assign(p);
    nw.block = p;
    nw.bytes = c.total;
    e.ws = nw;
    // look-back descriptors start at generation 0, which no sweep uses
    LM_CK(ctx, cudaMemsetAsync(e.ws.lb_desc, 0, 4 * ((size_t)nw.cap_t + 1) * sizeof(uint32_t), e.stream));
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

SweepArgs base_sweep_args(Engine& e, uint32_t nvert) {
    SweepArgs a;
    memset(&a, 0, sizeof a);
    Workspace& w = e.ws;
    a.cnbr = w.cnbr;
    a.dead = w.dead;
    a.nvert = nvert;
    a.lb_desc = w.lb_desc;
    a.lb_part = w.lb_part;
    a.lb_cap = w.cap_t + 1;
    a.st = e.st;
    a.out_cap = w.cap_e;
    a.out_rows_cap = w.cap_r;
    return a;
}

VertexArgs base_vertex_args(Engine& e, uint32_t nvert, uint32_t* mate) {
    VertexArgs v;
    memset(&v, 0, sizeof v);
    v.nvert = nvert;
    v.cnbr = e.ws.cnbr;
    v.dead = e.ws.dead;
    v.mate = mate;
    v.tilemap = e.ws.tilemap;
    v.tilemap_cap = e.ws.cap_t + 2;
    v.st = e.st;
    return v;
}

}  // namespace lm

// ============================================================ the round loop
namespace {

// Per-kernel CUDA-event timing of one call (LM_F_PROFILE).
struct Prof {
    lm_ctx* ctx;
    cudaStream_t s;
    bool on;
    int kind[MAX_PROFILE_EVENTS / 2];
    int n = 0;
    uint32_t launches[LM_K_COUNT] = {0, 0, 0, 0, 0};
    Prof(lm_ctx* c, cudaStream_t st) : ctx(c), s(st), on((c->flags & LM_F_PROFILE) && c->ev_ready) {}
    void begin(int k) {
        launches[k]++;
        if (!on || n >= MAX_PROFILE_EVENTS / 2) return;
        kind[n] = k;
        cudaEventRecord(ctx->ev[2 * n], s);
    }
    void end() {
        if (!on || n >= MAX_PROFILE_EVENTS / 2) return;
        cudaEventRecord(ctx->ev[2 * n + 1], s);
        n++;
    }
    void fill(lm_stats* st) {
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
};

// A set of input graphs (segments) over one union vertex space.
struct Job {
    std::vector<SegDesc> segs;       // non-empty graphs only
    uint32_t nvert = 0;              // union vertices
    uint32_t nent = 0, ntiles = 0;
    uint32_t* mate = nullptr;        // union result (device)
    const uint32_t* gvbase = nullptr;
    uint32_t ngraphs = 0;
    uint32_t* grounds = nullptr;
};

int check_err(lm_ctx* ctx, Engine& e) {
    const uint32_t err = e.st_host->err;
    if (err & ERR_BOUNDS) return fail(ctx, LM_ECUDA, "device index check failed (index %u)", e.st_host->err_info);
    if (err & ERR_TIMEOUT) return fail(ctx, LM_ETIMEOUT, "look-back wait timed out at tile %u", e.st_host->err_info);
    return LM_OK;
}

// Whole local-max loop for `job`: result in job.mate, DevState mirror refreshed.
int run_job(lm_ctx* ctx, Engine& e, Job& job, Prof& prof) {
    Workspace& w = e.ws;
    cudaStream_t s = e.stream;
    if (!job.segs.empty()) {
        int rc = ensure_pinned(ctx, e, job.segs.size() * sizeof(SegDesc));
        if (rc) return rc;
        memcpy(e.pinned, job.segs.data(), job.segs.size() * sizeof(SegDesc));
        LM_CK(ctx, cudaMemcpyAsync(w.segs, e.pinned, job.segs.size() * sizeof(SegDesc), cudaMemcpyHostToDevice, s));
    }
    prof.begin(LM_K_INIT);
    LM_CK(ctx, launch_init(s, job.mate, w.cnbr, w.dead, job.nvert, e.st));
    prof.end();

    if (job.nent > 0) {
        SweepArgs a = base_sweep_args(e, job.nvert);
        a.segs = w.segs;
        a.nsegs = (uint32_t)job.segs.size();
        a.ntiles_in = job.ntiles;
        a.round = 0;
        // round 0, step 2 (Sec. 2): candidates from the graphs' own adjacency arrays
        prof.begin(LM_K_SWEEP);
        LM_CK(ctx, launch_sweep_input_cand(s, a, e.sweep_grid));
        prof.end();
        // round 0, step 3: mutual choice
        VertexArgs va = base_vertex_args(e, job.nvert, job.mate);
        va.vbegin = 0;
        va.vcount = job.nvert;
        va.gvbase = job.gvbase;
        va.ngraphs = job.ngraphs;
        va.grounds = job.grounds;
        va.round = 0;
        prof.begin(LM_K_VERTEX);
        LM_CK(ctx, launch_vertex_all(s, va, e.vertex_grid));
        prof.end();
        // round 0, steps 4-6, fused with step 2 of round 1
        a.out_key = w.key[1];
        a.out_nbr = w.nbr[1];
        a.out_off = w.off[1];
        a.out_vid = w.vid[1];
        a.out_buf = 1;
        prof.begin(LM_K_SWEEP);
        LM_CK(ctx, launch_sweep_input_compact(s, a, e.sweep_grid));
        prof.end();

        // rounds >= 1 in chunks; the live edge count is read back between chunks
        uint32_t r = 1, chunk = 4;
        for (;;) {
            for (uint32_t k = 0; k < chunk; k++, r++) {
                const uint32_t b = r & 1u;
                VertexArgs vl = base_vertex_args(e, job.nvert, job.mate);
                vl.off = w.off[b];
                vl.vid = w.vid[b];
                vl.in_buf = b;
                vl.round = r;
                vl.gvbase = job.gvbase;
                vl.ngraphs = job.ngraphs;
                vl.grounds = job.grounds;
                prof.begin(LM_K_VERTEX);
                LM_CK(ctx, launch_vertex_live(s, vl, e.vertex_grid));
                prof.end();
                SweepArgs l = base_sweep_args(e, job.nvert);
                l.in_key = w.key[b];
                l.in_nbr = w.nbr[b];
                l.in_off = w.off[b];
                l.in_vid = w.vid[b];
                l.in_tilemap = w.tilemap;
                l.in_buf = b;
                l.out_key = w.key[b ^ 1u];
                l.out_nbr = w.nbr[b ^ 1u];
                l.out_off = w.off[b ^ 1u];
                l.out_vid = w.vid[b ^ 1u];
                l.out_buf = b ^ 1u;
                l.round = r;
                prof.begin(LM_K_SWEEP);
                LM_CK(ctx, launch_sweep_live(s, l, e.sweep_grid));
                prof.end();
            }
            LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            LM_CK(ctx, cudaStreamSynchronize(s));
            if (e.st_host->err) break;
            if (e.st_host->cnt[r & 1u][0] == 0) break;
            chunk = std::min<uint32_t>(chunk * 2, 64);
        }
    }
    LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    return check_err(ctx, e);
}

void fill_round_stats(const DevState& d, lm_stats* st, uint64_t m0, uint64_t n0) {
    st->rounds = d.rounds;
    st->matched = d.matched2 / 2;
    for (int i = 0; i < LM_STATS_ROUNDS; i++) {
        st->round_m[i] = d.ring_m[i];
        st->round_n[i] = d.ring_n[i];
    }
    st->round_m[0] = m0;
    st->round_n[0] = n0;
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
    std::unique_ptr<lm_ctx> ctx(new lm_ctx());
    ctx->device = cfg->device;
    ctx->budget = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : (40ull << 30);
    ctx->max_slots = cfg->max_slots ? cfg->max_slots : 4096;
    ctx->flags = cfg->flags;
    int rc = engine_init(ctx.get(), ctx->eng, (cudaStream_t)cfg->stream);
    if (rc) {
        engine_free(ctx->eng);
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
    g->ntiles = tiles_of(g->nent);

    const uint32_t* d_eu = eu;
    const uint32_t* d_ev = ev;
    const float* d_w = w;
    const size_t nn = (size_t)n + 1;
    const size_t scan_words = exclusive_scan_tmp_words(n + 1);
    Carver tc;
    uint32_t *t_eu = nullptr, *t_ev = nullptr, *deg = nullptr, *offall = nullptr, *cursor = nullptr;
    uint32_t *flags = nullptr, *rowidx = nullptr, *scan_tmp = nullptr, *err = nullptr;
    float* t_w = nullptr;
    if (mem == LM_HOST && m > 0) {
        tc.add(&t_eu, m);
        tc.add(&t_ev, m);
        tc.add(&t_w, m);
    }
    tc.add(&deg, nn);
    tc.add(&offall, nn);
    tc.add(&cursor, nn);
    tc.add(&flags, nn);
    tc.add(&rowidx, nn);
    tc.add(&scan_tmp, scan_words);
    tc.add(&err, 4);
    void* tmp = nullptr;
    cudaError_t ce = cudaMallocAsync(&tmp, tc.total, s);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "graph staging");
    tc.assign(tmp);
    struct TmpFree {
        void* p;
        cudaStream_t s;
        ~TmpFree() { if (p) cudaFreeAsync(p, s); }
    } tf{tmp, s};
    if (mem == LM_HOST && m > 0) {
        LM_CK(ctx, cudaMemcpyAsync(t_eu, eu, (size_t)m * 4, cudaMemcpyHostToDevice, s));
        LM_CK(ctx, cudaMemcpyAsync(t_ev, ev, (size_t)m * 4, cudaMemcpyHostToDevice, s));
        LM_CK(ctx, cudaMemcpyAsync(t_w, w, (size_t)m * 4, cudaMemcpyHostToDevice, s));
        d_eu = t_eu;
        d_ev = t_ev;
        d_w = t_w;
    }
    LM_CK(ctx, cudaMemsetAsync(deg, 0, nn * 4, s));
    LM_CK(ctx, cudaMemsetAsync(err, 0, 16, s));
    // validation rides on the degree count: endpoint < n, no self loop, no NaN
    if (m > 0) LM_CK(ctx, launch_build_degrees(s, d_eu, d_ev, d_w, n, m, deg, err));
    LM_CK(ctx, launch_exclusive_scan(s, deg, offall, n + 1, scan_tmp, scan_words));
    LM_CK(ctx, launch_nonzero_flags(s, deg, n + 1, flags));
    LM_CK(ctx, launch_exclusive_scan(s, flags, rowidx, n + 1, scan_tmp, scan_words));
    int rc = ensure_pinned(ctx, e, 64);
    if (rc) return rc;
    uint32_t* hp = static_cast<uint32_t*>(e.pinned);
    LM_CK(ctx, cudaMemcpyAsync(&hp[0], rowidx + n, 4, cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaMemcpyAsync(&hp[1], err, 4, cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (hp[1]) return fail(ctx, LM_EINVAL, "edge list: endpoint >= n, self loop or NaN weight");
    g->nrows = hp[0];

    Carver gc;
    gc.add(&g->off, (size_t)g->nrows + 1);
    gc.add(&g->vid, (size_t)g->nrows + 1);
    gc.add(&g->nbr, (size_t)g->nent + 4);
    gc.add(&g->eid, (size_t)g->nent + 4);
    gc.add(&g->ordw, (size_t)g->nent + 4);
    gc.add(&g->tilemap, (size_t)g->ntiles + 2);
    ce = cudaMalloc(&g->block, gc.total);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "graph arrays");
    gc.assign(g->block);
    g->bytes = gc.total;
    if (m > 0) {
        LM_CK(ctx, cudaMemcpyAsync(cursor, offall, nn * 4, cudaMemcpyDeviceToDevice, s));
        LM_CK(ctx, launch_build_fill(s, d_eu, d_ev, d_w, m, offall, cursor, g->nbr, g->eid, g->ordw));
    }
    LM_CK(ctx, launch_build_rows(s, deg, rowidx, offall, n, g->nrows, g->nent, g->off, g->vid));
    if (g->nrows > 0) LM_CK(ctx, launch_build_tilemap(s, g->off, g->nrows, g->nent, g->tilemap));
    LM_CK(ctx, cudaStreamSynchronize(s));
    *out = g.release();
    return LM_OK;
}

void lm_graph_destroy(lm_graph* g) {
    if (!g) return;
    DevGuard dg(g->ctx->device);
    if (g->ctx->eng.stream) cudaStreamSynchronize(g->ctx->eng.stream);
    else cudaDeviceSynchronize();
    if (g->block) cudaFree(g->block);
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
    Engine& e = ctx->eng;
    if (stats) memset(stats, 0, sizeof *stats);
    const bool dev_out = is_device_ptr(mate);
    int rc = ensure_ws(ctx, e, g->n, g->nent, g->nrows, g->ntiles + 1, 1);
    if (rc) return rc;
    Job job;
    job.nvert = g->n;
    job.nent = g->nent;
    job.ntiles = g->ntiles;
    job.mate = dev_out ? mate : e.ws.mate;
    if (g->nent > 0) job.segs.push_back(seg_of(g, seed, 0, 0));
    Prof prof(ctx, e.stream);
    rc = run_job(ctx, e, job, prof);
    if (rc) return rc;
    if (!dev_out && g->n > 0) {
        LM_CK(ctx, cudaMemcpyAsync(mate, job.mate, (size_t)g->n * 4, cudaMemcpyDeviceToHost, e.stream));
        LM_CK(ctx, cudaStreamSynchronize(e.stream));
    }
    if (stats) {
        fill_round_stats(*e.st_host, stats, g->m, g->nrows);
        prof.fill(stats);
    }
    return LM_OK;
}

int lm_batch_match(lm_ctx* ctx, const lm_graph* const* gs, uint32_t count, const uint64_t* seeds,
                   uint32_t* const* mates, lm_stats* stats) {
    if (!ctx) return LM_EINVAL;
    if (ctx->poisoned) return LM_ECUDA;
    if (count == 0) return LM_OK;
    if (!gs || !seeds || !mates) return fail(ctx, LM_EINVAL, "null array");
    uint64_t nv = 0, ne = 0, nr = 0, nt = 0;
    for (uint32_t i = 0; i < count; i++) {
        if (!gs[i] || !mates[i]) return fail(ctx, LM_EINVAL, "null graph or mate at %u", i);
        if (gs[i]->ctx->device != ctx->device) return fail(ctx, LM_EINVAL, "graph %u lives on another device", i);
        nv += gs[i]->n;
        ne += gs[i]->nent;
        nr += gs[i]->nrows;
        nt += gs[i]->ntiles;
    }
    if (nv > 0xFFFFFFF0ull || ne > 0xFFFFFFF0ull || nt + count > 0xFFFFFFF0ull)
        return fail(ctx, LM_EINVAL, "batch too large for 32-bit union ids (split it)");
    std::lock_guard<std::mutex> lk(ctx->call_mu);
    DevGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, LM_ECUDA, "cudaSetDevice failed");
    Engine& e = ctx->eng;
    cudaStream_t s = e.stream;
    if (stats) memset(stats, 0, sizeof(lm_stats) * count);
    int rc = ensure_ws(ctx, e, (uint32_t)nv, (uint32_t)ne, (uint32_t)nr, (uint32_t)(nt + 1), count);
    if (rc) return rc;
    Workspace& w = e.ws;
    Job job;
    job.nvert = (uint32_t)nv;
    job.nent = (uint32_t)ne;
    job.mate = w.mate;
    job.ngraphs = count;
    job.gvbase = w.gvbase;
    job.grounds = w.grounds;
    std::vector<uint32_t> gvb(count + 1);
    std::vector<uint32_t*> dst(count);
    std::vector<char> host_dst(count);
    uint32_t vb = 0, tb = 0;
    for (uint32_t i = 0; i < count; i++) {
        gvb[i] = vb;
        if (gs[i]->nent > 0) {
            job.segs.push_back(seg_of(gs[i], seeds[i], vb, tb));
            tb += gs[i]->ntiles;
        }
        host_dst[i] = !is_device_ptr(mates[i]);
        dst[i] = host_dst[i] ? nullptr : mates[i];
        vb += gs[i]->n;
    }
    gvb[count] = vb;
    job.ntiles = tb;
    rc = ensure_pinned(ctx, e, std::max((count + 1) * sizeof(uint32_t) + count * sizeof(uint32_t*),
                                        job.segs.size() * sizeof(SegDesc)) + 64);
    if (rc) return rc;
    memcpy(e.pinned, gvb.data(), (count + 1) * sizeof(uint32_t));
    LM_CK(ctx, cudaMemcpyAsync(w.gvbase, e.pinned, (count + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    LM_CK(ctx, cudaMemsetAsync(w.grounds, 0, count * sizeof(uint32_t), s));
    LM_CK(ctx, cudaMemsetAsync(w.gmatched, 0, count * sizeof(unsigned long long), s));
    LM_CK(ctx, cudaStreamSynchronize(s));  // the pinned staging is reused by run_job
    Prof prof(ctx, s);
    rc = run_job(ctx, e, job, prof);
    if (rc) return rc;
    // device destinations are written directly; host ones go through the cnbr array as staging
    bool any_host = false;
    for (uint32_t i = 0; i < count; i++) {
        if (host_dst[i]) {
            any_host = true;
            dst[i] = w.cnbr + gvb[i];
        }
    }
    memcpy(e.pinned, dst.data(), count * sizeof(uint32_t*));
    LM_CK(ctx, cudaMemcpyAsync(w.gdst, e.pinned, count * sizeof(uint32_t*), cudaMemcpyHostToDevice, s));
    prof.begin(LM_K_OTHER);
    LM_CK(ctx, launch_to_local_batch(s, w.mate, w.gvbase, count, w.gdst, w.gmatched, (uint32_t)nv));
    prof.end();
    std::vector<uint32_t> hmate;
    if (any_host) {
        hmate.resize(nv);
        LM_CK(ctx, cudaMemcpyAsync(hmate.data(), w.cnbr, nv * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    }
    std::vector<uint32_t> grounds(count);
    std::vector<unsigned long long> gm(count);
    LM_CK(ctx, cudaMemcpyAsync(grounds.data(), w.grounds, count * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaMemcpyAsync(gm.data(), w.gmatched, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (any_host)
        for (uint32_t i = 0; i < count; i++)
            if (host_dst[i] && gs[i]->n) memcpy(mates[i], hmate.data() + gvb[i], (size_t)gs[i]->n * sizeof(uint32_t));
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

}  // extern "C"
