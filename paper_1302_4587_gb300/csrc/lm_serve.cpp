// Serving: lm_submit / lm_poll / lm_wait (include/lm.h).
//
// A scheduler thread owns an engine of its own (stream, device state and a
// workspace sized from the context's HBM budget).  Each scheduler step runs
// one local-max round for every request in flight, in the same launches:
//   - requests admitted since the last step run their round 0 (candidate
//     sweep over their own adjacency arrays, mutual choice, compacting sweep
//     appended behind the survivors of the requests already in flight);
//   - requests in flight run their next round on the shared live arrays.
// A request joins between rounds as soon as its footprint (live entries,
// rows, a contiguous range of union vertex ids) fits, FIFO, and leaves as
// soon as it has no live row: its result is converted to local vertex ids
// and written to the caller's buffer.  Every request keeps its own seed and
// edge ids, and requests share no vertex, so a result does not depend on
// what else is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lm_host.h"

namespace lm {

struct Request {
    uint64_t ticket = 0;
    const lm_graph* g = nullptr;
    uint64_t seed = 0;
    uint32_t* mate = nullptr;
    bool host_dst = false;
    uint32_t vbase = 0;
    uint32_t rounds = 0;
    int state = 0;          // 0 queued, 1 in flight, 2 done
    int rc = LM_OK;
    uint64_t matched = 0;
};

struct ServeState {
    lm_ctx* ctx = nullptr;
    Engine eng;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread th;
    bool stop = false;
    int fatal = LM_OK;
    uint64_t next_ticket = 1;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::unordered_map<uint64_t, Request*> all;
    uint32_t cap_v = 0, cap_e = 0, cap_r = 0, cap_t = 0;
    uint64_t used_e = 0, used_r = 0;
    std::map<uint32_t, uint32_t> free_v;  // first vertex -> length
    uint32_t cur_buf = 0;
    bool live_any = false;
};

namespace {

constexpr size_t MAX_QUEUE = 1u << 20;

bool alloc_range(ServeState* S, uint32_t n, uint32_t* out) {
    if (n == 0) { *out = 0; return true; }
    for (auto it = S->free_v.begin(); it != S->free_v.end(); ++it) {
        if (it->second >= n) {
            *out = it->first;
            const uint32_t start = it->first + n, len = it->second - n;
            S->free_v.erase(it);
            if (len) S->free_v[start] = len;
            return true;
        }
    }
    return false;
}

void free_range(ServeState* S, uint32_t start, uint32_t n) {
    if (n == 0) return;
    auto it = S->free_v.emplace(start, n).first;
    auto nx = std::next(it);
    if (nx != S->free_v.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        S->free_v.erase(nx);
    }
    if (it != S->free_v.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            S->free_v.erase(it);
        }
    }
}

// One scheduler step (see the file comment).  Returns LM_OK or an error code.
int step(ServeState* S, const std::vector<Request*>& fresh, std::vector<Request*>& finished) {
    lm_ctx* ctx = S->ctx;
    Engine& e = S->eng;
    Workspace& w = e.ws;
    cudaStream_t s = e.stream;
    const uint32_t nvert = S->cap_v;
    LM_CK(ctx, cudaMemsetAsync(&e.st->err, 0, 2 * sizeof(uint32_t), s));

    for (Request* r : fresh)
        if (r->g->n) LM_CK(ctx, launch_init(s, w.mate + r->vbase, w.cnbr + r->vbase, w.dead + r->vbase, r->g->n, nullptr));
    std::vector<SegDesc> segs;
    uint32_t tb = 0;
    for (Request* r : fresh) {
        if (r->g->nent == 0) continue;
        segs.push_back(seg_of(r->g, r->seed, r->vbase, tb));
        tb += r->g->ntiles;
    }
    // active requests sorted by their vertex ranges (for the per-request row count)
    std::vector<Request*> act = S->active;
    std::sort(act.begin(), act.end(), [](const Request* a, const Request* b) { return a->vbase < b->vbase; });
    const uint32_t na = (uint32_t)act.size();
    const size_t seg_bytes = segs.size() * sizeof(SegDesc);
    const size_t gv_off = (seg_bytes + 255) / 256 * 256;
    int rc = ensure_pinned(ctx, e, gv_off + (size_t)(na + 1) * 4 + (size_t)na * 4 + 256);
    if (rc) return rc;
    char* pin = static_cast<char*>(e.pinned);
    if (!segs.empty()) {
        memcpy(pin, segs.data(), seg_bytes);
        LM_CK(ctx, cudaMemcpyAsync(w.segs, pin, seg_bytes, cudaMemcpyHostToDevice, s));
    }
    uint32_t* gv = reinterpret_cast<uint32_t*>(pin + gv_off);
    for (uint32_t i = 0; i < na; i++) gv[i] = act[i]->vbase;
    gv[na] = nvert;
    LM_CK(ctx, cudaMemcpyAsync(w.gvbase, gv, (size_t)(na + 1) * 4, cudaMemcpyHostToDevice, s));
    LM_CK(ctx, cudaMemsetAsync(w.rows_per, 0, (size_t)std::max(na, 1u) * 4, s));

    const uint32_t b = S->cur_buf, o = b ^ 1u;
    SweepArgs in = base_sweep_args(e, nvert);
    in.segs = w.segs;
    in.nsegs = (uint32_t)segs.size();
    in.ntiles_in = tb;
    if (!segs.empty()) LM_CK(ctx, launch_sweep_input_cand(s, in, e.sweep_grid));
    if (S->live_any) {
        VertexArgs vl = base_vertex_args(e, nvert, w.mate);
        vl.off = w.off[b];
        vl.vid = w.vid[b];
        vl.in_buf = b;
        LM_CK(ctx, launch_vertex_live(s, vl, e.vertex_grid));
    }
    for (Request* r : fresh) {
        if (r->g->nent == 0) continue;
        VertexArgs va = base_vertex_args(e, nvert, w.mate);
        va.vbegin = r->vbase;
        va.vcount = r->g->n;
        LM_CK(ctx, launch_vertex_all(s, va, e.vertex_grid));
    }
    if (S->live_any) {
        SweepArgs l = base_sweep_args(e, nvert);
        l.in_key = w.key[b];
        l.in_nbr = w.nbr[b];
        l.in_off = w.off[b];
        l.in_vid = w.vid[b];
        l.in_tilemap = w.tilemap;
        l.in_buf = b;
        l.out_key = w.key[o];
        l.out_nbr = w.nbr[o];
        l.out_off = w.off[o];
        l.out_vid = w.vid[o];
        l.out_buf = o;
        LM_CK(ctx, launch_sweep_live(s, l, e.sweep_grid));
    } else {
        LM_CK(ctx, cudaMemsetAsync(&e.st->cnt[o][0], 0, 2 * sizeof(uint32_t), s));
        LM_CK(ctx, cudaMemsetAsync(w.off[o], 0, sizeof(uint32_t), s));
    }
    if (!segs.empty()) {
        in.out_key = w.key[o];
        in.out_nbr = w.nbr[o];
        in.out_off = w.off[o];
        in.out_vid = w.vid[o];
        in.out_buf = o;
        in.prefix_in = &e.st->cnt[o][0];
        LM_CK(ctx, launch_sweep_input_compact(s, in, e.sweep_grid));
    }
    if (na) LM_CK(ctx, launch_rows_per_graph(s, w.vid[o], e.st, o, w.gvbase, na, w.rows_per, e.vertex_grid));
    uint32_t* rows_h = gv + na + 1;
    if (na) LM_CK(ctx, cudaMemcpyAsync(rows_h, w.rows_per, (size_t)na * 4, cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (e.st_host->err & ERR_BOUNDS) return fail(ctx, LM_ECUDA, "device index check failed (serving)");
    if (e.st_host->err & ERR_TIMEOUT) return fail(ctx, LM_ETIMEOUT, "look-back wait timed out (serving)");
    S->cur_buf = o;
    S->live_any = e.st_host->cnt[o][0] > 0;

    // requests without live rows are complete
    std::vector<Request*> done;
    for (uint32_t i = 0; i < na; i++) {
        Request* r = act[i];
        if (r->g->nent > 0) r->rounds++;  // fresh requests ran round 0, the others their next round
        if (rows_h[i] == 0) done.push_back(r);
    }
    if (!done.empty()) {
        LM_CK(ctx, cudaMemsetAsync(w.gmatched, 0, done.size() * sizeof(unsigned long long), s));
        for (size_t k = 0; k < done.size(); k++) {
            Request* r = done[k];
            if (!r->g->n) continue;
            uint32_t* dst = r->host_dst ? w.cnbr + r->vbase : r->mate;
            LM_CK(ctx, launch_to_local(s, w.mate, r->vbase, r->g->n, dst, &w.gmatched[k]));
            if (r->host_dst)
                LM_CK(ctx, cudaMemcpyAsync(r->mate, dst, (size_t)r->g->n * 4, cudaMemcpyDeviceToHost, s));
        }
        std::vector<unsigned long long> gm(done.size());
        LM_CK(ctx, cudaMemcpyAsync(gm.data(), w.gmatched, done.size() * sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, s));
        LM_CK(ctx, cudaStreamSynchronize(s));
        for (size_t k = 0; k < done.size(); k++) done[k]->matched = gm[k] / 2;
    }
    finished = done;
    return LM_OK;
}

void scheduler(ServeState* S) {
    cudaSetDevice(S->ctx->device);
    for (;;) {
        std::vector<Request*> fresh;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop) return;
            while (!S->queue.empty() && S->active.size() < S->ctx->max_slots) {
                Request* r = S->queue.front();
                if (S->used_e + r->g->nent > S->cap_e || S->used_r + r->g->nrows > S->cap_r) break;
                uint32_t vb = 0;
                if (!alloc_range(S, r->g->n, &vb)) break;
                S->queue.pop_front();
                r->vbase = vb;
                r->state = 1;
                S->used_e += r->g->nent;
                S->used_r += r->g->nrows;
                S->active.push_back(r);
                fresh.push_back(r);
            }
        }
        std::vector<Request*> finished;
        int rc = S->fatal ? S->fatal : step(S, fresh, finished);
        std::lock_guard<std::mutex> lk(S->mu);
        if (rc) {
            // the shared live state is lost: fail every request in flight
            finished = S->active;
            for (Request* r : finished) r->rc = rc;
            S->live_any = false;
            if (rc == LM_ECUDA) S->fatal = rc;
        }
        for (Request* r : finished) {
            r->state = 2;
            free_range(S, r->vbase, r->g->n);
            S->used_e -= r->g->nent;
            S->used_r -= r->g->nrows;
            S->active.erase(std::find(S->active.begin(), S->active.end(), r));
        }
        if (!finished.empty()) S->cv_done.notify_all();
    }
}

int serve_start(lm_ctx* ctx) {
    if (ctx->serve) return LM_OK;
    std::unique_ptr<ServeState> S(new ServeState());
    S->ctx = ctx;
    cudaStream_t st = nullptr;
    LM_CK(ctx, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = engine_init(ctx, S->eng, st);
    if (rc) {
        engine_free(S->eng);
        cudaStreamDestroy(st);
        return rc;
    }
    // capacities from the budget: live entries 24 B (two 12-byte buffers),
    // vertices 9 B, rows 16 B, plus look-back records per tile
    const double B = (double)ctx->budget;
    const double lim = 4.0e9;
    S->cap_e = (uint32_t)std::min(lim, B * 0.70 / 24.0);
    S->cap_v = (uint32_t)std::min(lim, B * 0.15 / 9.0);
    S->cap_r = (uint32_t)std::min((double)S->cap_v, std::min(lim, B * 0.12 / 16.0));
    S->cap_t = S->cap_e / SWEEP_T + ctx->max_slots + 2;
    rc = ensure_ws(ctx, S->eng, S->cap_v, S->cap_e, S->cap_r, S->cap_t, ctx->max_slots + 1);
    if (rc) {
        engine_free(S->eng);
        cudaStreamDestroy(st);
        return rc;
    }
    S->free_v[0] = S->cap_v;
    ServeState* raw = S.release();
    ctx->serve = raw;
    raw->th = std::thread(scheduler, raw);
    return LM_OK;
}

}  // namespace
}  // namespace lm

using namespace lm;

extern "C" {

__attribute__((visibility("hidden"))) void lm_serve_shutdown(lm_ctx* ctx) {
    if (!ctx || !ctx->serve) return;
    ServeState* S = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    cudaStream_t st = S->eng.stream;
    engine_free(S->eng);
    if (st) cudaStreamDestroy(st);
    for (auto& kv : S->all) delete kv.second;
    delete S;
    ctx->serve = nullptr;
}

int lm_submit(lm_ctx* ctx, const lm_graph* g, uint64_t seed, uint32_t* mate, uint64_t* ticket) {
    if (!ctx) return LM_EINVAL;
    if (ctx->poisoned) return LM_ECUDA;
    if (!g || !mate || !ticket) return fail(ctx, LM_EINVAL, "null graph, mate or ticket");
    if (g->ctx->device != ctx->device) return fail(ctx, LM_EINVAL, "graph lives on another device");
    {
        std::lock_guard<std::mutex> lk(ctx->call_mu);
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != ctx->device) cudaSetDevice(ctx->device);
        int rc = serve_start(ctx);
        if (cur >= 0 && cur != ctx->device) cudaSetDevice(cur);
        if (rc) return rc;
    }
    ServeState* S = ctx->serve;
    if (S->fatal) return S->fatal;
    if (g->n > S->cap_v || g->nent > S->cap_e || g->nrows > S->cap_r)
        return fail(ctx, LM_ENOMEM, "request exceeds the serving budget");
    std::unique_ptr<Request> r(new Request());
    r->g = g;
    r->seed = seed;
    r->mate = mate;
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != ctx->device) cudaSetDevice(ctx->device);
        r->host_dst = !is_device_ptr(mate);
        if (cur >= 0 && cur != ctx->device) cudaSetDevice(cur);
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queue.size() >= MAX_QUEUE) return LM_EAGAIN;
    r->ticket = S->next_ticket++;
    *ticket = r->ticket;
    S->all[r->ticket] = r.get();
    S->queue.push_back(r.release());
    S->cv_work.notify_one();
    return LM_OK;
}

int lm_poll(lm_ctx* ctx, uint64_t ticket, int* done, lm_stats* stats) {
    if (!ctx || !done) return LM_EINVAL;
    *done = 0;
    ServeState* S = ctx->serve;
    if (!S) return LM_ENOTFOUND;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return LM_ENOTFOUND;
    Request* r = it->second;
    if (r->state != 2) return LM_OK;
    *done = 1;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->rounds = r->rounds;
        stats->matched = r->matched;
        stats->round_m[0] = r->g->m;
        stats->round_n[0] = r->g->nrows;
    }
    const int rc = r->rc;
    S->all.erase(it);
    delete r;
    return rc;
}

int lm_wait(lm_ctx* ctx, uint64_t ticket, uint32_t timeout_ms) {
    if (!ctx) return LM_EINVAL;
    ServeState* S = ctx->serve;
    if (!S) return LM_ENOTFOUND;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return LM_ENOTFOUND;
    Request* r = it->second;
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->state == 2; });
    return ok ? LM_OK : LM_ETIMEOUT;
}

}  // extern "C"
