// Serving: lm_submit / lm_poll / lm_wait (include/lm.h).
//
// A scheduler thread owns an engine of its own (stream, device state and a
// workspace sized from the context's HBM budget).  Each scheduler step runs
// one local-max round for every request in flight, in shared launches:
//   - requests admitted since the last step run their round 0 (filing of
//     their rows, candidate sweep over their own adjacency arrays, mutual
//     choice, compacting sweep into their range of the shared entry space);
//   - requests already in flight run their next round on the shared arrays.
// A request joins between rounds as soon as its footprint (a contiguous
// range of union vertex ids and one of union entries) fits and a slot is
// free, in arrival order, and leaves after the first round in which it has no
// live unmatched row: its result is converted to local vertex ids and written
// to the caller's buffer.  When nothing is in flight, a short queue instead runs
// to completion as one job graph (the batched path, or the plain one for a
// single request): at light load that answers sooner than round-by-round steps.  Every request keeps its own seed and edge ids and
// shares no vertex with another, so its result does not depend on what else
// is in flight.
//
// List sets of the engine: 0 and 1 hold the rows of in-flight requests
// (alternating by step parity), 2 the rows of fresh requests before their
// candidate sweep, 3 the round-0 tasks of fresh requests.
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
    uint32_t vbase = 0, ebase = 0, slot = 0;
    uint32_t rounds = 0;
    int state = 0;          // 0 queued, 1 in flight, 2 done
    int rc = LM_OK;
    uint64_t matched = 0;
};

// first-fit allocator of contiguous id ranges
struct RangeAlloc {
    std::map<uint32_t, uint32_t> free_;  // first id -> length
    void init(uint32_t cap) { free_.clear(); if (cap) free_[0] = cap; }
    bool alloc(uint32_t n, uint32_t* out) {
        if (n == 0) { *out = 0; return true; }
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *out = it->first;
                const uint32_t st = it->first + n, len = it->second - n;
                free_.erase(it);
                if (len) free_[st] = len;
                return true;
            }
        }
        return false;
    }
    void release(uint32_t start, uint32_t n) {
        if (n == 0) return;
        auto it = free_.emplace(start, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
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
    std::vector<uint32_t> free_slots;
    std::unordered_map<uint64_t, Request*> all;
    uint32_t cap_v = 0, cap_e = 0;
    RangeAlloc vspace, espace;
    uint32_t step = 0;
};

namespace {

constexpr size_t MAX_QUEUE = 1u << 20;

constexpr uint32_t MAX_FRESH = 64;  // admissions per step (kernel arguments of one step fit the argument area)
constexpr uint32_t MAX_ROUNDS_PER_STEP = 8;  // a step without admissions runs up to this many rounds
constexpr size_t MAX_GROUP = 16;  // queued requests that run together as one job when nothing is in flight

struct StepArgs {
    InitArgs init[MAX_FRESH];
    VertexArgs pre[MAX_FRESH];
    VertexArgs v_live, v_prev_fresh, v_fresh;
    SweepArgs cand, s_live, s_fresh;
    VertexArgs v_more[MAX_ROUNDS_PER_STEP];  // rounds 1.. of a step without admissions
    SweepArgs s_more[MAX_ROUNDS_PER_STEP];
};

// One scheduler step (see the file comment).  A step that admits nothing and has
// nobody waiting runs `rounds` rounds before it returns to the host (fewer host
// round trips while the load is light).  Returns LM_OK or an error code.
int step(ServeState* S, const std::vector<Request*>& fresh, std::vector<Request*>& finished, uint32_t rounds) {
    lm_ctx* ctx = S->ctx;
    Engine& e = S->eng;
    Workspace& w = e.ws;
    cudaStream_t s = e.stream;
    const uint32_t par = S->step & 1u;
    const VertexArrays va = vertex_arrays(e, S->cap_v, nullptr, true, w.mate);
    static_assert(sizeof(StepArgs) <= ARG_AREA, "argument area too small");
    StepArgs& A = *reinterpret_cast<StepArgs*>(e.hargs);
    StepArgs* D = reinterpret_cast<StepArgs*>(e.dargs);
    memset(&A, 0, sizeof A);
    LM_CK(ctx, cudaMemsetAsync(&e.st->err, 0, 2 * sizeof(uint32_t), s));

    // tables of the fresh requests
    const uint32_t na = (uint32_t)S->active.size();
    int rc = ensure_pinned(ctx, e, MAX_FRESH * sizeof(SegIn));
    if (rc) return rc;
    SegIn* segs_h = static_cast<SegIn*>(e.pinned);
    for (size_t k = 0; k < fresh.size(); k++) {
        Request* r = fresh[k];
        segs_h[k] = seg_of(r->g, r->seed, r->vbase, r->ebase, 0);
        LM_CK(ctx, cudaMemcpyAsync(&w.segs[r->slot], &segs_h[k], sizeof(SegIn), cudaMemcpyHostToDevice, s));
        LM_CK(ctx, launch_req_setup(s, r->g->off, r->g->n, r->vbase, r->ebase, r->slot, w.start, w.gid));
        InitArgs& ia = A.init[k];
        ia.mate = w.mate + r->vbase;
        ia.dead = w.dead;
        ia.dbase = r->vbase;
        ia.bcnt = w.bcnt + r->vbase;
        ia.bkey = w.bkey + r->vbase;
        ia.n = r->g->n;
        ia.st = nullptr;
        VertexArgs& pre = A.pre[k];
        pre.va = va;
        pre.in = lists_of(e, 2);
        pre.in.cnt = nullptr;
        pre.in_set = 4;
        pre.vlist = r->g->vid;
        pre.nvlist = r->g->nrows;
        pre.vlist_base = r->vbase;
        pre.deg0 = r->g->rdeg;
        pre.out = lists_of(e, 2);
        pre.out_set = 2;
        pre.par = par;
        pre.rmax = e.cfg.rmax;
        pre.chunk_shift = e.cfg.chunk_shift;
        pre.batch_shift = e.cfg.batch_shift;
        pre.st = e.st;
    }
    auto vpass = [&](VertexArgs& v, int in_set, int out_set, uint32_t p = 2, uint32_t rnd = 0) {
        v.va = va;
        v.in = lists_of(e, in_set);
        v.in_set = in_set;
        v.out = lists_of(e, out_set);
        v.out_set = out_set;
        v.par = p < 2 ? p : par;
        v.round = rnd;  // round index within the step (per-request round counts)
        v.match = 1;
        v.glive = w.glive;
        v.grounds = w.grounds;
        v.rmax = e.cfg.rmax;
        v.chunk_shift = e.cfg.chunk_shift;
        v.batch_shift = e.cfg.batch_shift;
        v.st = e.st;
    };
    vpass(A.v_live, par, par ^ 1u);
    vpass(A.v_prev_fresh, 3, par ^ 1u);
    vpass(A.v_fresh, 2, 3);
    auto sargs = [&](SweepArgs& c, int in_set, bool input, uint32_t p = 2) {
        const uint32_t pp = p < 2 ? p : par;
        c.va = va;
        c.in = lists_of(e, in_set);
        c.in_set = in_set;
        c.par = pp;
        c.segs = w.segs;
        c.nsegs = ctx->max_slots;
        if (!input) { c.in_key = w.key[pp]; c.in_nbr = w.nbr[pp]; }
        c.out_key = w.key[pp ^ 1u];
        c.out_nbr = w.nbr[pp ^ 1u];
        c.ecap = S->cap_e;
        c.rmax = e.cfg.rmax;
        c.chunk_shift = e.cfg.chunk_shift;
        c.st = e.st;
    };
    sargs(A.cand, 2, true);
    sargs(A.s_live, par ^ 1u, false);
    sargs(A.s_fresh, 3, true);
    // each sweep its own task counter; the vertex pass before each zeroes them
    A.cand.task_ctr = &e.st->task[0];
    A.s_live.task_ctr = &e.st->task[1];
    A.s_fresh.task_ctr = &e.st->task[2];
    if (!fresh.empty()) rounds = 1;
    rounds = std::max(1u, std::min(rounds, MAX_ROUNDS_PER_STEP));
    for (uint32_t r = 1; r < rounds; r++) {
        const uint32_t pr = (S->step + r) & 1u;
        vpass(A.v_more[r], (int)pr, (int)(pr ^ 1u), pr, r);
        sargs(A.s_more[r], (int)(pr ^ 1u), false, pr);
        A.s_more[r].task_ctr = &e.st->task[1];
    }
    LM_CK(ctx, cudaMemcpyAsync(D, &A, sizeof A, cudaMemcpyHostToDevice, s));
    LM_CK(ctx, cudaMemsetAsync(w.glive, 0, (size_t)ctx->max_slots * sizeof(uint32_t), s));
    LM_CK(ctx, cudaMemsetAsync(w.grounds, 0, (size_t)ctx->max_slots * sizeof(uint32_t), s));

    // fresh requests: reset their vertex state, file their rows (set 2), find their candidates
    bool any_fresh_edges = false;
    for (size_t k = 0; k < fresh.size(); k++) {
        if (fresh[k]->g->n) LM_CK(ctx, launch_init(s, &D->init[k]));
        if (fresh[k]->g->nent == 0) continue;
        any_fresh_edges = true;
        LM_CK(ctx, launch_vertex(s, &D->pre[k], e.cfg));
    }
    if (any_fresh_edges) LM_CK(ctx, launch_sweep_cand(s, &D->cand, e.cfg));
    // mutual choice: in-flight rows (sets par and 3), then the fresh rows (set 2 -> set 3)
    LM_CK(ctx, launch_vertex(s, &D->v_live, e.cfg));
    LM_CK(ctx, launch_vertex(s, &D->v_prev_fresh, e.cfg));
    if (any_fresh_edges) LM_CK(ctx, launch_vertex(s, &D->v_fresh, e.cfg));
    // sweeps: in-flight rows from the live buffers, fresh rows from their own arrays
    LM_CK(ctx, launch_sweep_live(s, &D->s_live, e.cfg));
    if (any_fresh_edges) LM_CK(ctx, launch_sweep_input(s, &D->s_fresh, e.cfg));
    // further rounds of a step without admissions; the live-row counts that decide
    // completion are those of the last round
    for (uint32_t r = 1; r < rounds; r++) {
        if (r == rounds - 1) LM_CK(ctx, cudaMemsetAsync(w.glive, 0, (size_t)ctx->max_slots * sizeof(uint32_t), s));
        LM_CK(ctx, launch_vertex(s, &D->v_more[r], e.cfg));
        LM_CK(ctx, launch_sweep_live(s, &D->s_more[r], e.cfg));
    }
    // which requests still have live rows
    std::vector<uint32_t> glive(ctx->max_slots), gr(ctx->max_slots);
    LM_CK(ctx, cudaMemcpyAsync(glive.data(), w.glive, (size_t)ctx->max_slots * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaMemcpyAsync(gr.data(), w.grounds, (size_t)ctx->max_slots * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaMemcpyAsync(e.st_host, e.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    LM_CK(ctx, cudaStreamSynchronize(s));
    if (e.st_host->err & ERR_BOUNDS) return fail(ctx, LM_ECUDA, "device index check failed (serving)");
    if (e.st_host->err & ERR_TIMEOUT) return fail(ctx, LM_ETIMEOUT, "a bounded device wait gave up (serving)");
    (void)na;
    // grounds[slot] = 1 + the last round of the step in which the request had live
    // rows (its rounds are consecutive); it is complete once no live row is left unmatched
    std::vector<Request*> done;
    for (Request* r : S->active) {
        r->rounds += gr[r->slot];
        if (glive[r->slot] == 0) done.push_back(r);
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
    S->step += rounds;
    finished = done;
    return LM_OK;
}

void scheduler(ServeState* S) {
    cudaSetDevice(S->ctx->device);
    for (;;) {
        std::vector<Request*> fresh, group;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty() || !S->active.empty(); });
            if (S->stop) return;
            // with nothing in flight, the few requests queued so far run together to
            // completion as one job graph (one request: the plain path; several: the
            // batched path), whose round loop stays on the device.  At light load this
            // answers sooner than stepping round by round, which returns to the host
            // after every round; requests arriving meanwhile queue for the next
            // dispatch.  A longer queue, or requests in flight, go round by round with
            // admissions between rounds (continuous batching).
            if (S->active.empty() && S->queue.size() <= MAX_GROUP && !S->fatal) {
                group.assign(S->queue.begin(), S->queue.end());
                S->queue.clear();
                for (Request* r : group) r->state = 1;
            }
            while (group.empty() && !S->queue.empty() && !S->free_slots.empty() && fresh.size() < MAX_FRESH) {
                Request* r = S->queue.front();
                uint32_t vb = 0, eb = 0;
                if (!S->vspace.alloc(r->g->n, &vb)) break;
                if (!S->espace.alloc(r->g->nent, &eb)) {
                    S->vspace.release(vb, r->g->n);
                    break;
                }
                S->queue.pop_front();
                r->vbase = vb;
                r->ebase = eb;
                r->slot = S->free_slots.back();
                S->free_slots.pop_back();
                r->state = 1;
                S->active.push_back(r);
                fresh.push_back(r);
            }
        }
        if (!group.empty()) {
            Prof off(nullptr, S->eng.stream);
            const size_t k = group.size();
            std::vector<uint32_t> rounds(k);
            std::vector<unsigned long long> m2(k);
            int rc;
            if (k == 1) {
                Request* r = group[0];
                rc = match_one(S->ctx, S->eng, r->g, r->seed, r->mate, !r->host_dst, off);
                if (rc == LM_OK) {
                    rounds[0] = S->eng.st_host->rounds;
                    m2[0] = S->eng.st_host->matched2;
                }
            } else {
                std::vector<const lm_graph*> gs(k);
                std::vector<uint64_t> seeds(k);
                std::vector<uint32_t*> mates(k);
                for (size_t i = 0; i < k; i++) {
                    gs[i] = group[i]->g;
                    seeds[i] = group[i]->seed;
                    mates[i] = group[i]->mate;
                }
                rc = match_batch(S->ctx, S->eng, gs.data(), (uint32_t)k, seeds.data(), mates.data(), rounds.data(),
                                 m2.data(), off);
            }
            std::lock_guard<std::mutex> lk(S->mu);
            if (rc == LM_ECUDA) S->fatal = rc;
            for (size_t i = 0; i < k; i++) {
                Request* r = group[i];
                r->rc = rc;
                if (rc == LM_OK) {
                    r->rounds = rounds[i];
                    r->matched = m2[i] / 2;
                }
                r->state = 2;
            }
            S->cv_done.notify_all();
            continue;
        }
        std::vector<Request*> finished;
        bool waiting;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            waiting = !S->queue.empty();
        }
        const int rc = S->fatal ? S->fatal : step(S, fresh, finished, waiting ? 1u : MAX_ROUNDS_PER_STEP);
        std::lock_guard<std::mutex> lk(S->mu);
        if (rc) {
            // the shared live state is lost: fail every request in flight
            finished = S->active;
            for (Request* r : finished) r->rc = rc;
            if (rc == LM_ECUDA) S->fatal = rc;
            // start over with empty lists
            cudaMemsetAsync(&S->eng.st->lcnt[0][0], 0, sizeof(S->eng.st->lcnt), S->eng.stream);
        }
        for (Request* r : finished) {
            r->state = 2;
            S->vspace.release(r->vbase, r->g->n);
            S->espace.release(r->ebase, r->g->nent);
            S->free_slots.push_back(r->slot);
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
    S->eng.cfg = ctx->eng.cfg;  // the context's launch parameters when serving starts
    // capacities from the budget: per entry 24 B (two 12-byte buffers) + list and
    // partial space; per vertex 9 words of vertex state and task lists
    const double B = (double)ctx->budget;
    const double lim = 4.0e9;
    S->cap_e = (uint32_t)std::min(lim, B * 0.80 / 25.0);
    S->cap_v = (uint32_t)std::min(lim, B * 0.15 / 110.0);
    rc = ensure_ws(ctx, S->eng, S->cap_v, S->cap_e, ctx->max_slots);
    if (rc) {
        engine_free(S->eng);
        cudaStreamDestroy(st);
        return rc;
    }
    LM_CK(ctx, cudaMemsetAsync(S->eng.st, 0, sizeof(DevState), st));
    LM_CK(ctx, cudaStreamSynchronize(st));
    S->vspace.init(S->cap_v);
    S->espace.init(S->cap_e);
    for (uint32_t i = 0; i < ctx->max_slots; i++) S->free_slots.push_back(ctx->max_slots - 1 - i);
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
    if (ctx->flags & LM_F_RENEW) return fail(ctx, LM_EINVAL, "serving does not renew the order (LM_F_RENEW)");
    if (g->ctx->device != ctx->device) return fail(ctx, LM_EINVAL, "graph lives on another device");
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != ctx->device) cudaSetDevice(ctx->device);
    int rc;
    {
        std::lock_guard<std::mutex> lk(ctx->call_mu);
        rc = serve_start(ctx);
    }
    const bool host_dst = rc == LM_OK && !is_device_ptr(mate);
    if (cur >= 0 && cur != ctx->device) cudaSetDevice(cur);
    if (rc) return rc;
    ServeState* S = ctx->serve;
    if (S->fatal) return S->fatal;
    if (g->n > S->cap_v || g->nent > S->cap_e) return fail(ctx, LM_ENOMEM, "request exceeds the serving budget");
    std::unique_ptr<Request> r(new Request());
    r->g = g;
    r->seed = seed;
    r->mate = mate;
    r->host_dst = host_dst;
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
