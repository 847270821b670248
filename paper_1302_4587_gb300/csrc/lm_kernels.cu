// sm_103a kernels of the local-max matching path.
//
// One round of local max (the phase of Sec. 2: every live vertex picks its
// heaviest live edge, edges picked by both ends join M, edges touching M are
// deleted) is two launches:
//
//   k_vertex  over the rows that were live after the previous round: a row v
//             whose chosen neighbour u = cnbr[v] chose v back is matched
//             (both ends write their own mate slot, so there is no conflict;
//             step 3).  Every other live row is filed into this round's task
//             lists by its length.  Rows of matched vertices are never read
//             again: deleting a vertex's edges costs nothing (steps 4-6).
//   k_sweep   one warp per task: reads the row's live entries, keeps an entry
//             when its neighbour is unmatched, writes the survivors to the
//             front of the row's range in the other buffer, and takes the
//             maximum key of the survivors -- the row's candidate for the
//             next round (step 2 of the next round; the segmented maximum of
//             Lemma "broadcast" restricted to one row).
//
// Round 0 first files every row (k_vertex without matching), runs a
// candidate-only sweep over the graphs' own arrays, then the match and a
// compacting sweep that builds the 64-bit keys
//     K(e) = ord(w_e) << 32 | perm_seed(e)
// from (ord(weight), edge id) on the fly.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include "lm_internal.h"

namespace lm {

#define FULL 0xFFFFFFFFu

// ---------------------------------------------------------------- order
// MurmurHash3 32-bit finaliser (Appleby, public domain).
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ uint32_t perm_seed(uint32_t e, uint32_t k0, uint32_t k1) {
    return fmix32(fmix32(e ^ k0) ^ k1);
}
// monotone float32 -> uint32 (-0 == +0); NaN is rejected before this runs
__device__ __forceinline__ uint32_t ord_of_bits(uint32_t b) {
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// ---------------------------------------------------------------- utilities
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}
__device__ __forceinline__ void set_err(DevState* st, uint32_t bit, uint32_t info) {
    if ((atomicOr(&st->err, bit) & bit) == 0) st->err_info = info;
}
// warp-wide maximum of (key, neighbour); keys are unique among live entries of a row
__device__ __forceinline__ void warp_kv_max(uint64_t& k, uint32_t& u) {
    const uint32_t hi = __reduce_max_sync(FULL, (uint32_t)(k >> 32));
    const uint32_t lo = __reduce_max_sync(FULL, ((uint32_t)(k >> 32) == hi) ? (uint32_t)k : 0u);
    const uint64_t best = ((uint64_t)hi << 32) | lo;
    const uint32_t owner = __ballot_sync(FULL, k == best && best != 0);
    u = owner ? __shfl_sync(FULL, u, __ffs(owner) - 1) : NIL;
    k = owner ? best : 0;
}

// ---------------------------------------------------------------- init
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_init(const InitArgs* __restrict__ pa) {
    const InitArgs& A = *pa;
    uint32_t* mate = A.mate;
    uint8_t* dead = A.dead;
    uint32_t* bcnt = A.bcnt;
    const uint32_t n = A.n;
    DevState* st = A.st;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (mate) mate[v] = NIL;
        dead[v] = 0;
        bcnt[v] = 0;
    }
    if (st && blockIdx.x == 0) {
        for (int i = threadIdx.x; i < 64; i += blockDim.x) { st->ring_m[i] = 0; st->ring_n[i] = 0; }
        if (threadIdx.x < 16) (&st->lcnt[0][0])[threadIdx.x] = 0;
        if (threadIdx.x == 0) {
            st->err = 0; st->err_info = 0; st->rounds = 0; st->done = 0;
            st->live_rows = 0; st->live_ent = 0; st->matched2 = 0;
            st->round = 1;
            st->max_rounds = A.max_rounds;
            st->t0_ns = globaltimer_ns();
        }
    }
}

// ---------------------------------------------------------------- vertex pass
constexpr int VT = 256;  // threads
constexpr int VI = 8;    // rows per thread per block iteration

// exclusive scan of three counters over the block (a, b, c become their
// prefixes; tot receives the block totals)
__device__ __forceinline__ void block_excl_scan3(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t* tmp,
                                                 uint32_t tot[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ia = warp_incl_scan(a, lane), ib = warp_incl_scan(b, lane), ic = warp_incl_scan(c, lane);
    if (lane == 31) { tmp[warp * 3] = ia; tmp[warp * 3 + 1] = ib; tmp[warp * 3 + 2] = ic; }
    __syncthreads();
    uint32_t pa = 0, pb = 0, pc = 0;
    tot[0] = tot[1] = tot[2] = 0;
#pragma unroll
    for (int w = 0; w < VT / 32; w++) {
        const uint32_t x = tmp[w * 3], y = tmp[w * 3 + 1], z = tmp[w * 3 + 2];
        if (w < warp) { pa += x; pb += y; pc += z; }
        tot[0] += x; tot[1] += y; tot[2] += z;
    }
    a = pa + ia - a;
    b = pb + ib - b;
    c = pc + ic - c;
}

__global__ void __launch_bounds__(VT) k_vertex(const VertexArgs* __restrict__ pav) {
    const VertexArgs& a = *pav;
    __shared__ uint32_t s_tmp[3 * (VT / 32)];
    __shared__ uint32_t s_base[3];
    __shared__ unsigned long long s_red[3 * (VT / 32)];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    DevState* st = a.st;
    const VertexArrays& va = a.va;
    const uint32_t par = a.par;
    const uint32_t round = a.round_from_state ? ld_volatile_u32(&st->round) : a.round;

    uint32_t nT = 0, nM = 0, nC = 0, total;
    if (a.vlist || !a.in.cnt) {
        total = a.nvlist;
    } else {
        nT = ld_volatile_u32(&a.in.cnt[0]);
        nM = ld_volatile_u32(&a.in.cnt[1]);
        nC = ld_volatile_u32(&a.in.cnt[2]);
        total = nC + nM + nT;
    }
    unsigned long long my_rows = 0, my_ent = 0, my_match = 0;

    for (uint32_t base = blockIdx.x * (VT * VI); base < total; base += gridDim.x * (VT * VI)) {
        uint32_t vv[VI], LL[VI], cls[VI], uu[VI];
        uint32_t cT = 0, cM = 0, cC = 0;
        // phase 1: the row's vertex
#pragma unroll
        for (int i = 0; i < VI; i++) {
            const uint32_t idx = base + i * VT + tid;
            uint32_t v = NIL, L = 0;
            if (idx < total) {
                if (a.vlist) {
                    v = a.vlist[idx] + a.vlist_base;
                    if (a.deg0) L = a.deg0[idx];
                } else if (!a.in.cnt) {
                    v = idx;  // dense range of vertices
                } else if (idx < nC) {
                    const uint2 c = a.in.C[idx];
                    if (c.y == 0) v = c.x;
                } else if (idx < nC + nM) {
                    v = a.in.M[idx - nC].x;
                } else {
                    v = a.in.T[idx - nC - nM].x;
                }
                if (v != NIL && v >= va.nvert) { set_err(st, ERR_BOUNDS, v); v = NIL; }
            }
            vv[i] = v;
            LL[i] = L;
        }
        // phase 2: its live length
#pragma unroll
        for (int i = 0; i < VI; i++) {
            if (vv[i] == NIL) continue;
            if (a.vlist && a.deg0) va.len[par][vv[i]] = LL[i];
            else LL[i] = va.len[par][vv[i]];
        }
        // phase 3: the mutual-choice test (two dependent gathers)
#pragma unroll
        for (int i = 0; i < VI; i++) {
            uu[i] = NIL;
            if (a.match && vv[i] != NIL && LL[i] > 0) uu[i] = va.cnbr[vv[i]];
        }
#pragma unroll
        for (int i = 0; i < VI; i++) {
            cls[i] = 0;
            if (uu[i] != NIL && uu[i] >= va.nvert) { set_err(st, ERR_BOUNDS, uu[i]); uu[i] = NIL; }
            const uint32_t back = (uu[i] != NIL) ? va.cnbr[uu[i]] : NIL;
            const uint32_t v = vv[i], L = LL[i];
            bool open_row = false;
            if (v != NIL && L > 0) {
                my_rows++;
                my_ent += L;
                const bool matched = a.match && back == v;
                if (matched) {
                    va.mate[v] = uu[i];
                    va.dead[v] = 1;
                    my_match++;
                } else {
                    open_row = true;
                    if (L <= TINY_MAX) { cls[i] = 1; cT++; }
                    else if (L <= CHUNK) { cls[i] = 2; cM++; }
                    else {
                        cls[i] = 3;
                        cC += (L + CHUNK - 1) / CHUNK;
                        if (a.match) va.len[par ^ 1][v] = 0;  // long rows gather their survivors atomically
                    }
                }
            }
            // per-graph counters, aggregated over the lanes of a warp that share a graph
            if (a.grounds) {
                const uint32_t g = (v != NIL && L > 0) ? (va.gid ? va.gid[v] : 0u) : NIL;
                const uint32_t same = __match_any_sync(FULL, g);
                if (g != NIL && lane == __ffs(same) - 1) atomicMax(&a.grounds[g], round + 1);
            }
            if (a.glive) {
                const uint32_t g = open_row ? (va.gid ? va.gid[v] : 0u) : NIL;
                const uint32_t same = __match_any_sync(FULL, g);
                if (g != NIL && lane == __ffs(same) - 1) atomicAdd(&a.glive[g], (uint32_t)__popc(same));
            }
        }
        // block-aggregated appends to the task lists
        uint32_t tot[3];
        block_excl_scan3(cT, cM, cC, s_tmp, tot);
        if (tid == 0) {
            s_base[0] = tot[0] ? atomicAdd(&a.out.cnt[0], tot[0]) : 0;
            s_base[1] = tot[1] ? atomicAdd(&a.out.cnt[1], tot[1]) : 0;
            s_base[2] = tot[2] ? atomicAdd(&a.out.cnt[2], tot[2]) : 0;
        }
        __syncthreads();
        uint32_t pT = s_base[0] + cT, pM = s_base[1] + cM, pC = s_base[2] + cC;
#pragma unroll
        for (int i = 0; i < VI; i++) {
            if (cls[i] == 1) {
                if (pT < a.out.capT) a.out.T[pT] = make_uint2(vv[i], LL[i]); else set_err(st, ERR_BOUNDS, pT);
                pT++;
            } else if (cls[i] == 2) {
                if (pM < a.out.capM) a.out.M[pM] = make_uint2(vv[i], LL[i]); else set_err(st, ERR_BOUNDS, pM);
                pM++;
            } else if (cls[i] == 3) {
                const uint32_t nch = (LL[i] + CHUNK - 1) / CHUNK;
                for (uint32_t c = 0; c < nch; c++, pC++) {
                    if (pC < a.out.capC) a.out.C[pC] = make_uint2(vv[i], c); else set_err(st, ERR_BOUNDS, pC);
                }
            }
        }
        __syncthreads();  // s_base / s_tmp reuse
    }

    // statistics of the round: live rows, live entries, matched vertices
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_rows += __shfl_xor_sync(FULL, my_rows, o);
        my_ent += __shfl_xor_sync(FULL, my_ent, o);
        my_match += __shfl_xor_sync(FULL, my_match, o);
    }
    if (lane == 0) { s_red[warp * 3] = my_rows; s_red[warp * 3 + 1] = my_ent; s_red[warp * 3 + 2] = my_match; }
    __syncthreads();
    if (tid == 0) {
        unsigned long long r = 0, e = 0, mt = 0;
        for (int w = 0; w < VT / 32; w++) { r += s_red[w * 3]; e += s_red[w * 3 + 1]; mt += s_red[w * 3 + 2]; }
        if (a.match) {
            if (r) atomicAdd(&st->live_rows, (uint32_t)r);
            if (e) atomicAdd(&st->live_ent, e);
            if (mt) atomicAdd(&st->matched2, mt);
        }
        // the last CTA closes the pass: consumed lists are emptied, round statistics recorded
        __threadfence();
        const uint32_t done = atomicAdd(&st->exit_v, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            if (a.in_set < 4) { st->lcnt[a.in_set][0] = 0; st->lcnt[a.in_set][1] = 0; st->lcnt[a.in_set][2] = 0; }
            if (a.match) {
                const uint32_t rows = ld_volatile_u32(&st->live_rows);
                const unsigned long long ent = *reinterpret_cast<volatile unsigned long long*>(&st->live_ent);
                if (round < 64) { st->ring_m[round] = ent / 2; st->ring_n[round] = rows; }
                if (rows == 0 && !st->done) { st->done = 1; st->rounds = round; }
                st->live_rows = 0;
                st->live_ent = 0;
                if (a.round_from_state) st->round = round + 1;
            }
            st->exit_v = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------- sweep
// Tasks: [0, nC) chunks of long rows, [nC, nC + nM) medium rows,
// [nC + nM, ...) batches of 32 tiny rows.  Warps take tasks round-robin.
#ifndef LM_SG
#define LM_SG 4
#endif
#ifndef LM_SWEEP_MINB
#define LM_SWEEP_MINB 1
#endif
constexpr int ST = 256;        // threads per CTA (8 independent warps)
constexpr int SG = LM_SG;      // groups of 32 entries loaded together by a warp

struct Src {                   // where one row's entries come from
    const uint32_t* nbr;
    const uint32_t* eid;
    const uint32_t* ordw;
    const uint64_t* key;
    uint32_t off;              // index of the row's entry 0 in those arrays
    uint32_t vbase, k0, k1;
};

template <bool INPUT>
__device__ __forceinline__ Src src_of(const SweepArgs& a, uint32_t v, uint32_t s0) {
    Src s;
    if (INPUT) {
        const SegIn& g = a.segs[a.va.gid ? a.va.gid[v] : 0];
        s.nbr = g.nbr; s.eid = g.eid; s.ordw = g.ordw; s.key = nullptr;
        s.off = s0 - g.ebase; s.vbase = g.vbase; s.k0 = g.k0; s.k1 = g.k1;
    } else {
        s.nbr = a.in_nbr; s.eid = nullptr; s.ordw = nullptr; s.key = a.in_key;
        s.off = s0; s.vbase = 0; s.k0 = 0; s.k1 = 0;
    }
    return s;
}

// Loads SG groups of a row's entries [j, j + 32*SG) (valid below `end`),
// applies the deletion test and yields (key, neighbour) per lane and group;
// key = 0 for entries that are not live.
template <bool INPUT, bool COMPACT>
__device__ __forceinline__ void load_groups(const SweepArgs& a, const Src& s, uint32_t j, uint32_t end, int lane,
                                            uint64_t key[SG], uint32_t u[SG]) {
    uint32_t e[SG], o[SG];
    // independent loads first: neighbours, and for round 0 the edge ids (and,
    // without a deletion test, the weights too)
#pragma unroll
    for (int i = 0; i < SG; i++) {
        const uint32_t q = j + i * 32 + lane;
        u[i] = NIL;
        key[i] = 0;
        e[i] = 0;
        o[i] = 0;
        if (q < end) {
            u[i] = __ldcs(s.nbr + s.off + q);
            if (INPUT) e[i] = __ldcs(s.eid + s.off + q);
            if (INPUT && !COMPACT) o[i] = __ldcs(s.ordw + s.off + q);
            if (!INPUT && !COMPACT) key[i] = __ldcs(s.key + s.off + q);
        }
    }
    bool keep[SG];
#pragma unroll
    for (int i = 0; i < SG; i++) {
        keep[i] = u[i] != NIL;
        if (keep[i]) {
            if (INPUT) u[i] += s.vbase;
            if (u[i] >= a.va.nvert) { set_err(a.st, ERR_BOUNDS, u[i]); keep[i] = false; }
            else if (COMPACT) keep[i] = a.va.dead[u[i]] == 0;
        }
    }
    // keys of the surviving entries
#pragma unroll
    for (int i = 0; i < SG; i++) {
        if (keep[i]) {
            const uint32_t q = j + i * 32 + lane;
            if (INPUT) {
                const uint32_t ow = COMPACT ? __ldcs(s.ordw + s.off + q) : o[i];
                key[i] = ((uint64_t)ow << 32) | perm_seed(e[i], s.k0, s.k1);
            } else if (COMPACT) {
                key[i] = __ldcs(s.key + s.off + q);
            }
        } else {
            key[i] = 0;
        }
    }
}

template <bool INPUT, bool COMPACT>
__device__ void do_warp_row(const SweepArgs& a, uint32_t v, uint32_t L, uint32_t j_begin, uint32_t j_end,
                            bool chunked, uint32_t task, int lane) {
    const VertexArrays& va = a.va;
    const uint32_t s0 = va.start[v];
    if ((uint64_t)s0 + L > a.ecap) { if (lane == 0) set_err(a.st, ERR_BOUNDS, v); return; }
    const Src s = src_of<INPUT>(a, v, s0);
    uint32_t* len_next = va.len[a.par ^ 1u];
    uint32_t cnt = 0;
    uint64_t bk = 0;
    uint32_t bu = NIL;
    const uint32_t lt = lanemask_lt();
    for (uint32_t j = j_begin; j < j_end; j += 32 * SG) {
        uint64_t key[SG];
        uint32_t u[SG];
        load_groups<INPUT, COMPACT>(a, s, j, j_end, lane, key, u);
        uint32_t ball[SG], sub = 0;
#pragma unroll
        for (int i = 0; i < SG; i++) {
            ball[i] = __ballot_sync(FULL, key[i] != 0);
            sub += __popc(ball[i]);
            kv_max(bk, bu, key[i], u[i]);
        }
        if (COMPACT && sub) {
            uint32_t base;
            if (chunked) {
                base = 0;
                if (lane == 0) base = atomicAdd(&len_next[v], sub);
                base = __shfl_sync(FULL, base, 0);
            } else {
                base = cnt;
            }
#pragma unroll
            for (int i = 0; i < SG; i++) {
                if (key[i] != 0) {
                    const uint32_t pos = base + __popc(ball[i] & lt);
                    a.out_key[s0 + pos] = key[i];
                    a.out_nbr[s0 + pos] = u[i];
                }
                base += __popc(ball[i]);
            }
        }
        cnt += sub;
    }
    warp_kv_max(bk, bu);
    if (!chunked) {
        if (lane == 0) {
            if (COMPACT) len_next[v] = cnt;
            if (bk) va.cnbr[v] = bu;
        }
        return;
    }
    // chunk of a long row: publish the partial maximum; the last chunk to finish
    // combines all partials of the row
    const uint32_t nch = (L + CHUNK - 1) / CHUNK;
    const uint32_t cbase = task - j_begin / CHUNK;
    uint32_t old = 0;
    if (lane == 0) {
        a.part[task] = make_ulonglong2(bk, bu);
        __threadfence();
        old = atomicAdd(&va.bcnt[v], 1u);
    }
    old = __shfl_sync(FULL, old, 0);
    if (old != nch - 1) return;
    __threadfence();
    uint64_t k = 0;
    uint32_t nb = NIL;
    for (uint32_t q = lane; q < nch; q += 32) {
        const ulonglong2 p = __ldcg(&a.part[cbase + q]);
        kv_max(k, nb, p.x, (uint32_t)p.y);
    }
    warp_kv_max(k, nb);
    if (lane == 0) {
        va.bcnt[v] = 0;
        if (k) va.cnbr[v] = nb;
    }
}

template <bool INPUT, bool COMPACT>
__device__ void do_tiny(const SweepArgs& a, uint32_t tb, uint32_t nT, int lane) {
    const VertexArrays& va = a.va;
    const uint32_t idx = tb * 32 + lane;
    if (idx >= nT) return;
    const uint2 tv = a.in.T[idx];
    const uint32_t v = tv.x, L = tv.y;
    if (v >= va.nvert || L > TINY_MAX) { set_err(a.st, ERR_BOUNDS, v); return; }
    const uint32_t s0 = va.start[v];
    if ((uint64_t)s0 + L > a.ecap) { set_err(a.st, ERR_BOUNDS, v); return; }
    const Src s = src_of<INPUT>(a, v, s0);
    uint32_t u[TINY_MAX], e[TINY_MAX];
#pragma unroll
    for (uint32_t i = 0; i < TINY_MAX; i++) {
        u[i] = NIL;
        e[i] = 0;
        if (i < L) {
            u[i] = s.nbr[s.off + i];
            if (INPUT) e[i] = s.eid[s.off + i];
        }
    }
    bool keep[TINY_MAX];
#pragma unroll
    for (uint32_t i = 0; i < TINY_MAX; i++) {
        keep[i] = u[i] != NIL;
        if (keep[i]) {
            if (INPUT) u[i] += s.vbase;
            if (u[i] >= va.nvert) { set_err(a.st, ERR_BOUNDS, u[i]); keep[i] = false; }
            else if (COMPACT) keep[i] = va.dead[u[i]] == 0;
        }
    }
    uint64_t key[TINY_MAX];
#pragma unroll
    for (uint32_t i = 0; i < TINY_MAX; i++) {
        key[i] = 0;
        if (keep[i]) {
            if (INPUT) key[i] = ((uint64_t)s.ordw[s.off + i] << 32) | perm_seed(e[i], s.k0, s.k1);
            else key[i] = s.key[s.off + i];
        }
    }
    uint32_t cnt = 0;
    uint64_t bk = 0;
    uint32_t bu = NIL;
#pragma unroll
    for (uint32_t i = 0; i < TINY_MAX; i++) {
        if (key[i]) {
            if (COMPACT) {
                a.out_key[s0 + cnt] = key[i];
                a.out_nbr[s0 + cnt] = u[i];
            }
            cnt++;
            kv_max(bk, bu, key[i], u[i]);
        }
    }
    if (COMPACT) va.len[a.par ^ 1u][v] = cnt;
    if (bk) va.cnbr[v] = bu;
}

template <bool INPUT, bool COMPACT>
__global__ void __launch_bounds__(ST, LM_SWEEP_MINB) k_sweep(const SweepArgs* __restrict__ pav) {
    const SweepArgs& a = *pav;
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * ST + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * ST) >> 5;
    const uint32_t nT = ld_volatile_u32(&a.in.cnt[0]);
    const uint32_t nM = ld_volatile_u32(&a.in.cnt[1]);
    const uint32_t nC = ld_volatile_u32(&a.in.cnt[2]);
    if (nT > a.in.capT || nM > a.in.capM || nC > a.in.capC) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(a.st, ERR_BOUNDS, nC);
        return;
    }
    const uint32_t total = nC + nM + (nT + 31) / 32;
    for (uint32_t t = gw; t < total; t += nw) {
        if (t < nC) {
            const uint2 c = a.in.C[t];
            const uint32_t v = c.x;
            if (v >= a.va.nvert) { if (lane == 0) set_err(a.st, ERR_BOUNDS, v); continue; }
            const uint32_t L = a.va.len[a.par][v];
            const uint32_t jb = c.y * CHUNK, je = min(L, jb + CHUNK);
            if (jb >= L) { if (lane == 0) set_err(a.st, ERR_BOUNDS, t); continue; }
            do_warp_row<INPUT, COMPACT>(a, v, L, jb, je, true, t, lane);
        } else if (t < nC + nM) {
            const uint2 mv = a.in.M[t - nC];
            if (mv.x >= a.va.nvert || mv.y > CHUNK) { if (lane == 0) set_err(a.st, ERR_BOUNDS, mv.x); continue; }
            do_warp_row<INPUT, COMPACT>(a, mv.x, mv.y, 0, mv.y, false, t, lane);
        } else {
            do_tiny<INPUT, COMPACT>(a, t - nC - nM, nT, lane);
        }
    }
}

// ---------------------------------------------------------------- graph construction
__global__ void k_build_degrees(const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n, uint32_t m,
                                uint32_t* deg, uint32_t* err) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t u = eu[e], v = ev[e];
        const uint32_t wb = __float_as_uint(w[e]);
        const bool nan = ((wb & 0x7F800000u) == 0x7F800000u) && (wb & 0x007FFFFFu);
        if (u >= n || v >= n || u == v || nan) {
            atomicOr(err, 1u);
            continue;
        }
        atomicAdd(&deg[u], 1u);
        atomicAdd(&deg[v], 1u);
    }
}

__global__ void k_build_fill(const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t m,
                             uint32_t* cursor, uint32_t* nbr, uint32_t* eid, uint32_t* ordw) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const uint32_t u = eu[e], v = ev[e];
        const uint32_t o = ord_of_bits(__float_as_uint(w[e]));
        const uint32_t pu = atomicAdd(&cursor[u], 1u);
        nbr[pu] = v; eid[pu] = e; ordw[pu] = o;
        const uint32_t pv = atomicAdd(&cursor[v], 1u);
        nbr[pv] = u; eid[pv] = e; ordw[pv] = o;
    }
}

__global__ void k_nonzero_flags(const uint32_t* deg, uint32_t n, uint32_t* flags) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) flags[v] = deg[v] ? 1u : 0u;
}

__global__ void k_build_rows(const uint32_t* deg, const uint32_t* rowidx, uint32_t n, uint32_t* vid0, uint32_t* rdeg0) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (deg[v]) {
            const uint32_t i = rowidx[v];
            vid0[i] = v;
            rdeg0[i] = deg[v];
        }
    }
}

__device__ __forceinline__ uint32_t graph_of(const uint32_t* gvbase, uint32_t ngraphs, uint32_t v) {
    uint32_t lo = 0, hi = ngraphs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (gvbase[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void k_union_setup(const uint32_t* gvbase, const uint32_t* ebase, const uint32_t* const* offs,
                              uint32_t ngraphs, uint32_t nvert, uint32_t* start, uint32_t* gid, uint32_t* len0) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nvert; v += stride) {
        const uint32_t g = graph_of(gvbase, ngraphs, v);
        const uint32_t i = v - gvbase[g];
        const uint32_t* off = offs[g];
        const uint32_t o0 = off[i], o1 = off[i + 1];
        start[v] = ebase[g] + o0;
        gid[v] = g;
        len0[v] = o1 - o0;
    }
}

// serving: vertices [vbase, vbase + n) of one request get their row starts and slot
__global__ void k_req_setup(const uint32_t* off, uint32_t n, uint32_t vbase, uint32_t ebase, uint32_t slot,
                            uint32_t* start, uint32_t* gid) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        start[vbase + i] = ebase + off[i];
        gid[vbase + i] = slot;
    }
}

__global__ void k_to_local(const uint32_t* mate_g, uint32_t vbase, uint32_t n, uint32_t* out,
                           unsigned long long* matched2) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const uint32_t v = base + threadIdx.x;
        bool m = false;
        if (v < n) {
            const uint32_t x = mate_g[vbase + v];
            out[v] = (x == NIL) ? NIL : x - vbase;
            m = x != NIL;
        }
        const uint32_t b = __ballot_sync(FULL, m);
        if (matched2 && (threadIdx.x & 31) == 0 && b) atomicAdd(matched2, (unsigned long long)__popc(b));
    }
}

__global__ void k_to_local_batch(const uint32_t* mate_u, const uint32_t* gvbase, uint32_t ngraphs,
                                 uint32_t* const* dst, unsigned long long* matched2, uint32_t nvert) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nvert; v += stride) {
        const uint32_t g = graph_of(gvbase, ngraphs, v);
        const uint32_t vb = gvbase[g];
        const uint32_t x = mate_u[v];
        uint32_t* d = dst[g];
        if (d) d[v - vb] = (x == NIL) ? NIL : x - vb;
        if (x != NIL && matched2) atomicAdd(&matched2[g], 1ull);
    }
}

// ---------------------------------------------------------------- exclusive scan (graph set-up only)
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 16, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* tmp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan(x, lane);
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    uint32_t before = 0;
    total = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) {
        if (w < warp) before += tmp[w];
        total += tmp[w];
    }
    __syncthreads();
    return before + incl - x;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* in, uint32_t count, uint32_t* sums) {
    __shared__ uint32_t tmp[SCAN_THREADS / 32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t x = 0;
    for (int i = 0; i < SCAN_ITEMS; i++)
        if (base + i < count) x += in[base + i];
    uint32_t total;
    block_excl_scan(x, tmp, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const uint32_t* in, uint32_t count,
                                                             const uint32_t* offsets, uint32_t* out) {
    __shared__ uint32_t tmp[SCAN_THREADS / 32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t x = 0;
    for (int i = 0; i < SCAN_ITEMS; i++) {
        v[i] = (base + i < count) ? in[base + i] : 0u;
        x += v[i];
    }
    uint32_t total;
    uint32_t run = block_excl_scan(x, tmp, total) + (offsets ? offsets[blockIdx.x] : 0u);
    for (int i = 0; i < SCAN_ITEMS; i++) {
        if (base + i < count) out[base + i] = run;
        run += v[i];
    }
}

size_t exclusive_scan_tmp_words(uint32_t count) {
    size_t words = 0;
    uint64_t c = count;
    while (c > SCAN_TILE) {
        c = (c + SCAN_TILE - 1) / SCAN_TILE;
        words += 2 * c + 2;  // block sums and their scan at this level
    }
    return words + 4;
}

int launch_exclusive_scan(void* stream, const uint32_t* in, uint32_t* out, uint32_t count, uint32_t* tmp,
                          size_t tmp_words) {
    cudaStream_t s = (cudaStream_t)stream;
    if (count == 0) return 0;
    const uint32_t blocks = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (blocks == 1) {
        k_scan_apply<<<1, SCAN_THREADS, 0, s>>>(in, count, nullptr, out);
        return (int)cudaGetLastError();
    }
    if (tmp_words < (size_t)blocks * 2 + 2) return (int)cudaErrorInvalidValue;
    uint32_t* sums = tmp;
    uint32_t* sums_scan = tmp + blocks;
    k_scan_reduce<<<blocks, SCAN_THREADS, 0, s>>>(in, count, sums);
    int e = launch_exclusive_scan(stream, sums, sums_scan, blocks, tmp + 2 * (size_t)blocks,
                                  tmp_words - 2 * (size_t)blocks);
    if (e) return e;
    k_scan_apply<<<blocks, SCAN_THREADS, 0, s>>>(in, count, sums_scan, out);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- launchers
static int g_sm_count[64];

int device_sm_count(int dev) {
    if (dev < 0 || dev >= 64) return 1;
    if (!g_sm_count[dev]) {
        int c = 0;
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        g_sm_count[dev] = c > 0 ? c : 1;
    }
    return g_sm_count[dev];
}

static int current_sms() {
    int dev = 0;
    cudaGetDevice(&dev);
    return device_sm_count(dev);
}

static uint32_t grid_for(uint64_t n, uint32_t per_block, uint32_t per_sm = 32) {
    uint64_t b = (n + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)current_sms() * per_sm;
    if (b > cap) b = cap;
    return b ? (uint32_t)b : 1u;
}

int launch_init(void* stream, const InitArgs* dargs) {
    k_init<<<current_sms() * 16, 256, 0, (cudaStream_t)stream>>>(dargs);
    return (int)cudaGetLastError();
}

static uint32_t vertex_grid() { return (uint32_t)current_sms() * 4; }

int launch_vertex(void* stream, const VertexArgs* dargs) {
    // a fixed grid: the pass iterates its rows block-strided (row counts live on the device)
    k_vertex<<<vertex_grid(), VT, 0, (cudaStream_t)stream>>>(dargs);
    return (int)cudaGetLastError();
}

template <bool I, bool C>
static uint32_t sweep_grid() {
    static int blocks_per_sm = 0;
    if (!blocks_per_sm) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<I, C>, ST, 0);
        blocks_per_sm = per > 0 ? per : 1;
    }
    return (uint32_t)(current_sms() * blocks_per_sm);
}

template <bool I, bool C>
static int launch_sweep_t(void* stream, const SweepArgs* dargs) {
    k_sweep<I, C><<<sweep_grid<I, C>(), ST, 0, (cudaStream_t)stream>>>(dargs);
    return (int)cudaGetLastError();
}
int launch_sweep_cand(void* stream, const SweepArgs* d) { return launch_sweep_t<true, false>(stream, d); }
int launch_sweep_input(void* stream, const SweepArgs* d) { return launch_sweep_t<true, true>(stream, d); }
int launch_sweep_live(void* stream, const SweepArgs* d) { return launch_sweep_t<false, true>(stream, d); }

int launch_build_degrees(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n,
                         uint32_t m, uint32_t* deg, uint32_t* err) {
    k_build_degrees<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(eu, ev, w, n, m, deg, err);
    return (int)cudaGetLastError();
}
int launch_build_fill(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t m,
                      uint32_t* cursor, uint32_t* nbr, uint32_t* eid, uint32_t* ordw) {
    k_build_fill<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(eu, ev, w, m, cursor, nbr, eid, ordw);
    return (int)cudaGetLastError();
}
int launch_nonzero_flags(void* stream, const uint32_t* deg, uint32_t n, uint32_t* flags) {
    k_nonzero_flags<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(deg, n, flags);
    return (int)cudaGetLastError();
}
int launch_build_rows(void* stream, const uint32_t* deg, const uint32_t* rowidx_excl, uint32_t n, uint32_t* vid0,
                      uint32_t* rdeg0) {
    k_build_rows<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(deg, rowidx_excl, n, vid0, rdeg0);
    return (int)cudaGetLastError();
}
int launch_union_setup(void* stream, const uint32_t* gvbase, const uint32_t* ebase, const uint32_t* const* offs,
                       uint32_t ngraphs, uint32_t nvert, uint32_t* start, uint32_t* gid, uint32_t* len0) {
    if (nvert == 0 || ngraphs == 0) return 0;
    k_union_setup<<<grid_for(nvert, 256), 256, 0, (cudaStream_t)stream>>>(gvbase, ebase, offs, ngraphs, nvert, start,
                                                                          gid, len0);
    return (int)cudaGetLastError();
}
int launch_req_setup(void* stream, const uint32_t* off, uint32_t n, uint32_t vbase, uint32_t ebase, uint32_t slot,
                     uint32_t* start, uint32_t* gid) {
    if (n == 0) return 0;
    k_req_setup<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(off, n, vbase, ebase, slot, start, gid);
    return (int)cudaGetLastError();
}
int launch_to_local(void* stream, const uint32_t* mate_global, uint32_t vbase, uint32_t n, uint32_t* out,
                    unsigned long long* matched2) {
    if (n == 0) return 0;
    k_to_local<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(mate_global, vbase, n, out, matched2);
    return (int)cudaGetLastError();
}
int launch_to_local_batch(void* stream, const uint32_t* mate_union, const uint32_t* gvbase, uint32_t ngraphs,
                          uint32_t* const* dst, unsigned long long* matched2, uint32_t nvert) {
    if (nvert == 0 || ngraphs == 0) return 0;
    k_to_local_batch<<<grid_for(nvert, 256), 256, 0, (cudaStream_t)stream>>>(mate_union, gvbase, ngraphs, dst,
                                                                             matched2, nvert);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- device-driven loop
// Decides whether the conditional loop of a job graph runs another pair of
// rounds: not once the edge set is empty or an error was recorded; after the
// round cap or LOOP_LIMIT_NS it records ERR_TIMEOUT and stops.
__global__ void k_loop_check(DevState* st, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    unsigned int go = 1;
    if (ld_volatile_u32(&st->done) || ld_volatile_u32(&st->err)) go = 0;
    else if (ld_volatile_u32(&st->round) > ld_volatile_u32(&st->max_rounds) ||
             globaltimer_ns() - st->t0_ns > LOOP_LIMIT_NS) {
        set_err(st, ERR_TIMEOUT, ld_volatile_u32(&st->round));
        go = 0;
    }
    cudaGraphSetConditional(h, go);
}

static cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, cudaGraphNode_t dep, void* func, dim3 grid,
                              dim3 block, void** params) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = params;
    return cudaGraphAddKernelNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

int build_job_graph(const JobArgs* dargs, DevState* st, void** exec_out) {
    *exec_out = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return (int)e;
    cudaGraphNode_t prev = nullptr, node = nullptr;
    // kernel parameters: one pointer to the arguments in device memory
    const InitArgs* p_init = &dargs->init;
    const VertexArgs* pv[4] = {&dargs->v[0], &dargs->v[1], &dargs->v[2], &dargs->v[3]};
    const SweepArgs* ps[4] = {&dargs->s[0], &dargs->s[1], &dargs->s[2], &dargs->s[3]};
    void* init_params[1] = {&p_init};
    void* vparams[4][1], *sparams[4][1];
    for (int k = 0; k < 4; k++) {
        vparams[k][0] = &pv[k];
        sparams[k][0] = &ps[k];
    }
    const dim3 vgrid(vertex_grid()), vblock(VT), sblock(ST);
    do {
        if ((e = add_kernel(g, &node, prev, (void*)k_init, dim3(current_sms() * 16), dim3(256), init_params))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_vertex, vgrid, vblock, vparams[0]))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_sweep<true, false>, dim3(sweep_grid<true, false>()), sblock,
                            sparams[0]))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_vertex, vgrid, vblock, vparams[1]))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_sweep<true, true>, dim3(sweep_grid<true, true>()), sblock,
                            sparams[1]))) break;
        prev = node;
        cudaGraphConditionalHandle h;
        if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault))) break;
        alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
        memset(cp_raw, 0, sizeof cp_raw);
        cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if ((e = cudaGraphAddNode(&node, g, &prev, nullptr, 1, &cp))) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t bp = nullptr, bn = nullptr;
        for (int k = 2; k < 4 && e == cudaSuccess; k++) {
            if ((e = add_kernel(body, &bn, bp, (void*)k_vertex, vgrid, vblock, vparams[k]))) break;
            bp = bn;
            if ((e = add_kernel(body, &bn, bp, (void*)k_sweep<false, true>, dim3(sweep_grid<false, true>()), sblock,
                                sparams[k]))) break;
            bp = bn;
        }
        if (e) break;
        void* cparams[2] = {&st, &h};
        if ((e = add_kernel(body, &bn, bp, (void*)k_loop_check, dim3(1), dim3(32), cparams))) break;
        cudaGraphExec_t ex = nullptr;
        if ((e = cudaGraphInstantiate(&ex, g, 0))) break;
        *exec_out = ex;
    } while (0);
    cudaGraphDestroy(g);
    return (int)e;
}

int launch_job_graph(void* exec, void* stream) {
    return (int)cudaGraphLaunch((cudaGraphExec_t)exec, (cudaStream_t)stream);
}

void destroy_job_graph(void* exec) {
    if (exec) cudaGraphExecDestroy((cudaGraphExec_t)exec);
}

}  // namespace lm
