// sm_103a kernels of the local-max matching path.
//
// One local-max round (the phase of Sec. 2, steps 1-6) is two launches:
//
//   k_vertex   one thread per live vertex v: u = cnbr[v] is the neighbour of
//              v's heaviest live edge; if cnbr[u] == v the edge is chosen by
//              both ends and joins M (step 3; both ends write their own mate
//              slot, so no conflict).  The same pass indexes the live entries
//              in tiles for the coming sweep.
//   k_sweep    one persistent pass over the live adjacency entries, in tiles
//              of SWEEP_T entries: an entry survives when neither endpoint is
//              matched (steps 4 and 5: the deletion flag of a vertex is its
//              own dead[] byte, so spreading it over the vertex's edges is
//              one read per row); survivors are compacted in order (step 6)
//              and, in the same pass, every vertex's heaviest surviving edge
//              is found by a segmented maximum over its row (step 2 of the
//              next round, Lemma "broadcast").  Tile results are chained by a
//              decoupled look-back whose carried state is the segmented
//              aggregate of lm_internal.h, so rows cut by tile boundaries get
//              both their compacted position and their maximum in this pass.
//
// Round 0 reads the graph's own CSR (neighbour, edge id, ord(weight)) and
// builds the 64-bit keys K(e) = ord(w) << 32 | perm_seed(e) on the fly; it
// runs one candidate-only sweep, the match, then a compacting sweep.
#include <cuda_runtime.h>
#include <stdint.h>
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
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}
__device__ __forceinline__ void set_err(DevState* st, uint32_t bit, uint32_t info) {
    if ((atomicOr(&st->err, bit) & bit) == 0) st->err_info = info;
}

// The wait for a predecessor tile is bounded: after LOOKBACK_LIMIT_NS (or as
// soon as any tile of the launch has given up) the sweep records ERR_TIMEOUT,
// treats the missing tiles as empty and carries on; every index stays
// checked, so nothing runs out of bounds and the kernel ends.
constexpr uint64_t LOOKBACK_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ uint4 ld_volatile_v4(const uint32_t* p) {
    uint4 v;
    asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_volatile_v4(uint32_t* p, uint4 v) {
    asm volatile("st.volatile.global.v4.u32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}
// A tile's descriptor is one aligned 16-byte word written and read with
// single vector accesses, so a reader sees either the aggregate or the
// inclusive prefix, never a mix.
__device__ __forceinline__ void publish_desc(uint32_t* desc, uint32_t t, uint32_t epoch, uint32_t kind, const Agg& A) {
    st_volatile_v4(desc + 4 * (size_t)t, make_uint4((epoch << 2) | kind, A.S, A.nr, A.f));
}

// Exclusive prefix of tile t >= 1, computed by one full warp; every lane
// returns the same value.  A window covers LB_PER_LANE * 32 predecessors read
// in one round trip: lane l watches tiles base - LB_PER_LANE*l - q.  Only the
// tiles between this one and the nearest inclusive prefix are waited for; the
// window is combined oldest first (inside a lane, then by an ordered tree
// reduction over lanes).
constexpr int LB_PER_LANE = 4;

__device__ Agg lookback(const SweepArgs& a, uint32_t t, uint32_t epoch, int lane, bool& timed_out) {
    Agg suf = agg_identity();
    int64_t base = (int64_t)t - 1;
    const uint64_t t_start = globaltimer_ns();
    const uint4 empty_incl = make_uint4((epoch << 2) | 2u, 0u, 0u, F_H);  // below tile 0: an empty prefix
    for (;;) {
        uint4 d[LB_PER_LANE];
        bool valid[LB_PER_LANE];
#pragma unroll
        for (int q = 0; q < LB_PER_LANE; q++) {
            d[q] = empty_incl;
            valid[q] = base - (int64_t)(LB_PER_LANE * lane + q) < 0;
        }
        uint32_t my_incl = LB_PER_LANE;  // nearest inclusive element inside this lane
        for (int spins = 0;; spins++) {
#pragma unroll
            for (int q = 0; q < LB_PER_LANE; q++) {
                if (!valid[q]) {
                    d[q] = ld_volatile_v4(a.lb_desc + 4 * (size_t)(base - (LB_PER_LANE * lane + q)));
                    valid[q] = (d[q].x >> 2) == epoch && (d[q].x & 3u) != 0;
                }
            }
            // this lane is ready when its elements up to its first inclusive one are valid
            bool ready = true;
            my_incl = LB_PER_LANE;
#pragma unroll
            for (int q = LB_PER_LANE - 1; q >= 0; q--)
                if (valid[q] && (d[q].x & 3u) == 2u) my_incl = q;
#pragma unroll
            for (int q = 0; q < LB_PER_LANE; q++)
                if (q <= (int)my_incl && q < LB_PER_LANE && !valid[q]) ready = false;
            const uint32_t imask = __ballot_sync(FULL, my_incl < LB_PER_LANE);
            const uint32_t rmask = __ballot_sync(FULL, ready);
            const uint32_t need = imask ? ((2u << (__ffs(imask) - 1)) - 1u) : FULL;  // lanes up to the first inclusive
            if ((rmask & need) == need) break;
            if (spins > 8) {
                bool give_up = false;
                if (lane == 0)
                    give_up = globaltimer_ns() - t_start > LOOKBACK_LIMIT_NS || (ld_volatile_u32(&a.st->err) & ERR_TIMEOUT);
                if (__shfl_sync(FULL, give_up, 0)) {
                    timed_out = true;
#pragma unroll
                    for (int q = 0; q < LB_PER_LANE; q++)
                        if (!valid[q]) { d[q] = empty_incl; valid[q] = true; }
                    my_incl = 0;
                    break;
                }
                __nanosleep(spins < 64 ? 32 : 256);
            }
        }
        const uint32_t imask = __ballot_sync(FULL, my_incl < LB_PER_LANE);
        const int jl = imask ? __ffs(imask) - 1 : 32;
        // combine this lane's elements oldest first, cut at the nearest inclusive one
        Agg v = agg_identity();
        if (lane <= jl) {
            const int qmax = (lane == jl) ? (int)my_incl : LB_PER_LANE - 1;
#pragma unroll
            for (int q = LB_PER_LANE - 1; q >= 0; q--) {
                if (q <= qmax) {
                    Agg x;
                    x.S = d[q].y; x.nr = d[q].z; x.f = d[q].w;
                    v = agg_combine(v, x);
                }
            }
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Agg w;
            w.S = __shfl_down_sync(FULL, v.S, o);
            w.nr = __shfl_down_sync(FULL, v.nr, o);
            w.f = __shfl_down_sync(FULL, v.f, o);
            if (lane + o < 32) v = agg_combine(w, v);
        }
        v.S = __shfl_sync(FULL, v.S, 0);
        v.nr = __shfl_sync(FULL, v.nr, 0);
        v.f = __shfl_sync(FULL, v.f, 0);
        suf = agg_combine(v, suf);
        if (imask) return suf;
        base -= 32 * LB_PER_LANE;
    }
}

// ---------------------------------------------------------------- sweep
struct SweepSmem {
    uint64_t kmax[SWEEP_T + 1];      // per local row: max surviving key (0 = none)
    uint32_t off[SWEEP_T + 2];       // offsets of rows r_lo .. r_lo + nload
    uint32_t vid[SWEEP_T + 1];       // global vertex id per local row
    uint32_t knbr[SWEEP_T + 1];      // neighbour of kmax
    uint32_t cnt[SWEEP_T + 1];       // survivors per local row
    uint32_t rsw[SWEEP_GROUPS];      // row-start bitmap of the tile's entries
    uint32_t rsw_pre[SWEEP_GROUPS];  // exclusive popcount prefix of rsw
    uint32_t wS[SWEEP_WARPS];        // survivors per warp
    uint32_t scanS[SWEEP_WARPS], scanE[SWEEP_WARPS];
    Agg pre;                         // exclusive prefix of the tile
    Agg tot;                         // aggregate of the tile
    uint64_t hk_fin;                 // head row: maximum over earlier tiles (0 = none)
    uint32_t hu_fin;
    uint32_t tile, j0, nent, r_lo, nload, nrt, b0, seg, tile_begin;
    uint32_t vbase, k0, k1, last, bad;
    uint8_t rdead[SWEEP_T + 4];      // per local row: vertex matched this round
};

template <bool INPUT, bool COMPACT>
__global__ void __launch_bounds__(SWEEP_THREADS, 3) k_sweep(const SweepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepSmem& s = *reinterpret_cast<SweepSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    DevState* st = a.st;

    uint32_t ntiles, live_ent = 0, live_rows = 0;
    if (INPUT) {
        ntiles = a.ntiles_in;
    } else {
        live_ent = ld_volatile_u32(&st->cnt[a.in_buf][0]);
        live_rows = ld_volatile_u32(&st->cnt[a.in_buf][1]);
        ntiles = (live_ent + SWEEP_T - 1) / SWEEP_T;
    }
    if (ntiles == 0) {
        if (COMPACT && blockIdx.x == 0 && tid == 0) {
            const uint32_t S0 = a.prefix_in ? ld_volatile_u32(&a.prefix_in[0]) : 0u;
            const uint32_t N0 = a.prefix_in ? ld_volatile_u32(&a.prefix_in[1]) : 0u;
            st->cnt[a.out_buf][0] = S0;
            st->cnt[a.out_buf][1] = N0;
            if (N0 <= a.out_rows_cap) a.out_off[N0] = S0;
        }
        return;
    }
    const uint32_t epoch = ld_volatile_u32(&st->epoch) & 0x3FFFFFFFu;
    if (ntiles > a.lb_cap) {
        if (blockIdx.x == 0 && tid == 0) set_err(st, ERR_BOUNDS, ntiles);
        return;  // no tile is processed, so no look-back record is awaited
    }

    for (;;) {
        // ------------------------------------------------ locate the tile
        // (ids are taken when a tile starts, so every earlier tile has started)
        if (tid == 0) {
            const uint32_t t = atomicAdd(&st->tile_ctr, 1u);
            s.tile = t;
            if (t < ntiles) {
                uint32_t lt = t, nrows_seg, nent_seg;
                const uint32_t* tm;
                if (INPUT) {
                    uint32_t lo = 0, hi = a.nsegs - 1;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (a.segs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
                    }
                    const SegDesc& sg = a.segs[lo];
                    s.seg = lo;
                    s.tile_begin = sg.tile_begin;
                    lt = t - sg.tile_begin;
                    tm = sg.tilemap;
                    nrows_seg = sg.nrows;
                    nent_seg = sg.nent;
                    s.vbase = sg.vbase; s.k0 = sg.k0; s.k1 = sg.k1;
                } else {
                    tm = a.in_tilemap;
                    nrows_seg = live_rows;
                    nent_seg = live_ent;
                    s.seg = 0; s.tile_begin = 0; s.vbase = 0; s.k0 = 0; s.k1 = 0;
                }
                const uint32_t j0 = lt * SWEEP_T;
                uint32_t nent = min((uint32_t)SWEEP_T, nent_seg - j0);
                uint32_t r_lo = tm[lt];
                const uint32_t r_nx = tm[lt + 1];
                uint32_t bad = 0;
                uint32_t r_cap = 0;
                if (nrows_seg == 0 || r_lo >= nrows_seg) {
                    bad = 1;
                } else {
                    r_cap = min(r_nx, nrows_seg - 1);
                    if (r_lo > r_cap || r_cap - r_lo > (uint32_t)SWEEP_T) bad = 1;
                }
                if (bad) {
                    // inconsistent tile index: record it and process the tile as empty
                    set_err(st, ERR_BOUNDS, t);
                    nent = 0; r_lo = 0; r_cap = 0;
                }
                s.bad = bad;
                s.j0 = j0; s.nent = nent; s.r_lo = r_lo; s.nload = bad ? 0u : r_cap - r_lo + 1;
                s.last = (t == ntiles - 1);
            }
        }
        __syncthreads();
        const uint32_t t = s.tile;
        if (t >= ntiles) break;

        const uint32_t* r_off;
        const uint32_t* r_vid;
        if (INPUT) { r_off = a.segs[s.seg].off; r_vid = a.segs[s.seg].vid; }
        else { r_off = a.in_off; r_vid = a.in_vid; }
        const uint32_t j0 = s.j0, nent = s.nent, r_lo = s.r_lo, nload = s.nload, vbase = s.vbase;

        // ------------------------------------------------ row data
        const bool bad = s.bad != 0;
        if (!bad)
            for (uint32_t i = tid; i <= nload; i += SWEEP_THREADS) s.off[i] = r_off[r_lo + i];
        else if (tid == 0) { s.off[0] = j0; s.off[1] = j0; s.vid[0] = 0; s.kmax[0] = 0; s.knbr[0] = NIL; s.cnt[0] = 0; s.rdead[0] = 1; }
        for (uint32_t i = tid; i < nload; i += SWEEP_THREADS) {
            uint32_t v = r_vid[r_lo + i] + vbase;
            if (v >= a.nvert) { set_err(st, ERR_BOUNDS, v); v = 0; }
            s.vid[i] = v;
            s.kmax[i] = 0;
            s.knbr[i] = NIL;
            s.cnt[i] = 0;
            s.rdead[i] = COMPACT ? a.dead[v] : 0;
        }
        for (int i = tid; i < SWEEP_GROUPS; i += SWEEP_THREADS) s.rsw[i] = 0;
        __syncthreads();
        for (uint32_t i = tid; i < nload; i += SWEEP_THREADS) {
            const uint32_t p = s.off[i];
            if (p >= j0 && p < j0 + nent) atomicOr(&s.rsw[(p - j0) >> 5], 1u << ((p - j0) & 31));
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t w0 = s.rsw[2 * lane], w1 = s.rsw[2 * lane + 1];
            const uint32_t c0 = __popc(w0), sum = c0 + __popc(w1);
            const uint32_t incl = warp_incl_scan(sum, lane);
            s.rsw_pre[2 * lane] = incl - sum;
            s.rsw_pre[2 * lane + 1] = incl - sum + c0;
            if (lane == 31) {
                const uint32_t b0 = (s.off[0] == j0) ? 1u : 0u;
                s.b0 = b0;
                s.nrt = incl + (1u - b0);
            }
        }
        __syncthreads();
        const uint32_t b0 = s.b0, nrt = s.nrt;

        // ------------------------------------------------ entries: load
        uint64_t key[SWEEP_GPW];
        uint32_t ug[SWEEP_GPW], lr[SWEEP_GPW], sm[SWEEP_GPW];
        const uint32_t* in_nbr;
        const uint32_t* in_eid = nullptr;
        const uint32_t* in_ordw = nullptr;
        if (INPUT) {
            const SegDesc& sg = a.segs[s.seg];
            in_nbr = sg.nbr; in_eid = sg.eid; in_ordw = sg.ordw;
        } else {
            in_nbr = a.in_nbr;
        }
        const uint32_t k0 = s.k0, k1 = s.k1;
        uint32_t eidv[SWEEP_GPW];
#pragma unroll
        for (int i = 0; i < SWEEP_GPW; i++) {
            const int g = warp * SWEEP_GPW + i;
            const uint32_t q = (uint32_t)g * 32u + lane;
            const uint32_t word = s.rsw[g];
            const uint32_t r = s.rsw_pre[g] + __popc(word & (FULL >> (31 - lane))) - b0;
            lr[i] = r;
            bool live = false;
            if (q < nent) live = (r < nrt) ? (s.rdead[r] == 0) : false;
            key[i] = 0;
            ug[i] = NIL;
            eidv[i] = 0;
            if (live) {
                const uint32_t j = j0 + q;
                ug[i] = in_nbr[j];
                if (INPUT) {
                    eidv[i] = in_eid[j];
                    key[i] = (uint64_t)in_ordw[j] << 32;
                } else {
                    key[i] = a.in_key[j];
                }
            }
        }
        // ------------------------------------------------ entries: deletion test, per-row max / count
#pragma unroll
        for (int i = 0; i < SWEEP_GPW; i++) {
            bool surv = key[i] != 0;
            if (surv) {
                if (INPUT) {
                    ug[i] += vbase;
                    key[i] |= perm_seed(eidv[i], k0, k1);
                }
                if (ug[i] >= a.nvert) { set_err(st, ERR_BOUNDS, ug[i]); surv = false; }
                else if (COMPACT) surv = a.dead[ug[i]] == 0;
            }
            if (!surv) key[i] = 0;
        }
#pragma unroll
        for (int i = 0; i < SWEEP_GPW; i++) {
            const int g = warp * SWEEP_GPW + i;
            const bool surv = key[i] != 0;
            const uint32_t ball = __ballot_sync(FULL, surv);
            sm[i] = ball;
            if ((s.rsw[g] & 0xFFFFFFFEu) == 0) {
                // the whole group lies in one row (the row of lane 0)
                if (ball) {
                    const uint32_t hi = __reduce_max_sync(FULL, (uint32_t)(key[i] >> 32));
                    const uint32_t lo = __reduce_max_sync(FULL, ((uint32_t)(key[i] >> 32) == hi) ? (uint32_t)key[i] : 0u);
                    if (lane == 0) {
                        atomicMax(reinterpret_cast<unsigned long long*>(&s.kmax[lr[i]]),
                                  (unsigned long long)(((uint64_t)hi << 32) | lo));
                        if (COMPACT) atomicAdd(&s.cnt[lr[i]], (uint32_t)__popc(ball));
                    }
                }
            } else if (surv) {
                atomicMax(reinterpret_cast<unsigned long long*>(&s.kmax[lr[i]]), (unsigned long long)key[i]);
                if (COMPACT) atomicAdd(&s.cnt[lr[i]], 1u);
            }
        }
        __syncthreads();
        uint32_t wsum = 0;
#pragma unroll
        for (int i = 0; i < SWEEP_GPW; i++) {
            if (key[i] != 0 && key[i] == s.kmax[lr[i]]) s.knbr[lr[i]] = ug[i];
            wsum += __popc(sm[i]);
        }
        if (lane == 0) s.wS[warp] = wsum;

        // ------------------------------------------------ row scans (survivor counts, new rows)
        const uint32_t rbeg = min((uint32_t)tid * SWEEP_RPT, nrt);
        const uint32_t rend = min(rbeg + SWEEP_RPT, nrt);
        __syncthreads();
        uint32_t cS = 0, cE = 0;
        if (COMPACT) {
            for (uint32_t r = rbeg; r < rend; r++) {
                const uint32_t c = s.cnt[r];
                cS += c;
                if ((r > 0 || b0) && c > 0) cE++;
            }
        }
        uint32_t oS = 0, oE = 0;
        if (COMPACT) {
            const uint32_t iS = warp_incl_scan(cS, lane), iE = warp_incl_scan(cE, lane);
            if (lane == 31) { s.scanS[warp] = iS; s.scanE[warp] = iE; }
            __syncthreads();
            uint32_t bS = 0, bE = 0, TS = 0, TE = 0;
#pragma unroll
            for (int w = 0; w < SWEEP_WARPS; w++) {
                if (w < warp) { bS += s.scanS[w]; bE += s.scanE[w]; }
                TS += s.scanS[w]; TE += s.scanE[w];
            }
            oS = bS + iS - cS;
            oE = bE + iE - cE;
            if (tid == 0) { s.tot.S = TS; s.tot.nr = TE; }
        }
        if (tid == 0) {
            // aggregate flags and partial maxima of the tile
            Agg& A = s.tot;
            if (!COMPACT) { A.S = 0; A.nr = 0; }
            const bool h = b0 || nrt > 1;
            Part P;
            P.pad0 = P.pad1 = 0;
            if (!b0 && nrt > 0) { P.hk = s.kmax[0]; P.hu = s.knbr[0]; } else { P.hk = 0; P.hu = NIL; }
            if (h && nrt > 0) { P.tk = s.kmax[nrt - 1]; P.tu = s.knbr[nrt - 1]; }
            else if (h) { P.tk = 0; P.tu = NIL; }
            else { P.tk = P.hk; P.tu = P.hu; }
            A.f = (h ? F_H : 0u) | (P.hk ? F_HS : 0u) | (P.tk ? F_TS : 0u);
            __stcg(reinterpret_cast<ulonglong2*>(&a.lb_part[t]), make_ulonglong2(P.hk, P.tk));
            __stcg(reinterpret_cast<uint4*>(&a.lb_part[t]) + 1, make_uint4(P.hu, P.tu, 0u, 0u));
        }
        __syncthreads();

        // ------------------------------------------------ look-back
        if (warp == 0) {
            const Agg A = s.tot;
            Agg P = agg_identity();
            bool to = false;
            if (t == 0) {
                P.f = F_H;
                if (a.prefix_in) {
                    P.S = ld_volatile_u32(&a.prefix_in[0]);
                    P.nr = ld_volatile_u32(&a.prefix_in[1]);
                }
            } else {
                if (lane == 0) {
                    __threadfence();  // partial maxima before the aggregate
                    publish_desc(a.lb_desc, t, epoch, 1u, A);
                }
                P = lookback(a, t, epoch, lane, to);
                to = __any_sync(FULL, to);
            }
            Agg I = agg_combine(P, A);
            I.f = F_H | (I.f & F_TS);
            if (lane == 0) {
                if (to) set_err(st, ERR_TIMEOUT, t);
                if (t == 0) __threadfence();
                publish_desc(a.lb_desc, t, epoch, 2u, I);
                s.pre = P;
                if (COMPACT && s.last) {
                    // totals of the sweep: sentinel offset and the next round's counts
                    uint32_t S_tot = I.S, N_tot = I.nr;
                    if (N_tot > a.out_rows_cap || S_tot > a.out_cap) {
                        set_err(st, ERR_BOUNDS, N_tot);
                        S_tot = 0; N_tot = 0;  // stop the loop rather than read past the arrays
                    }
                    a.out_off[N_tot] = S_tot;
                    st->cnt[a.out_buf][0] = S_tot;
                    st->cnt[a.out_buf][1] = N_tot;
                    const uint32_t rn = a.round + 1;
                    if (rn < 64) { st->ring_m[rn] = S_tot / 2; st->ring_n[rn] = N_tot; }
                    if (S_tot == 0) st->rounds = rn;
                }
            }
            // head row continuing from earlier tiles: gather its maximum from their
            // partials (all earlier tiles have published them: the look-back saw
            // every one of them at least as an aggregate)
            const bool need_head = !bad && !b0 && nrt > 0 && (nrt > 1 || s.off[nrt] == j0 + nent);
            uint64_t hk = 0;
            uint32_t hu = NIL;
            if (need_head) {
                __threadfence();
                const uint32_t gt_start = s.tile_begin + s.off[0] / SWEEP_T;  // tile where the row starts
                for (uint32_t k = gt_start + lane; k < t; k += 32) {
                    const Part* pp = &a.lb_part[k];
                    const ulonglong2 kk = __ldcg(reinterpret_cast<const ulonglong2*>(pp));
                    const uint4 uu = __ldcg(reinterpret_cast<const uint4*>(pp) + 1);
                    // the start tile contributes its tail, the tiles after it their whole (head) part
                    if (k == gt_start) kv_max(hk, hu, kk.y, uu.y);
                    else kv_max(hk, hu, kk.x, uu.x);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint64_t k2 = __shfl_xor_sync(FULL, hk, o);
                    const uint32_t u2 = __shfl_xor_sync(FULL, hu, o);
                    kv_max(hk, hu, k2, u2);
                }
            }
            if (lane == 0) { s.hk_fin = hk; s.hu_fin = hu; }
        }
        __syncthreads();
        const Agg P = s.pre;

        // ------------------------------------------------ compacted entries
        if (COMPACT) {
            uint32_t base = P.S;
            for (int w = 0; w < warp; w++) base += s.wS[w];
            const uint32_t lt_mask = lanemask_lt();
#pragma unroll
            for (int i = 0; i < SWEEP_GPW; i++) {
                if (key[i] != 0) {
                    const uint32_t pos = base + __popc(sm[i] & lt_mask);
                    if (pos < a.out_cap) {
                        a.out_key[pos] = key[i];
                        a.out_nbr[pos] = ug[i];
                    } else {
                        set_err(st, ERR_BOUNDS, pos);
                    }
                }
                base += __popc(sm[i]);
            }
        }
        // ------------------------------------------------ rows: compacted rows, next candidates
        {
            const bool head_cont = (b0 == 0);
            const bool prev_surv = (P.f & F_TS) != 0;
            const bool head_new = COMPACT && head_cont && s.cnt[0] > 0 && !prev_surv;
            uint32_t posr = P.S + oS;
            uint32_t idx = P.nr + (head_new ? 1u : 0u) + oE;
            const bool last_ends = (s.off[nrt] == j0 + nent);
            for (uint32_t r = rbeg; r < rend; r++) {
                const bool is_head = head_cont && r == 0;
                if (COMPACT) {
                    const uint32_t c = s.cnt[r];
                    const bool isnew = !bad && (is_head ? head_new : (c > 0));
                    if (isnew) {
                        const uint32_t ni = is_head ? P.nr : idx;
                        if (ni < a.out_rows_cap) {
                            a.out_off[ni] = posr;
                            a.out_vid[ni] = s.vid[r];
                        } else {
                            set_err(st, ERR_BOUNDS, ni);
                        }
                        if (!is_head) idx++;
                    }
                    posr += c;
                }
                if (!bad && (r + 1 < nrt || last_ends)) {
                    uint64_t k = s.kmax[r];
                    uint32_t u = s.knbr[r];
                    if (is_head) kv_max(k, u, s.hk_fin, s.hu_fin);
                    if (k != 0) a.cnbr[s.vid[r]] = u;
                }
            }
        }
        __syncthreads();
    }

    // every CTA passes here once; the last one resets the tile counter for
    // the next sweep and advances the look-back generation
    if (tid == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&st->exit_ctr, 1u);
        if (done == gridDim.x - 1) {
            st->tile_ctr = 0;
            st->exit_ctr = 0;
            uint32_t e = (st->epoch + 1) & 0x3FFFFFFFu;
            st->epoch = e ? e : 1u;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------- vertex pass
__device__ __forceinline__ void count_matched(DevState* st, bool m) {
    const uint32_t b = __ballot_sync(FULL, m);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&st->matched2, (unsigned long long)__popc(b));
}

__device__ __forceinline__ void note_round(const VertexArgs& a, uint32_t v) {
    if (!a.grounds) return;
    uint32_t lo = 0, hi = a.ngraphs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (a.gvbase[mid] <= v) lo = mid; else hi = mid - 1;
    }
    atomicMax(&a.grounds[lo], a.round + 1);
}

// round 0: the vertices [vbegin, vbegin + vcount); a vertex with a candidate has cnbr != NIL
__global__ void __launch_bounds__(256) k_vertex_all(const VertexArgs a) {
    const uint32_t n = a.nvert;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x; base < a.vcount; base += stride) {
        const uint32_t v = a.vbegin + base + threadIdx.x;
        bool m = false;
        if (base + threadIdx.x < a.vcount && v < n) {
            const uint32_t u = a.cnbr[v];
            if (u != NIL) {
                if (u >= n) set_err(a.st, ERR_BOUNDS, u);
                else if (a.cnbr[u] == v) {
                    a.mate[v] = u;
                    a.dead[v] = 1;
                    m = true;
                    note_round(a, v);
                }
            }
        }
        count_matched(a.st, m);
    }
}

// rounds >= 1: the live rows of the compacted arrays
__global__ void __launch_bounds__(256) k_vertex_live(const VertexArgs a) {
    DevState* st = a.st;
    const uint32_t R = ld_volatile_u32(&st->cnt[a.in_buf][1]);
    const uint32_t E = ld_volatile_u32(&st->cnt[a.in_buf][0]);
    if (R == 0) return;
    const uint32_t ntiles = (E + SWEEP_T - 1) / SWEEP_T;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = blockIdx.x * blockDim.x; base < R; base += stride) {
        const uint32_t i = base + threadIdx.x;
        bool m = false;
        if (i < R) {
            const uint32_t v = a.vid[i];
            if (v >= a.nvert) {
                set_err(st, ERR_BOUNDS, v);
            } else {
                const uint32_t u = a.cnbr[v];
                if (u >= a.nvert) set_err(st, ERR_BOUNDS, u);
                else if (a.cnbr[u] == v) {
                    a.mate[v] = u;
                    a.dead[v] = 1;
                    m = true;
                    note_round(a, v);
                }
            }
            const uint32_t lo = a.off[i], hi = a.off[i + 1];
            for (uint32_t tt = (lo + SWEEP_T - 1) / SWEEP_T; tt < (hi + SWEEP_T - 1) / SWEEP_T; tt++) {
                if (tt < a.tilemap_cap) a.tilemap[tt] = i;
                else set_err(st, ERR_BOUNDS, tt);
            }
            if (i == R - 1) {
                if (ntiles < a.tilemap_cap) a.tilemap[ntiles] = R;
                else set_err(st, ERR_BOUNDS, ntiles);
            }
        }
        count_matched(st, m);
    }
}

// ---------------------------------------------------------------- init
__global__ void k_init(uint32_t* mate, uint32_t* cnbr, uint8_t* dead, uint32_t n, DevState* st) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (mate) mate[v] = NIL;
        cnbr[v] = NIL;
        dead[v] = 0;
    }
    if (st && blockIdx.x == 0) {
        for (int i = threadIdx.x; i < 64; i += blockDim.x) { st->ring_m[i] = 0; st->ring_n[i] = 0; }
        if (threadIdx.x == 0) {
            st->cnt[0][0] = st->cnt[0][1] = st->cnt[1][0] = st->cnt[1][1] = 0;
            st->err = 0;
            st->err_info = 0;
            st->rounds = 0;
            st->matched2 = 0;
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

__global__ void k_build_rows(const uint32_t* deg, const uint32_t* rowidx, const uint32_t* off_all, uint32_t n,
                             uint32_t nrows, uint32_t nent, uint32_t* off0, uint32_t* vid0) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (deg[v]) {
            const uint32_t i = rowidx[v];
            off0[i] = off_all[v];
            vid0[i] = v;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off0[nrows] = nent;
}

__global__ void k_build_tilemap(const uint32_t* off0, uint32_t nrows, uint32_t nent, uint32_t* tilemap) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t ntiles = (nent + SWEEP_T - 1) / SWEEP_T;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += stride) {
        const uint32_t lo = off0[i], hi = off0[i + 1];
        for (uint32_t tt = (lo + SWEEP_T - 1) / SWEEP_T; tt < (hi + SWEEP_T - 1) / SWEEP_T; tt++) tilemap[tt] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) tilemap[ntiles] = nrows;
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

__device__ __forceinline__ uint32_t graph_of(const uint32_t* gvbase, uint32_t ngraphs, uint32_t v) {
    uint32_t lo = 0, hi = ngraphs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (gvbase[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
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

__global__ void k_rows_per_graph(const uint32_t* vid, const DevState* st, uint32_t buf, const uint32_t* gvbase,
                                 uint32_t ngraphs, uint32_t* rows_per) {
    const uint32_t R = ld_volatile_u32(&st->cnt[buf][1]);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += stride)
        atomicAdd(&rows_per[graph_of(gvbase, ngraphs, vid[i])], 1u);
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
static int g_sweep_blocks[64];

static int device_sms(int dev) {
    if (dev < 0 || dev >= 64) return 1;
    if (!g_sm_count[dev]) {
        int c = 0;
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        g_sm_count[dev] = c > 0 ? c : 1;
    }
    return g_sm_count[dev];
}

template <bool I, bool C>
static int prep_sweep() {
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<I, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(SweepSmem));
        if (e != cudaSuccess) return (int)e;
        done = true;
    }
    return 0;
}

int sweep_grid(int device) {
    if (device < 0 || device >= 64) return 1;
    if (!g_sweep_blocks[device]) {
        prep_sweep<false, true>();
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<false, true>, SWEEP_THREADS, sizeof(SweepSmem));
        if (per < 1) per = 1;
        g_sweep_blocks[device] = per * device_sms(device);
    }
    return g_sweep_blocks[device];
}

int vertex_grid(int device) { return device_sms(device) * 8; }

int launch_init(void* stream, uint32_t* mate, uint32_t* cnbr, uint8_t* dead, uint32_t n, DevState* st) {
    int dev = 0;
    cudaGetDevice(&dev);
    uint32_t blocks = (n + 255) / 256;
    const uint32_t cap = (uint32_t)device_sms(dev) * 16;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    k_init<<<blocks, 256, 0, (cudaStream_t)stream>>>(mate, cnbr, dead, n, st);
    return (int)cudaGetLastError();
}

template <bool I, bool C>
static int launch_sweep_t(void* stream, const SweepArgs& a, int grid) {
    int e = prep_sweep<I, C>();
    if (e) return e;
    k_sweep<I, C><<<grid, SWEEP_THREADS, sizeof(SweepSmem), (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}
int launch_sweep_input_cand(void* stream, const SweepArgs& a, int grid) { return launch_sweep_t<true, false>(stream, a, grid); }
int launch_sweep_input_compact(void* stream, const SweepArgs& a, int grid) { return launch_sweep_t<true, true>(stream, a, grid); }
int launch_sweep_live(void* stream, const SweepArgs& a, int grid) { return launch_sweep_t<false, true>(stream, a, grid); }

int launch_vertex_all(void* stream, const VertexArgs& a, int grid) {
    k_vertex_all<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}
int launch_vertex_live(void* stream, const VertexArgs& a, int grid) {
    k_vertex_live<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

static uint32_t grid_for(uint64_t n, uint32_t per_block) {
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t b = (n + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)device_sms(dev) * 32;
    if (b > cap) b = cap;
    return b ? (uint32_t)b : 1u;
}

int launch_build_degrees(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n,
                         uint32_t m, uint32_t* deg, uint32_t* err) {
    k_build_degrees<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(eu, ev, w, n, m, deg, err);
    return (int)cudaGetLastError();
}
int launch_build_fill(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t m,
                      const uint32_t* rowstart_all, uint32_t* cursor, uint32_t* nbr, uint32_t* eid,
                      uint32_t* ordw) {
    (void)rowstart_all;
    k_build_fill<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(eu, ev, w, m, cursor, nbr, eid, ordw);
    return (int)cudaGetLastError();
}
int launch_nonzero_flags(void* stream, const uint32_t* deg, uint32_t n, uint32_t* flags) {
    k_nonzero_flags<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(deg, n, flags);
    return (int)cudaGetLastError();
}
int launch_build_rows(void* stream, const uint32_t* deg, const uint32_t* rowidx_excl, const uint32_t* off_all,
                      uint32_t n, uint32_t nrows, uint32_t nent, uint32_t* off0, uint32_t* vid0) {
    k_build_rows<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(deg, rowidx_excl, off_all, n, nrows, nent,
                                                                      off0, vid0);
    return (int)cudaGetLastError();
}
int launch_build_tilemap(void* stream, const uint32_t* off0, uint32_t nrows, uint32_t nent, uint32_t* tilemap) {
    k_build_tilemap<<<grid_for(nrows, 256), 256, 0, (cudaStream_t)stream>>>(off0, nrows, nent, tilemap);
    return (int)cudaGetLastError();
}
int launch_to_local_batch(void* stream, const uint32_t* mate_union, const uint32_t* gvbase, uint32_t ngraphs,
                          uint32_t* const* dst, unsigned long long* matched2, uint32_t nvert) {
    if (nvert == 0 || ngraphs == 0) return 0;
    k_to_local_batch<<<grid_for(nvert, 256), 256, 0, (cudaStream_t)stream>>>(mate_union, gvbase, ngraphs, dst,
                                                                             matched2, nvert);
    return (int)cudaGetLastError();
}
int launch_rows_per_graph(void* stream, const uint32_t* vid, const DevState* st, uint32_t buf,
                          const uint32_t* gvbase, uint32_t ngraphs, uint32_t* rows_per, int grid) {
    if (ngraphs == 0) return 0;
    k_rows_per_graph<<<grid, 256, 0, (cudaStream_t)stream>>>(vid, st, buf, gvbase, ngraphs, rows_per);
    return (int)cudaGetLastError();
}
int launch_to_local(void* stream, const uint32_t* mate_global, uint32_t vbase, uint32_t n, uint32_t* out,
                    unsigned long long* matched2) {
    if (n == 0) return 0;
    k_to_local<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(mate_global, vbase, n, out, matched2);
    return (int)cudaGetLastError();
}

}  // namespace lm
