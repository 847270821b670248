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
//   k_sweep   warps take tasks (32 rows walked as one flattened sequence of
//             entries, or one chunk of a long row): an entry survives when its
//             neighbour is unmatched; survivors go to the front of the row's
//             range in the other buffer, and the heaviest surviving key of the
//             row is its candidate for the next round (step 2 of the next
//             round; the segmented maximum of Lemma "broadcast" restricted to
//             one row).  The candidate's neighbour is recovered from the key:
//             its low half is perm_seed(e), inverted to the edge index e.
//
// Round 0 first files every row (k_vertex without matching), runs a
// candidate-only sweep over the graphs' own arrays, then the match and a
// compacting sweep that builds the 64-bit keys
//     K(e) = ord(w_e) << 32 | perm_seed(e)
// from the per-entry word ord(weight) << 32 | edge id on the fly.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <mutex>

#include "../../include/lm.h"
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
// inverse of x -> x * a (mod 2^32) for odd a, by Newton's iteration
__host__ __device__ constexpr uint32_t inv_mul(uint32_t a) {
    uint32_t x = a;  // correct to 3 bits for odd a
    x *= 2u - a * x;
    x *= 2u - a * x;
    x *= 2u - a * x;
    x *= 2u - a * x;
    x *= 2u - a * x;
    return x;
}
constexpr uint32_t INV_M1 = inv_mul(0x85EBCA6Bu), INV_M2 = inv_mul(0xC2B2AE35u);
static_assert(0x85EBCA6Bu * INV_M1 == 1u && 0xC2B2AE35u * INV_M2 == 1u, "modular inverses");
__device__ __forceinline__ uint32_t fmix32_inv(uint32_t h) {
    h ^= h >> 16;                       // h ^ (h >> 16) is its own inverse on 32 bits
    h *= INV_M2;
    h ^= (h >> 13) ^ (h >> 26);         // inverse of h ^= h >> 13
    h *= INV_M1;
    h ^= h >> 16;
    return h;
}
// e = perm_seed^-1(x)
__device__ __forceinline__ uint32_t perm_seed_inv(uint32_t x, uint32_t k0, uint32_t k1) {
    return fmix32_inv(fmix32_inv(x) ^ k1) ^ k0;
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
__device__ __forceinline__ uint32_t lanemask_le() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
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
// matched bit of vertex u; the bitmap is read-only during a sweep, so it may go
// through the non-coherent (read-only) cache
// matched bit of u.  Between kernels the read-only cache path is safe; inside the
// tail kernel, which sets bits itself, COH reads through L2 (coherent with the atomics)
template <bool COH = false>
__device__ __forceinline__ bool is_dead(const VertexArrays& va, uint32_t u) {
    return ((COH ? __ldcg(&va.dead[u >> 5]) : __ldg(&va.dead[u >> 5])) >> (u & 31)) & 1u;
}
// device-scope fetch-and-add with acquire-release ordering
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void set_err(DevState* st, uint32_t bit, uint32_t info) {
    if ((atomicOr(&st->err, bit) & bit) == 0) st->err_info = info;
    atomicOr(&st->err_any, bit);  // not reset by the next job's init (asynchronous matches)
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
    uint32_t* dead = A.dead;
    uint32_t* bcnt = A.bcnt;
    unsigned long long* bkey = A.bkey;
    const uint32_t n = A.n;
    DevState* st = A.st;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (mate) mate[v] = NIL;
        bcnt[v] = 0;
        bkey[v] = 0;
    }
    // matched bits [dbase, dbase + n): whole words are stored, the partial words at
    // either end are cleared with atomicAnd (their other bits belong to other jobs)
    if (n) {
        const uint32_t b0 = A.dbase, b1 = A.dbase + n;
        const uint32_t w0 = b0 >> 5, w1 = (b1 - 1) >> 5;
        for (uint32_t w = w0 + blockIdx.x * blockDim.x + threadIdx.x; w <= w1; w += stride) {
            const uint32_t lo = max(b0, w * 32u), hi = min(b1, w * 32u + 32u);
            if (lo == w * 32u && hi == w * 32u + 32u) {
                dead[w] = 0;
            } else {
                const uint32_t width = hi - lo;
                const uint32_t mask = (width == 32u ? FULL : ((1u << width) - 1u)) << (lo & 31u);
                atomicAnd(&dead[w], ~mask);
            }
        }
    }
    if (st && blockIdx.x == 0) {
        for (int i = threadIdx.x; i < 64; i += blockDim.x) { st->ring_m[i] = 0; st->ring_n[i] = 0; }
        if (threadIdx.x < 16) (&st->lcnt[0][0])[threadIdx.x] = 0;
        if (threadIdx.x < 4) st->task[threadIdx.x] = 0;
        if (threadIdx.x == 0) {
            st->err = 0; st->err_info = 0; st->rounds = 0; st->done = 0;
            st->live_rows = 0; st->live_ent = 0; st->matched2 = 0;
            st->last_ent = ~0ull; st->tail = 0; st->tail_round = 0;
            st->round = 1;
            st->max_rounds = A.max_rounds;
            st->limit_ns = A.limit_ns ? A.limit_ns : LOOP_LIMIT_NS;
            st->t0_ns = globaltimer_ns();
        }
    }
}

// ---------------------------------------------------------------- vertex pass
#ifndef LM_VI
#define LM_VI 4
#endif
#ifndef LM_VMINB
#define LM_VMINB 4
#endif
constexpr int VT = 256;    // threads
constexpr int VI = LM_VI;  // rows per thread per block iteration

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

// exclusive scan of one counter over the block (x becomes its prefix); returns the total
__device__ __forceinline__ uint32_t block_excl_scan1(uint32_t& x, uint32_t* tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ix = warp_incl_scan(x, lane);
    if (lane == 31) tmp[warp] = ix;
    __syncthreads();
    uint32_t px = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < VT / 32; w++) {
        const uint32_t y = tmp[w];
        if (w < warp) px += y;
        tot += y;
    }
    x = px + ix - x;
    return tot;
}

// The vertex pass as CTA `cta` of `ncta` (k_vertex: the grid; the tail kernel: one CTA).
__device__ __forceinline__ void vertex_pass(const VertexArgs& a, uint32_t cta, uint32_t ncta) {
    __shared__ uint32_t s_tmp[3 * (VT / 32)];
    __shared__ uint32_t s_base[3];  // list bases of the block: R, C, B
    __shared__ unsigned long long s_red[3 * (VT / 32)];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    DevState* st = a.st;
    const VertexArrays& va = a.va;
    const uint32_t par = a.par;
    const uint32_t round = a.round_from_state ? ld_volatile_u32(&st->round) : a.round;

    uint32_t nR = 0, nC = 0, total;
    if (a.vlist || !a.in.cnt) {
        total = a.nvlist;
    } else {
        nR = ld_volatile_u32(&a.in.cnt[0]);
        nC = ld_volatile_u32(&a.in.cnt[1]);
        total = nC + nR;
    }
    // only CTAs with rows take part (CTA 0 closes an empty pass): idle CTAs leave
    // before touching the exit counter
    const uint32_t working = (uint32_t)min((uint64_t)ncta, ((uint64_t)total + VT * VI - 1) / (VT * VI));
    const uint32_t closers = working ? working : 1u;
    if (cta >= closers) return;
    unsigned long long my_rows = 0, my_ent = 0, my_match = 0;

    for (uint32_t base = cta * (VT * VI); base < total; base += ncta * (VT * VI)) {
        uint32_t vv[VI], LL[VI], cls[VI], uu[VI];
        uint32_t cR = 0, cC = 0, eR = 0;  // this thread's R rows, chunks and R entries
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
                } else {
                    // a short row: the sweep left its survivor count in the entry itself
                    const uint2 rr = a.in.R[idx - nC];
                    v = rr.x;
                    L = (rr.y & ~BATCH_START) | R_LEN_KNOWN;
                }
                if (v != NIL && v >= va.nvert) { set_err(st, ERR_BOUNDS, v); v = NIL; }
            }
            vv[i] = v;
            LL[i] = L;
        }
        // phase 2: its live length (long rows and dense ranges keep theirs in len[])
#pragma unroll
        for (int i = 0; i < VI; i++) {
            if (vv[i] == NIL) continue;
            if (LL[i] & R_LEN_KNOWN) LL[i] &= ~R_LEN_KNOWN;
            else if (a.vlist && a.deg0) va.len[par][vv[i]] = LL[i];
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
                    atomicOr(&va.dead[v >> 5], 1u << (v & 31));
                    my_match++;
                } else {
                    open_row = true;
                    if (L <= a.rmax) { cls[i] = 1; cR++; eR += L; }
                    else {
                        cls[i] = 2;
                        cC += ((L - 1) >> a.chunk_shift) + 1;
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
        block_excl_scan3(cR, cC, eR, s_tmp, tot);
        if (tid == 0) {
            s_base[0] = tot[0] ? atomicAdd(&a.out.cnt[0], tot[0]) : 0;
            s_base[1] = tot[1] ? atomicAdd(&a.out.cnt[1], tot[1]) : 0;
        }
        __syncthreads();
        // the block's R rows form one segment of R (row k of it at s_base[0] + k,
        // its entries from offset eR within the segment); a batch starts at every
        // 32nd row and at each row whose entries cross a multiple of 1 << batch_shift
        const uint32_t pR0 = s_base[0] + cR;
        uint32_t pR = pR0, pC = s_base[1] + cC, firsts = 0;
#pragma unroll
        for (int i = 0; i < VI; i++) {
            if (cls[i] == 1) {
                const uint32_t k = pR - s_base[0];
                const bool first = (k & 31u) == 0 ||
                        (a.batch_shift < 32 && (eR >> a.batch_shift) != ((eR + LL[i]) >> a.batch_shift));
                if (pR < a.out.capR) a.out.R[pR] = make_uint2(vv[i], LL[i] | (first ? BATCH_START : 0u));
                else set_err(st, ERR_BOUNDS, pR);
                firsts |= (first ? 1u : 0u) << i;
                eR += LL[i];
                pR++;
            } else if (cls[i] == 2) {
                const uint32_t nch = ((LL[i] - 1) >> a.chunk_shift) + 1;
                for (uint32_t c = 0; c < nch; c++, pC++) {
                    if (pC < a.out.capC) a.out.C[pC] = make_uint2(vv[i], c); else set_err(st, ERR_BOUNDS, pC);
                }
            }
        }
        // the batches' first rows into B, block-aggregated (the first scan's reads of
        // s_tmp are behind the barrier above)
        uint32_t nb = __popc(firsts);
        const uint32_t nb_tot = block_excl_scan1(nb, s_tmp);
        if (tid == 0) s_base[2] = nb_tot ? atomicAdd(&a.out.cnt[2], nb_tot) : 0;
        __syncthreads();
        uint32_t pB = s_base[2] + nb;
        pR = pR0;
#pragma unroll
        for (int i = 0; i < VI; i++) {
            if (cls[i] != 1) continue;
            if ((firsts >> i) & 1u) {
                if (pB < a.out.capR) a.out.B[pB] = pR; else set_err(st, ERR_BOUNDS, pB);
                pB++;
            }
            pR++;
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
        if (done == closers - 1) {
            __threadfence();
            if (a.in_set < 4) { st->lcnt[a.in_set][0] = 0; st->lcnt[a.in_set][1] = 0; st->lcnt[a.in_set][2] = 0; }
            st->task[0] = 0; st->task[1] = 0; st->task[2] = 0; st->task[3] = 0;
            if (a.match) {
                const uint32_t rows = ld_volatile_u32(&st->live_rows);
                const unsigned long long ent = *reinterpret_cast<volatile unsigned long long*>(&st->live_ent);
                if (round < 64) { st->ring_m[round] = ent / 2; st->ring_n[round] = rows; }
                if (rows == 0 && !st->done) { st->done = 1; st->rounds = round; }
                st->last_ent = ent;
                st->live_rows = 0;
                st->live_ent = 0;
                if (a.round_from_state) st->round = round + 1;
            }
            st->exit_v = 0;
            __threadfence();
        }
    }
}

__global__ void __launch_bounds__(VT, LM_VMINB) k_vertex(const VertexArgs* __restrict__ pav) {
    vertex_pass(*pav, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- sweep
// Tasks: [0, nC) chunks of long rows, then the row batches listed in B.
// Warps take tasks from a counter and never synchronise with each other.
#ifndef LM_SWEEP_MINB
#define LM_SWEEP_MINB 6   // CTAs per SM (40 registers a thread)
#endif

constexpr int ST = 256;        // threads per CTA (8 independent warps)

template <bool RENEW>
struct WarpRows {              // one warp's batch of rows
    unsigned long long rkey[32];   // heaviest surviving key per row
    uint32_t rcnt[32];             // survivors per row
    uint32_t rstart[32];           // union entry index of the row (output base)
    uint32_t rseg[32];             // graph of the row
    uint32_t ru[32];               // neighbour over the heaviest surviving key (compaction sweeps)
    uint32_t rk0[RENEW ? 32 : 1], rk1[RENEW ? 32 : 1];  // renewed order: the row's keys this round
};

// SplitMix64 (Steele, Lea, Flood 2014): the r-th output (r >= 0) for state `seed`
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint32_t r) {
    uint64_t z = seed + (uint64_t)(r + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// keys ordering the entries of graph g in the round being prepared (nr): the graph's
// own keys, or with a renewed order those of the nr-th SplitMix64 output
template <bool RENEW>
__device__ __forceinline__ void round_keys(const SweepArgs& a, uint32_t g, uint32_t nr, uint32_t& k0, uint32_t& k1) {
    const SegIn& sg = a.segs[g];
    if (RENEW) {
        const uint64_t z = splitmix64_at(sg.seed, nr);
        k0 = (uint32_t)z;
        k1 = (uint32_t)(z >> 32);
    } else {
        k0 = sg.k0;
        k1 = sg.k1;
    }
}

// neighbour of v over the edge with key K (the edge is incident to v): the key's
// low half is perm_seed(e); its inverse gives e, whose record holds both ends
__device__ __forceinline__ uint32_t recover_nbr_keys(const SegIn& sg, DevState* st, uint32_t v, uint64_t K,
                                                     uint32_t k0, uint32_t k1) {
    const uint32_t e = perm_seed_inv((uint32_t)K, k0, k1);
    if (e >= sg.m) { set_err(st, ERR_BOUNDS, e); return NIL; }
    const uint64_t rec = sg.edges[e];
    const uint32_t x = (uint32_t)rec, y = (uint32_t)(rec >> 32), vl = v - sg.vbase;
    if (x != vl && y != vl) { set_err(st, ERR_BOUNDS, e); return NIL; }
    return (x == vl ? y : x) + sg.vbase;
}
__device__ __forceinline__ uint32_t recover_nbr_seg(const SegIn& sg, DevState* st, uint32_t v, uint64_t K) {
    return recover_nbr_keys(sg, st, v, K, sg.k0, sg.k1);
}

// the key under (k0, k1) of a stored word (input, or live with a renewed order:
// ord(w) << 32 | edge id; live otherwise: the key itself)
template <bool INPUT, bool RENEW>
__device__ __forceinline__ uint64_t word_key(uint32_t k0, uint32_t k1, uint64_t w) {
    if (INPUT || RENEW) return (w & 0xFFFFFFFF00000000ull) | perm_seed((uint32_t)w, k0, k1);
    return w;
}
// what a survivor stores: its key, or with a renewed order its edge id (keys change per round)
template <bool RENEW>
__device__ __forceinline__ uint64_t stored_word(uint32_t k0, uint32_t k1, uint64_t key) {
    if (RENEW) return (key & 0xFFFFFFFF00000000ull) | perm_seed_inv((uint32_t)key, k0, k1);
    return key;
}
// the key of stored word w of row r of a warp's batch
template <bool INPUT, bool RENEW>
__device__ __forceinline__ uint64_t row_word_key(const SweepArgs& a, const WarpRows<RENEW>& W, uint32_t r, uint64_t w) {
    if (RENEW) return word_key<INPUT, true>(W.rk0[r], W.rk1[r], w);
    if (INPUT) { const SegIn& sg = a.segs[W.rseg[r]]; return word_key<true, false>(sg.k0, sg.k1, w); }
    return w;
}
// ---- pipelined form: entry words and neighbours go through shared memory by
// cp.async, PD groups of 32 entries in flight per warp (no registers held for
// them), so a warp keeps loading while it tests, votes and stores.
#ifndef LM_PIPE_D
#define LM_PIPE_D 2
#endif
constexpr int PD = LM_PIPE_D;    // groups in flight
constexpr int PS = PD + 1;       // stages: the one being read is never a copy's target
struct WarpStage {
    unsigned long long key[PS][32];
    uint32_t nbr[PS][32];
};
__device__ __forceinline__ uint32_t sh_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(sh_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(sh_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// One 32-entry group of a row batch: r = the entry's row in the batch (32: no
// entry), sl = the group lane where that row starts, uni = one row for the whole
// group; w = the stored word, u = the neighbour (compaction sweeps).
template <bool INPUT, bool COMPACT, bool RENEW, bool COH>
__device__ __forceinline__ void row_group(const SweepArgs& a, WarpRows<RENEW>& W, uint32_t r, uint32_t sl, bool uni,
                                          uint64_t w, uint32_t u, int lane, uint32_t lt) {
    const VertexArrays& va = a.va;
    uint64_t key = 0;
    if (COMPACT) {
        bool keep = r != 32;
        if (keep) {
            if (u >= va.nvert) { set_err(a.st, ERR_BOUNDS, u); keep = false; }
            else keep = !is_dead<COH>(va, u);
        }
        if (keep) key = row_word_key<INPUT, RENEW>(a, W, r, w);
    } else if (r != 32) {
        key = row_word_key<INPUT, RENEW>(a, W, r, w);
    }
    const bool surv = key != 0;
    const uint32_t ball = __ballot_sync(FULL, surv);
    if (!ball) return;
    if (uni) {
        // the whole group lies in one row: full-warp reductions
        const uint32_t hi = __reduce_max_sync(FULL, (uint32_t)(key >> 32));
        const uint32_t lo = __reduce_max_sync(FULL, ((uint32_t)(key >> 32) == hi) ? (uint32_t)key : 0u);
        const uint64_t K = ((uint64_t)hi << 32) | lo;
        if (COMPACT) {
            uint32_t base = 0;
            if (surv) base = W.rcnt[r];
            __syncwarp();
            if (surv) {
                const uint32_t pos = W.rstart[r] + base + __popc(ball & lt);
                a.out_key[pos] = RENEW ? stored_word<RENEW>(W.rk0[r], W.rk1[r], key) : key;
                a.out_nbr[pos] = u;
            }
            // keys are distinct: exactly one lane (a survivor) holds the maximum
            if (key == K) {
                W.rcnt[r] = base + __popc(ball);
                if (K > W.rkey[r]) { W.rkey[r] = K; W.ru[r] = u; }
            }
        } else if (key == K && K > W.rkey[r]) {
            W.rkey[r] = K;
        }
        __syncwarp();
        return;
    }
    // several rows, each on a run of lanes from sl: segmented shuffle scan
    uint64_t mx = key;
    uint32_t mu = u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t o = __shfl_up_sync(FULL, mx, d);
        const uint32_t ou = COMPACT ? __shfl_up_sync(FULL, mu, d) : 0u;
        if ((uint32_t)lane >= sl + d && o > mx) { mx = o; mu = ou; }
    }
    const uint32_t rn = __shfl_down_sync(FULL, r, 1);
    const bool last = r != 32 && (lane == 31 || rn != r);
    if (COMPACT) {
        const uint32_t run = FULL << sl;
        const uint32_t base = r != 32 ? W.rcnt[r] : 0u;
        __syncwarp();
        if (last) W.rcnt[r] = base + __popc(ball & run & lanemask_le());
        if (surv) {
            const uint32_t pos = W.rstart[r] + base + __popc(ball & run & lt);
            a.out_key[pos] = RENEW ? stored_word<RENEW>(W.rk0[r], W.rk1[r], key) : key;
            a.out_nbr[pos] = u;
        }
    }
    if (last && mx > W.rkey[r]) {
        W.rkey[r] = mx;
        if (COMPACT) W.ru[r] = mu;
    }
    __syncwarp();
}

template <bool INPUT, bool COMPACT, bool RENEW, bool COH>
__device__ void do_rows_p(const SweepArgs& a, WarpRows<RENEW>& W, WarpStage& S, uint32_t b, uint32_t nR, uint32_t nr,
                          int lane) {
    const VertexArrays& va = a.va;
    const uint32_t idx = (COH ? __ldcg(a.in.B + b) : __ldg(a.in.B + b)) + lane;
    uint2 rv = make_uint2(NIL, 0);
    if (idx < nR) rv = a.in.R[idx];
    // the batch's rows: lane 0's (a batch start) up to the next batch start
    const uint32_t starts = __ballot_sync(FULL, (rv.y & BATCH_START) != 0);
    if (lane == 0 && idx < nR && !(starts & 1u)) set_err(a.st, ERR_BOUNDS, idx);
    uint32_t v = NIL, L = 0, s0 = 0, g = 0;
    if (idx < nR && (starts & 1u) && (starts & lanemask_le() & ~1u) == 0) {
        v = rv.x;
        L = rv.y & ~BATCH_START;
        if (v >= va.nvert || L > a.rmax) { set_err(a.st, ERR_BOUNDS, v); v = NIL; L = 0; }
        else {
            s0 = va.start[v];
            g = va.gid ? va.gid[v] : 0u;
            if ((uint64_t)s0 + L > a.ecap || g >= a.nsegs) { set_err(a.st, ERR_BOUNDS, v); v = NIL; L = 0; s0 = 0; g = 0; }
        }
    }
    W.rkey[lane] = 0;
    W.rcnt[lane] = 0;
    W.rstart[lane] = s0;
    W.rseg[lane] = g;
    uint32_t rk0 = 0, rk1 = 0;
    if (RENEW) {
        round_keys<true>(a, g, nr, rk0, rk1);
        W.rk0[lane] = rk0;
        W.rk1[lane] = rk1;
    }
    const uint32_t ro = INPUT ? s0 - a.segs[g].ebase : s0;  // source index of the row's entry 0
    const uint32_t incl = warp_incl_scan(L, lane);
    const uint32_t ex = incl - L;                             // the row's first flattened entry
    const uint32_t F = __shfl_sync(FULL, incl, 31);
    __syncwarp();
    const uint32_t lt = lanemask_lt();
    const uint32_t ng = (F + 31) >> 5;
    // group k holds flattened entries 32k .. 32k + 31.  The row of entry g0 + j is
    // the number of rows starting at or before g0 (a ballot) plus the rows starting
    // inside the group at positions 1..j (bits of an OR-reduction), minus one.
    auto map = [&](uint32_t g0, uint32_t& r, uint32_t& q, uint32_t& sl, bool& uni) {
        const uint32_t below = __ballot_sync(FULL, ex <= g0);
        const uint32_t st = __reduce_or_sync(FULL, (ex > g0 && ex - g0 < 32u) ? 1u << (ex - g0) : 0u);
        const uint32_t lim = F - g0;
        uni = (st & (lim >= 32u ? FULL : (1u << lim) - 1u)) == 0;
        const uint32_t rr = __popc(below) - 1 + __popc(st & (FULL >> (31 - lane)));
        const uint32_t exr = __shfl_sync(FULL, ex, rr & 31u), ror = __shfl_sync(FULL, ro, rr & 31u);
        r = 32;
        q = 0;
        if (g0 + lane < F) {
            r = rr;
            q = ror + (g0 + lane - exr);
        }
        sl = exr > g0 ? exr - g0 : 0u;
    };
    auto issue = [&](uint32_t k) {
        if (k < ng) {
            uint32_t r, q, sl;
            bool uni;
            map(k * 32, r, q, sl, uni);
            if (r != 32) {
                const uint32_t stg = k % PS;
                if (INPUT) {
                    const SegIn& sg = a.segs[W.rseg[r]];
                    cp_async8(&S.key[stg][lane], sg.pk + q);
                    if (COMPACT) cp_async4(&S.nbr[stg][lane], sg.nbr + q);
                } else {
                    cp_async8(&S.key[stg][lane], a.in_key + q);
                    if (COMPACT) cp_async4(&S.nbr[stg][lane], a.in_nbr + q);
                }
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < PD; d++) issue(d);
    for (uint32_t k = 0; k < ng; k++) {
        cp_async_wait<PD - 1>();
        uint32_t r, q, sl;
        bool uni;
        map(k * 32, r, q, sl, uni);
        uint64_t w = 0;
        uint32_t u = NIL;
        if (r != 32) {
            const uint32_t stg = k % PS;
            w = S.key[stg][lane];
            if (COMPACT) u = S.nbr[stg][lane] + (INPUT ? a.segs[W.rseg[r]].vbase : 0u);
        }
        issue(k + PD);
        row_group<INPUT, COMPACT, RENEW, COH>(a, W, r, sl, uni, w, u, lane, lt);
    }
    cp_async_wait<0>();
    __syncwarp();
    if (v != NIL) {
        // the survivor count goes into the row's own task-list entry (read there by
        // the next vertex pass; the batch-start bit stays for the other warps' scans)
        if (COMPACT) a.in.R[idx].y = W.rcnt[lane] | (rv.y & BATCH_START);
        const uint64_t K = W.rkey[lane];
        // compaction sweeps carried the neighbour along; the candidate-only sweep
        // recovers it from the key's edge id
        if (K) va.cnbr[v] = COMPACT ? W.ru[lane]
                                    : RENEW ? recover_nbr_keys(a.segs[g], a.st, v, K, rk0, rk1)
                                            : recover_nbr_seg(a.segs[g], a.st, v, K);
    }
    __syncwarp();
}

// One chunk of a long row, pipelined like the row batches.
template <bool INPUT, bool COMPACT, bool RENEW, bool COH>
__device__ void do_chunk_p(const SweepArgs& a, WarpStage& S, uint32_t t, uint32_t nr, int lane) {
    const VertexArrays& va = a.va;
    const uint2 c = a.in.C[t];
    const uint32_t v = c.x;
    if (v >= va.nvert) { if (lane == 0) set_err(a.st, ERR_BOUNDS, v); return; }
    const uint32_t L = va.len[a.par][v];
    const uint32_t jb = c.y << a.chunk_shift, je = min(L, jb + (1u << a.chunk_shift));
    const uint32_t s0 = va.start[v];
    const uint32_t g = va.gid ? va.gid[v] : 0u;
    if (jb >= L || (uint64_t)s0 + L > a.ecap || g >= a.nsegs) { if (lane == 0) set_err(a.st, ERR_BOUNDS, t); return; }
    const SegIn& sg = a.segs[g];
    const uint32_t off = INPUT ? s0 - sg.ebase : s0;
    const uint32_t vb = INPUT ? sg.vbase : 0u;
    uint32_t ck0 = 0, ck1 = 0;
    if (RENEW) round_keys<true>(a, g, nr, ck0, ck1);
    else if (INPUT) { ck0 = sg.k0; ck1 = sg.k1; }
    uint32_t* len_next = va.len[a.par ^ 1u];
    uint64_t bk = 0;
    const uint32_t lt = lanemask_lt();
    const uint32_t ng = (je - jb + 31) >> 5;
    auto issue = [&](uint32_t k) {
        const uint32_t jj = jb + k * 32 + lane;
        if (k < ng && jj < je) {
            const uint32_t stg = k % PS;
            if (INPUT) {
                cp_async8(&S.key[stg][lane], sg.pk + off + jj);
                if (COMPACT) cp_async4(&S.nbr[stg][lane], sg.nbr + off + jj);
            } else {
                cp_async8(&S.key[stg][lane], a.in_key + off + jj);
                if (COMPACT) cp_async4(&S.nbr[stg][lane], a.in_nbr + off + jj);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int d = 0; d < PD; d++) issue(d);
    for (uint32_t k = 0; k < ng; k++) {
        cp_async_wait<PD - 1>();
        const uint32_t jj = jb + k * 32 + lane, stg = k % PS;
        uint64_t key = 0;
        uint32_t u = NIL;
        if (jj < je) {
            key = S.key[stg][lane];
            if (COMPACT) u = S.nbr[stg][lane] + vb;
        }
        issue(k + PD);
        if (COMPACT) {
            bool keep = jj < je;
            if (keep) {
                if (u >= va.nvert) { set_err(a.st, ERR_BOUNDS, u); keep = false; }
                else keep = !is_dead<COH>(va, u);
            }
            key = keep ? word_key<INPUT, RENEW>(ck0, ck1, key) : 0ull;
        } else if (jj < je) {
            key = word_key<INPUT, RENEW>(ck0, ck1, key);
        }
        const uint32_t ball = __ballot_sync(FULL, key != 0);
        if (key > bk) bk = key;
        if (COMPACT && ball) {
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&len_next[v], (uint32_t)__popc(ball));
            base = __shfl_sync(FULL, base, 0);
            // the survivors of all chunks fit the row's L slots; a cursor that was not
            // reset to 0 before this sweep would carry the writes past the row
            if (base + (uint32_t)__popc(ball) > L) {
                if (lane == 0) set_err(a.st, ERR_BOUNDS, v);
            } else if (key != 0) {
                const uint32_t pos = s0 + base + __popc(ball & lt);
                a.out_key[pos] = stored_word<RENEW>(ck0, ck1, key);
                a.out_nbr[pos] = u;
            }
        }
    }
    cp_async_wait<0>();
    // chunk maximum into the row's slot; the last chunk of the row to finish
    // reads the row maximum and recovers its neighbour
    const uint32_t hi = __reduce_max_sync(FULL, (uint32_t)(bk >> 32));
    const uint32_t lo = __reduce_max_sync(FULL, ((uint32_t)(bk >> 32) == hi) ? (uint32_t)bk : 0u);
    if (lane == 0) {
        const uint64_t K = ((uint64_t)hi << 32) | lo;
        if (K) atomicMax(&va.bkey[v], (unsigned long long)K);
        const uint32_t nch = ((L - 1) >> a.chunk_shift) + 1;
        // release: this chunk's maximum is visible before its count; acquire: the last
        // chunk sees every other chunk's maximum
        const uint32_t old = atom_add_acq_rel(&va.bcnt[v], 1u);
        if (old == nch - 1) {
            const uint64_t R = *reinterpret_cast<volatile unsigned long long*>(&va.bkey[v]);
            va.bkey[v] = 0;
            va.bcnt[v] = 0;
            if (R) va.cnbr[v] = RENEW ? recover_nbr_keys(sg, a.st, v, R, ck0, ck1) : recover_nbr_seg(sg, a.st, v, R);
        }
    }
}


// The sweep as CTA `cta` of `ncta` (k_sweep: the grid; the tail kernel: one CTA);
// W and S are the calling warp's shared row state and copy stages.
template <bool INPUT, bool COMPACT, bool RENEW, bool COH>
__device__ __forceinline__ void sweep_pass(const SweepArgs& a, WarpRows<RENEW>& W, WarpStage& S, uint32_t cta,
                                           uint32_t ncta) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (cta * ST + threadIdx.x) >> 5;
    const uint32_t nw = (ncta * ST) >> 5;
    const uint32_t nR = ld_volatile_u32(&a.in.cnt[0]);
    const uint32_t nC = ld_volatile_u32(&a.in.cnt[1]);
    const uint32_t nB = ld_volatile_u32(&a.in.cnt[2]);
    if (nR > a.in.capR || nC > a.in.capC || nB > nR) {
        if (cta == 0 && threadIdx.x == 0) set_err(a.st, ERR_BOUNDS, nC);
        return;
    }
    const uint32_t total = nC + nB;
    // the round whose candidates this sweep prepares (its vertex pass advanced the round)
    const uint32_t nr = RENEW ? ld_volatile_u32(&a.st->round) : 0u;
    // a warp's first task is its own index (idle warps leave without an atomic), later
    // ones come from the counter; the next index is fetched while the current task runs
    uint32_t t = gw;
    if (t >= total) return;
    uint32_t t_next = 0;
    for (;; t = __shfl_sync(FULL, t_next, 0)) {
        if (t >= total) break;
        if (lane == 0) t_next = nw + atomicAdd(a.task_ctr, 1u);
        if (t < nC) do_chunk_p<INPUT, COMPACT, RENEW, COH>(a, S, t, nr, lane);
        else do_rows_p<INPUT, COMPACT, RENEW, COH>(a, W, S, t - nC, nR, nr, lane);
    }
}

template <bool INPUT, bool COMPACT, bool RENEW>
__global__ void __launch_bounds__(ST, LM_SWEEP_MINB) k_sweep(const SweepArgs* __restrict__ pav) {
    __shared__ WarpRows<RENEW> s_rows[ST / 32];
    __shared__ WarpStage s_stage[ST / 32];
    // the arguments in shared memory: the many re-reads of their pointers and sizes
    // are shared-memory loads instead of global-memory ones
    __shared__ __align__(16) unsigned char s_args_raw[sizeof(SweepArgs)];
    static_assert(sizeof(SweepArgs) % 4 == 0, "word copy");
    for (uint32_t i = threadIdx.x; i < sizeof(SweepArgs) / 4; i += ST)
        reinterpret_cast<uint32_t*>(s_args_raw)[i] = reinterpret_cast<const uint32_t*>(pav)[i];
    __syncthreads();
    sweep_pass<INPUT, COMPACT, RENEW, false>(*reinterpret_cast<const SweepArgs*>(s_args_raw), s_rows[threadIdx.x >> 5],
                                      s_stage[threadIdx.x >> 5], blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- round-0 candidates in TMA-fed tiles
// Round 0's candidate pass reads every graph's own adjacency array once, front
// to back, in tiles of TILE0 entries; a CTA owns tiles blockIdx.x, +gridDim.x,
// ...  One producer thread copies a tile's entry words and neighbours, the
// vertices of the rows it touches and its slice of the graph's row-start
// bitmap into a shared-memory stage with bulk asynchronous copies completed on
// the stage's "full" mbarrier; tile descriptors (precomputed per graph) are
// loaded R0AHEAD tiles early and the copies run up to R0S stages ahead of the
// consumers.  Each consumer lane takes 4 consecutive entries of the tile and
// derives their rows from the bitmap.  A row's candidate is its entry of
// largest key K = ord(w) << 32 | perm_seed(e); the maximum is taken on ord(w)
// alone (32-bit, no hashing), per lane, then per row across the lanes of a
// warp by a segmented scan, then per row across warps with one shared-memory
// atomic where a row ends; the entries that reach their row's maximum ord
// claim the row, and only a row claimed twice (equal weights) compares
// perm_seed of its tied entries.  Only the first and the last row of a tile
// can be cut by a tile boundary: their maxima meet in bkey[] and k_round0_cut
// resolves them after the pass.  A stage goes back to the producer through its
// "empty" mbarrier; every wait is bounded.

#ifndef LM_R0S
#define LM_R0S 2
#endif
#ifndef LM_R0C
#define LM_R0C 256
#endif
#ifndef LM_R0MINB
#define LM_R0MINB 5   // CTAs per SM (40 registers a thread, 32 bytes spilled; about 45 KB of shared memory a CTA)
#endif
constexpr int R0S = LM_R0S;                         // pipeline stages
constexpr int R0C = LM_R0C;                         // consumer threads
constexpr int R0T = R0C + 32;                       // and one producer warp (one thread of it works)
constexpr int R0RPT = ((int)TILE0 + 1 + R0C - 1) / R0C;  // rows per consumer thread when finishing
constexpr int R0W = (int)TILE0 / 32;                // bitmap words of a tile
constexpr int R0AHEAD = 4;                          // tile descriptors in flight ahead of the copies
static_assert(TILE0 == 1024 && R0C == 256, "each consumer lane takes 4 entries of a 1024-entry tile");
static_assert(R0W == 32, "one bitmap word per lane");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }"
                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
constexpr unsigned long long R0_WAIT_NS = 1000000000ull;
// wait for the phase of the given parity to complete; false after R0_WAIT_NS
__device__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > R0_WAIT_NS) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// barrier of the consumer warps only (the producer warp never joins it)
__device__ __forceinline__ void cbar() {
    asm volatile("bar.sync 1, %0;" :: "n"(R0C) : "memory");
}
__device__ __forceinline__ bool cbar_or(bool p) {
    uint32_t r;
    asm volatile("{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.or.pred q, 1, %2, p; selp.u32 %0, 1, 0, q; }"
                 : "=r"(r) : "r"((uint32_t)p), "n"(R0C) : "memory");
    return r != 0;
}
__device__ __forceinline__ uint32_t round16(uint32_t b) { return (b + 15u) & ~15u; }

struct alignas(16) R0Stage {
    unsigned long long pk[TILE0];     // entry words (first member: 16-byte aligned)
    uint32_t nbr[TILE0];              // neighbours
    uint32_t rvid[TILE0 + 8];         // row vertices from row (r_lo & ~3)
    uint32_t bits[R0W + 4];           // row-start bits of the tile, then of the next tile's first entries
    // written by the producer before the copies are issued
    uint32_t valid, seg, j0, nent, shift;
};
constexpr uint32_t R0_EMPTY = 0xFFFFFFFFu;  // rwin: no claim yet
constexpr uint32_t R0_TIED = 0xFFFFFFFEu;   // rwin: claimed twice, perm_seed decides
struct R0Smem {
    R0Stage stage[R0S];
    uint32_t rord[TILE0 + 1];    // per row of the current tile: largest ord(w) (0 between tiles)
    uint32_t rwin[TILE0 + 1];    // per row: tile position of its heaviest entry, R0_EMPTY or R0_TIED
    uint32_t rperm[TILE0 + 1];   // per tied row: largest perm_seed among its entries of ord rord (0 between tiles)
    unsigned long long full[R0S], empty[R0S];
};

__device__ __forceinline__ uint32_t seg_of_tile(const Round0Args& a, uint32_t t) {
    uint32_t lo = 0, hi = a.nsegs - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (a.segs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// where tile t lies: its graph and its descriptor (loaded, not yet used)
struct R0Desc {
    const SegIn* g;
    uint32_t t, seg, lt;
    uint4 d;                  // first row, rows touched, first row's offset
};
__device__ __forceinline__ R0Desc r0_desc(const Round0Args& a, uint32_t t) {
    R0Desc d;
    d.t = t;
    d.g = nullptr;
    d.seg = d.lt = 0;
    d.d = make_uint4(0, 0, 0, 0);
    if (t < a.ntiles) {
        d.seg = seg_of_tile(a, t);
        d.g = &a.segs[d.seg];
        d.lt = t - d.g->tile_begin;
        if (d.lt < d.g->ntiles) d.d = d.g->tdesc[d.lt];
    }
    return d;
}

__device__ void r0_producer(R0Smem& s, const Round0Args& a) {
    DevState* st = a.st;
    const uint32_t step = gridDim.x;
    R0Desc q0 = r0_desc(a, blockIdx.x), q1 = r0_desc(a, blockIdx.x + step);
    R0Desc q2 = r0_desc(a, blockIdx.x + 2 * step), q3 = r0_desc(a, blockIdx.x + 3 * step);
    static_assert(R0AHEAD == 4, "shift chain of four descriptors");
    for (uint32_t j = 0;; j++) {
        const int k = (int)(j % R0S);
        const uint32_t use = j / R0S;
        R0Stage& S = s.stage[k];
        const R0Desc d = q0;
        q0 = q1;
        q1 = q2;
        q2 = q3;
        q3 = r0_desc(a, blockIdx.x + (j + R0AHEAD) * step);
        bool valid = d.g != nullptr;
        uint32_t j0 = 0, nent = 0;
        if (valid) {
            const SegIn* g = d.g;
            j0 = d.lt * TILE0;
            valid = d.lt < g->ntiles && d.d.y >= 1 && d.d.y <= TILE0 + 1 && d.d.x + d.d.y <= g->nrows;
            if (valid) nent = min(TILE0, g->nent - j0);
            else set_err(st, ERR_BOUNDS, d.t);
        }
        // the stage must be free: its consumers released it after their last use
        if (use > 0 && !mbar_wait(&s.empty[k], (use - 1) & 1u)) {
            set_err(st, ERR_TIMEOUT, 0x10000000u | j);
            return;
        }
        if (!valid) {
            S.valid = 0;
            mbar_arrive(&s.full[k]);
            return;
        }
        const SegIn* g = d.g;
        const uint32_t r_lo = d.d.x, nload = d.d.y;
        const uint32_t a0 = r_lo & ~3u, shift = r_lo - a0;
        S.valid = 1;
        S.seg = d.seg;
        S.j0 = j0;
        S.nent = nent;
        S.shift = shift;
        const uint32_t b_pk = round16(nent * 8u);
        const uint32_t b_nbr = round16(nent * 4u);
        const uint32_t b_vid = round16((shift + nload) * 4u);
        const uint32_t b_bits = (uint32_t)(R0W + 4) * 4u;
        // order the consumers' earlier reads of this stage before the copies' writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&s.full[k], b_pk + b_nbr + b_vid + b_bits);
        bulk_g2s(S.pk, g->pk + j0, b_pk, &s.full[k]);
        bulk_g2s(S.nbr, g->nbr + j0, b_nbr, &s.full[k]);
        bulk_g2s(S.rvid, g->rvid + a0, b_vid, &s.full[k]);
        bulk_g2s(S.bits, g->rbits + j0 / 32, b_bits, &s.full[k]);
    }
}

// lane-local maxima of ord over a lane's 4 entries, one slot per row segment of
// the lane: segment t holds the entries after the t-th row start inside the lane
struct R0Lane {
    uint32_t bo[4];    // largest ord of segment t (0: none)
    uint32_t bj;       // 2 bits per segment: lane position of that entry
    uint32_t tie;      // bit t: two entries of segment t share the largest ord
};
__device__ __forceinline__ void r0_lane_max(const uint32_t o[4], uint32_t hb, R0Lane& L) {
    L.bo[0] = L.bo[1] = L.bo[2] = L.bo[3] = 0;
    L.bj = 0;
    L.tie = 0;
    if ((hb & 0xEu) == 0) {
        // one segment (the common case: no row starts inside the lane)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (o[j] > L.bo[0]) { L.bo[0] = o[j]; L.bj = (uint32_t)j; L.tie = 0; }
            else if (o[j] != 0 && o[j] == L.bo[0]) L.tie = 1;
        }
        return;
    }
    uint32_t t = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        if (j > 0) t += (hb >> j) & 1u;
#pragma unroll
        for (int q = 0; q <= j; q++) {
            if (t == (uint32_t)q) {
                if (o[j] > L.bo[q]) {
                    L.bo[q] = o[j];
                    L.bj = (L.bj & ~(3u << (2 * q))) | ((uint32_t)j << (2 * q));
                    L.tie &= ~(1u << q);
                } else if (o[j] != 0 && o[j] == L.bo[q]) {
                    L.tie |= 1u << q;
                }
            }
        }
    }
}

__device__ void r0_consumer(R0Smem& s, const Round0Args& a, int tid) {
    const int lane = tid & 31, warp = tid >> 5;
    const VertexArrays& va = a.va;
    DevState* st = a.st;
    const uint32_t base = (uint32_t)warp * 128u + (uint32_t)lane * 4u;  // the lane's first entry in a tile
    for (uint32_t i = 0;; i++) {
        const int k = (int)(i % R0S);
        const uint32_t use = i / R0S;
        const bool ok = mbar_wait(&s.full[k], use & 1u);
        if (cbar_or(!ok)) {
            if (tid == 0) set_err(st, ERR_TIMEOUT, 0x30000000u | i);
            return;
        }
        R0Stage& S = s.stage[k];
        if (!S.valid) return;
        const uint32_t j0 = S.j0, nent = S.nent, shift = S.shift;
        const SegIn& g = a.segs[S.seg];
        const uint32_t vbase = g.vbase;

        // rows of the tile: the row of entry e is the number of row starts at
        // positions 1 .. e (entry 0 is in row 0, whether or not a row starts there)
        const uint32_t b0 = S.bits[0] & 1u;
        const uint32_t wx = __popc(S.bits[lane]);
        const uint32_t nrt = __reduce_add_sync(FULL, wx) - b0 + 1u;  // rows with entries in the tile
        const uint32_t wb = __reduce_add_sync(FULL, lane < warp * 4 ? wx : 0u) - (warp > 0 ? b0 : 0u);
        uint32_t hb = (S.bits[base >> 5] >> (base & 31u)) & 0xFu;     // row starts among the lane's entries
        if (base == 0) hb &= ~1u;
        const bool cutL = (j0 + nent < g.nent) && !(S.bits[R0W] & 1u);
        const bool cut0 = !b0 || (nrt == 1 && cutL);

        // the entries' ord(w): the high words of their stored words
        uint32_t o[4];
        {
            const uint4 qa = *reinterpret_cast<const uint4*>(&S.pk[base]);
            const uint4 qb = *reinterpret_cast<const uint4*>(&S.pk[base + 2]);
            o[0] = qa.y; o[1] = qa.w; o[2] = qb.y; o[3] = qb.w;
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (base + j >= nent) o[j] = 0;
        }
        R0Lane L;
        r0_lane_max(o, hb, L);
        const uint32_t nseg = 1u + __popc(hb & 0xEu);
        // phase 1: the largest ord of every row into rord
        const bool mixed = __any_sync(FULL, (hb & (lane == 0 ? 0xEu : 0xFu)) != 0);
        uint32_t R;  // row of the lane's segment 0
        if (!mixed) {
            // the warp's 128 entries lie in one row
            R = wb + __shfl_sync(FULL, hb & 1u, 0);
            const uint32_t hi = __reduce_max_sync(FULL, L.bo[0]);
            if (lane == 0 && hi) atomicMax(&s.rord[R], hi);
        } else {
            const uint32_t c = __popc(hb);
            R = wb + warp_incl_scan(c, lane) - c + (hb & 1u);
            // segmented inclusive maximum over the lanes of the lane's last segment
            uint32_t v = nseg == 1 ? L.bo[0] : nseg == 2 ? L.bo[1] : nseg == 3 ? L.bo[2] : L.bo[3];
            uint32_t f = hb != 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t ov = __shfl_up_sync(FULL, v, d), of = __shfl_up_sync(FULL, f, d);
                if (lane >= d && !f) { v = max(v, ov); f = of; }
            }
            const uint32_t vprev = __shfl_up_sync(FULL, v, 1);
            const uint32_t nhead = __shfl_down_sync(FULL, hb & 1u, 1);
            if (nseg > 1) {
                // the lane's first segment ends a row (continued from the lanes before
                // unless it starts at the lane's first entry); middle ones are whole rows
                const uint32_t first = max(L.bo[0], (lane > 0 && !(hb & 1u)) ? vprev : 0u);
                if (first) atomicMax(&s.rord[R], first);
#pragma unroll
                for (uint32_t t = 1; t < 3; t++)
                    if (t + 1 < nseg && L.bo[t]) atomicMax(&s.rord[R + t], L.bo[t]);
            }
            // the row of the last segment ends here when the next lane starts a row
            if ((lane == 31 || nhead) && v) atomicMax(&s.rord[R + nseg - 1], v);
        }
        cbar();
        // phase 2: the entries at their row's largest ord claim the row; a second
        // claim (or a tie inside a lane) marks the row tied
        bool tied = false;
#pragma unroll
        for (uint32_t t = 0; t < 4; t++) {
            if (t < nseg && L.bo[t] && L.bo[t] == s.rord[R + t]) {
                const uint32_t p = base + ((L.bj >> (2 * t)) & 3u);
                const uint32_t old = atomicCAS(&s.rwin[R + t], R0_EMPTY, p);
                if (old != R0_EMPTY || ((L.tie >> t) & 1u)) {
                    atomicExch(&s.rwin[R + t], R0_TIED);
                    tied = true;
                }
            }
        }
        if (cbar_or(tied)) {
            // phase 3 (equal weights only): perm_seed decides among the tied entries
            const uint32_t k0 = g.k0, k1 = g.k1;
            uint32_t mine = 0;   // bit j: entry j of the lane is tied at its row's maximum
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t t = __popc(hb & 0xEu & ((2u << j) - 1u));
                if (o[j] && o[j] == s.rord[R + t] && s.rwin[R + t] == R0_TIED) {
                    mine |= 1u << j;
                    atomicMax(&s.rperm[R + t], perm_seed((uint32_t)S.pk[base + j], k0, k1));
                }
            }
            cbar();
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t t = __popc(hb & 0xEu & ((2u << j) - 1u));
                if (((mine >> j) & 1u) && perm_seed((uint32_t)S.pk[base + j], k0, k1) == s.rperm[R + t])
                    s.rwin[R + t] = base + (uint32_t)j;
            }
            cbar();
        }

        // phase 4: rows -- the winner names the candidate; cut rows leave their key in bkey
#pragma unroll
        for (int q = 0; q < R0RPT; q++) {
            const uint32_t r = (uint32_t)(tid + q * R0C);
            if (r < nrt) {
                const uint32_t v = S.rvid[shift + r] + vbase;
                const uint32_t ow = s.rord[r], p = s.rwin[r];
                s.rord[r] = 0;
                s.rwin[r] = R0_EMPTY;
                s.rperm[r] = 0;
                if (v >= va.nvert || p >= nent) {
                    set_err(st, ERR_BOUNDS, v);
                    continue;
                }
                const bool cut = (r == 0 && cut0) || (r == nrt - 1 && cutL);
                if (!cut) va.cnbr[v] = S.nbr[p] + vbase;
                else atomicMax(&va.bkey[v], ((unsigned long long)ow << 32) | perm_seed((uint32_t)S.pk[p], g.k0, g.k1));
            }
        }
        cbar();
        if (tid == 0) mbar_arrive(&s.empty[k]);
    }
}

__global__ void __launch_bounds__(R0T, LM_R0MINB) k_round0(const Round0Args* __restrict__ pa) {
    extern __shared__ __align__(128) unsigned char r0_raw[];
    R0Smem& s = *reinterpret_cast<R0Smem*>(r0_raw);
    const Round0Args& a = *pa;
    const int tid = threadIdx.x;
    for (uint32_t r = tid; r <= TILE0; r += R0T) {
        s.rord[r] = 0;
        s.rwin[r] = R0_EMPTY;
        s.rperm[r] = 0;
    }
    if (tid == 0) {
        for (int k = 0; k < R0S; k++) {
            mbar_init(&s.full[k], 1);
            mbar_init(&s.empty[k], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (a.ntiles == 0 || a.nsegs == 0) return;
    if (tid == R0C) r0_producer(s, a);
    else if (tid < R0C) r0_consumer(s, a, tid);
}

// Candidates of rows that tile boundaries cut: each such row is visited once,
// at the first boundary inside it, and recovers its neighbour from the maximum
// its pieces left in bkey[] (which goes back to zero).
__global__ void k_round0_cut(const Round0Args* __restrict__ pa) {
    const Round0Args& a = *pa;
    const VertexArrays& va = a.va;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < a.ntiles; t += stride) {
        const SegIn& g = a.segs[seg_of_tile(a, t)];
        const uint32_t lt = t - g.tile_begin;
        if (lt == 0 || lt >= g.ntiles) continue;
        const uint32_t r = g.tmap[lt];
        if (r >= g.nrows) { set_err(a.st, ERR_BOUNDS, t); continue; }
        const uint32_t o0 = g.roff[r];
        if (o0 >= lt * TILE0 || o0 < (lt - 1) * TILE0) continue;
        const uint32_t v = g.rvid[r] + g.vbase;
        if (v >= va.nvert) { set_err(a.st, ERR_BOUNDS, v); continue; }
        const unsigned long long K = va.bkey[v];
        if (K) {
            va.bkey[v] = 0;
            va.cnbr[v] = recover_nbr_seg(g, a.st, v, K);
        }
    }
}

// ---------------------------------------------------------------- edge-centric path
// The Combining CRCW formulation of Sec. 2 (LM_F_EDGE_CENTRIC): per round,
// (offer) every live edge raises best[] of both ends to its key with an atomic
// maximum, lanes of a warp on the same vertex combining first; (match) an edge
// that is the best offer at both ends joins M; (compact) edges with no matched
// end go to the next round's list; (close) one thread records the round.

constexpr int EC_T = 256;

__device__ __forceinline__ uint32_t ec_round(const EdgeArgs& a) { return ld_volatile_u32(&a.st->round) - 1u; }

// warp-combined atomic maximum: lanes with the same vertex reduce first
__device__ __forceinline__ void warp_max_at(unsigned long long* best, uint32_t x, unsigned long long K, bool act) {
    const uint32_t ball = __ballot_sync(FULL, act);
    const uint32_t peers = __match_any_sync(FULL, act ? x : NIL) & ball;
    if (!act) return;
    const uint32_t hi = __reduce_max_sync(peers, (uint32_t)(K >> 32));
    const uint32_t lo = __reduce_max_sync(peers, ((uint32_t)(K >> 32) == hi) ? (uint32_t)K : 0u);
    if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&best[x], ((unsigned long long)hi << 32) | lo);
}

// sum of x over the block, added to *dst by one thread (every thread calls it):
// one atomic per block instead of one per warp on a single hot counter
template <class T>
__device__ __forceinline__ void block_add(T* dst, T x, T* s_part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if (lane == 0) s_part[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_part[w];
        if (t) atomicAdd(dst, t);
    }
}

__global__ void __launch_bounds__(EC_T) k_ec_offer(const EdgeArgs* __restrict__ pa) {
    const EdgeArgs& a = *pa;
    const uint32_t r = ec_round(a);
    const uint32_t cnt = r == 0 ? a.m : ld_volatile_u32(&a.st->lcnt[0][r & 1u]);
    const uint32_t* L = a.live[r & 1u];
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->lcnt[0][(r + 1) & 1u] = 0;
    const uint32_t stride = gridDim.x * blockDim.x, cr = (cnt + 31) & ~31u;
    uint32_t fresh = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cr; i += stride) {
        bool act = i < cnt;
        uint32_t u = 0, v = 0;
        unsigned long long K = 0;
        if (act) {
            const uint32_t e = r == 0 ? i : L[i];
            if (e >= a.m) set_err(a.st, ERR_BOUNDS, e);
            act = e < a.m;  // (the whole warp stays in the loop for the collectives below)
        }
        if (act) {
            const uint32_t e = r == 0 ? i : L[i];
            const uint64_t rec = a.edges[e];
            u = (uint32_t)rec;
            v = (uint32_t)(rec >> 32);
            K = ((unsigned long long)a.eword[e] << 32) | perm_seed(e, a.k0, a.k1);
        }
        warp_max_at(a.best, u, K, act);
        warp_max_at(a.best, v, K, act);
        if (act) {  // live vertices of the round: the first offer stamps them
            fresh += atomicExch(&a.stamp[u], r + 1u) != r + 1u;
            fresh += atomicExch(&a.stamp[v], r + 1u) != r + 1u;
        }
    }
    __shared__ uint32_t s_part[EC_T / 32];
    block_add(&a.st->live_rows, fresh, s_part);
}

__global__ void __launch_bounds__(EC_T) k_ec_match(const EdgeArgs* __restrict__ pa) {
    const EdgeArgs& a = *pa;
    const uint32_t r = ec_round(a);
    const uint32_t cnt = r == 0 ? a.m : ld_volatile_u32(&a.st->lcnt[0][r & 1u]);
    const uint32_t* L = a.live[r & 1u];
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned long long matched = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
        const uint32_t e = r == 0 ? i : L[i];
        if (e >= a.m) continue;
        const uint64_t rec = a.edges[e];
        const uint32_t u = (uint32_t)rec, v = (uint32_t)(rec >> 32);
        const unsigned long long K = ((unsigned long long)a.eword[e] << 32) | perm_seed(e, a.k0, a.k1);
        if (a.best[u] == K && a.best[v] == K) {
            a.mate[u] = v;
            a.mate[v] = u;
            atomicOr(&a.dead[u >> 5], 1u << (u & 31));
            atomicOr(&a.dead[v >> 5], 1u << (v & 31));
            matched += 2;
        }
    }
    __shared__ unsigned long long s_part[EC_T / 32];
    block_add(&a.st->matched2, matched, s_part);
}

constexpr int EC_V = 4;  // edges per thread per step of the compaction
__global__ void __launch_bounds__(EC_T) k_ec_compact(const EdgeArgs* __restrict__ pa) {
    const EdgeArgs& a = *pa;
    __shared__ uint32_t s_cnt[EC_T / 32];
    __shared__ uint32_t s_base;
    const uint32_t r = ec_round(a);
    const uint32_t cnt = r == 0 ? a.m : ld_volatile_u32(&a.st->lcnt[0][r & 1u]);
    const uint32_t* L = a.live[r & 1u];
    uint32_t* N = a.live[(r + 1) & 1u];
    uint32_t* ncnt = &a.st->lcnt[0][(r + 1) & 1u];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = lanemask_lt();
    const uint32_t step = EC_T * EC_V;
    // block-uniform loop: each step keeps the survivors of EC_T * EC_V edges with one
    // atomic for the whole block (slots: warp prefix + vote)
    for (uint32_t b0 = blockIdx.x * step; b0 < cnt; b0 += gridDim.x * step) {
        bool keep[EC_V];
        uint32_t ee[EC_V], ball[EC_V], mine = 0;
#pragma unroll
        for (int k = 0; k < EC_V; k++) {
            const uint32_t i = b0 + k * EC_T + threadIdx.x;
            keep[k] = false;
            ee[k] = 0;
            if (i < cnt) {
                const uint32_t e = r == 0 ? i : L[i];
                ee[k] = e;
                if (e < a.m) {
                    const uint64_t rec = a.edges[e];
                    const uint32_t u = (uint32_t)rec, v = (uint32_t)(rec >> 32);
                    a.best[u] = 0;  // offers and stamps go back to zero for the next round
                    a.best[v] = 0;
                    a.stamp[u] = 0;
                    a.stamp[v] = 0;
                    keep[k] = !(((__ldg(&a.dead[u >> 5]) >> (u & 31)) | (__ldg(&a.dead[v >> 5]) >> (v & 31))) & 1u);
                }
            }
            ball[k] = __ballot_sync(FULL, keep[k]);
            mine += __popc(ball[k]);
        }
        if (lane == 0) s_cnt[warp] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < EC_T / 32; w++) { const uint32_t c = s_cnt[w]; s_cnt[w] = t; t += c; }
            s_base = t ? atomicAdd(ncnt, t) : 0u;
        }
        __syncthreads();
        uint32_t base = s_base + s_cnt[warp];
#pragma unroll
        for (int k = 0; k < EC_V; k++) {
            if (keep[k]) {
                const uint32_t pos = base + __popc(ball[k] & lt);
                if (pos < a.cap) N[pos] = ee[k];
                else set_err(a.st, ERR_BOUNDS, pos);
            }
            base += __popc(ball[k]);
        }
        __syncthreads();  // s_cnt / s_base reuse
    }
}

// one thread: the round's statistics, completion, the next round's index
__device__ void ec_close(const EdgeArgs& a) {
    DevState* st = a.st;
    const uint32_t r = ec_round(a);
    const uint32_t cnt = r == 0 ? a.m : ld_volatile_u32(&st->lcnt[0][r & 1u]);
    const uint32_t next = ld_volatile_u32(&st->lcnt[0][(r + 1) & 1u]);
    if (r < 64) {
        st->ring_m[r] = cnt;
        st->ring_n[r] = ld_volatile_u32(&st->live_rows);
    }
    st->live_rows = 0;
    if (next == 0 && !st->done) {
        st->done = 1;
        st->rounds = r + 1;
    }
    st->round = r + 2;
}
__global__ void k_ec_close(const EdgeArgs* __restrict__ pa) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ec_close(*pa);
}
__global__ void k_ec_check(const EdgeArgs* __restrict__ pa, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    const EdgeArgs& a = *pa;
    ec_close(a);
    DevState* st = a.st;
    unsigned int go = 1;
    if (ld_volatile_u32(&st->done) || ld_volatile_u32(&st->err)) go = 0;
    else if (ld_volatile_u32(&st->round) > ld_volatile_u32(&st->max_rounds) ||
             globaltimer_ns() - st->t0_ns > st->limit_ns) {
        set_err(st, ERR_TIMEOUT, ld_volatile_u32(&st->round));
        go = 0;
    }
    cudaGraphSetConditional(h, go);
}

// ---------------------------------------------------------------- graph construction
// Edge-list passes of the graph build.  Lanes of a warp that hit the same
// vertex (R-MAT hubs) combine into one atomic: the lowest of them adds the
// group's count and hands each its own slot.
__device__ __forceinline__ uint32_t warp_add(uint32_t* ctr, uint32_t key, bool active, uint32_t lane) {
    const uint32_t act = __ballot_sync(FULL, active);
    const uint32_t peers = __match_any_sync(FULL, key) & act;
    // every lane reads its group leader's slot through one full-warp shuffle (a shuffle
    // under each group's own mask inside a branch would run once per group)
    const uint32_t leader = active ? __ffs(peers) - 1 : lane;
    uint32_t base = 0;
    if (active && lane == leader) base = atomicAdd(ctr, (uint32_t)__popc(peers));
    base = __shfl_sync(FULL, base, leader);
    return active ? base + __popc(peers & ((1u << lane) - 1u)) : 0u;
}

__global__ void k_build_degrees(const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n, uint32_t m,
                                uint32_t* deg, uint32_t* err) {
    const uint32_t stride = gridDim.x * blockDim.x, lane = threadIdx.x & 31;
    const uint32_t mr = (m + 31) & ~31u;  // whole warps iterate together
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < mr; e += stride) {
        bool ok = e < m;
        uint32_t u = 0, v = 0;
        if (ok) {
            u = eu[e];
            v = ev[e];
            const uint32_t wb = __float_as_uint(w[e]);
            const bool nan = ((wb & 0x7F800000u) == 0x7F800000u) && (wb & 0x007FFFFFu);
            if (u >= n || v >= n || u == v || nan) {
                atomicOr(err, 1u);
                ok = false;
            }
        }
        warp_add(&deg[ok ? u : 0], u, ok, lane);
        warp_add(&deg[ok ? v : 0], v, ok, lane);
    }
}
// The fill writes every edge's two adjacency entries.  Entries of the first end
// follow the input's order (inputs listed by source vertex write them in runs);
// the second end's would land at random rows, each a partial sector anywhere in
// the arrays.  So they go through 256 buckets of vertex ranges first:
// k_build_vhist counts each tile of BF_TILE edges per bucket, a scan places every
// (bucket, tile) run, k_build_fill_u writes the first ends and appends each
// second-end record (row, neighbour, entry word) to its run, and k_build_fill_v
// walks the records in bucket order, so that the rows it writes at any time lie in
// a window of the arrays that L2 holds.
constexpr uint32_t BF_TILE = 4096, BF_T = 256, BF_NB = 256;

__global__ void __launch_bounds__(BF_T) k_build_vhist(const uint32_t* ev, uint32_t m, uint32_t shift, uint32_t tiles,
                                                      uint32_t* hist) {
    __shared__ uint32_t h[BF_NB];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * BF_TILE;
#pragma unroll 4
    for (uint32_t j = 0; j < BF_TILE / BF_T; j++) {
        const uint64_t e = t0 + j * BF_T + threadIdx.x;
        if (e < m) atomicAdd(&h[(ev[e] >> shift) & (BF_NB - 1)], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];  // bucket-major, for the scan
}

__global__ void __launch_bounds__(BF_T) k_build_fill_u(const uint32_t* eu, const uint32_t* ev, const float* w,
                                                       uint32_t m, uint32_t shift, uint32_t tiles,
                                                       const uint32_t* offs, uint32_t* cursor, uint32_t* nbr,
                                                       uint64_t* pk, uint64_t* edges, uint32_t* eword, uint4* vrec,
                                                       uint32_t* err) {
    __shared__ uint32_t gs[BF_NB], cnt[BF_NB];
    gs[threadIdx.x] = offs[threadIdx.x * tiles + blockIdx.x];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t t0 = (uint64_t)blockIdx.x * BF_TILE;
    for (uint32_t j = 0; j < BF_TILE / BF_T; j++) {  // whole warps iterate together
        const uint64_t e = t0 + j * BF_T + threadIdx.x;
        const bool ok = e < m;
        uint32_t u = 0, v = 0;
        uint64_t word = 0;
        if (ok) {
            u = eu[e];
            v = ev[e];
            const uint32_t ow = ord_of_bits(__float_as_uint(w[e]));
            word = ((uint64_t)ow << 32) | (uint32_t)e;
            edges[e] = (uint64_t)u | ((uint64_t)v << 32);
            eword[e] = ow;
        }
        const uint32_t pu = warp_add(&cursor[u], u, ok, lane);
        if (ok) {
            // the cursors start at the row offsets and the degrees were counted from the
            // same edges, so every slot is below 2m; a stale cursor is reported, not written
            if (pu >= 2 * m) {
                atomicOr(err, 2u);
            } else {
                nbr[pu] = v;
                pk[pu] = word;
            }
            const uint32_t b = (v >> shift) & (BF_NB - 1);
            const uint32_t q = gs[b] + atomicAdd(&cnt[b], 1u);
            if (q < m) vrec[q] = make_uint4(v, u, (uint32_t)word, (uint32_t)(word >> 32));
            else atomicOr(err, 2u);
        }
    }
}

__global__ void __launch_bounds__(BF_T) k_build_fill_v(const uint4* vrec, uint32_t m, uint32_t* cursor, uint32_t* nbr,
                                                       uint64_t* pk, uint32_t* err) {
    const uint32_t stride = gridDim.x * blockDim.x, lane = threadIdx.x & 31;
    const uint32_t mr = (m + 31) & ~31u;  // whole warps iterate together
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < mr; i += stride) {
        const bool ok = i < m;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (ok) r = vrec[i];
        const uint32_t pv = warp_add(&cursor[r.x], r.x, ok, lane);
        if (ok) {
            if (pv >= 2 * m) {
                atomicOr(err, 2u);
            } else {
                nbr[pv] = r.y;
                pk[pv] = ((uint64_t)r.w << 32) | r.z;
            }
        }
    }
}
__global__ void k_nonzero_flags(const uint32_t* deg, uint32_t n, uint32_t* flags) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) flags[v] = deg[v] ? 1u : 0u;
}

__global__ void k_build_rows(const uint32_t* deg, const uint32_t* rowidx, const uint32_t* off, uint32_t n,
                             uint32_t nrows, uint32_t nent, uint32_t* vid0, uint32_t* rdeg0, uint32_t* roff) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (deg[v]) {
            const uint32_t i = rowidx[v];
            vid0[i] = v;
            rdeg0[i] = deg[v];
            roff[i] = off[v];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) roff[nrows] = nent;
}

__global__ void k_build_tilemap(const uint32_t* roff, uint32_t nrows, uint32_t nent, uint32_t* tmap,
                                uint32_t* rbits) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t ntiles = (nent + TILE0 - 1) / TILE0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += stride) {
        const uint32_t lo = roff[i], hi = roff[i + 1];
        for (uint32_t t = (lo + TILE0 - 1) / TILE0; t < (hi + TILE0 - 1) / TILE0; t++) tmap[t] = i;
        atomicOr(&rbits[lo >> 5], 1u << (lo & 31));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) tmap[ntiles] = nrows;
}

// per tile: first row r_lo, rows touched (r_lo .. min(tmap[t + 1], nrows - 1)), offset of row r_lo
__global__ void k_build_tiledesc(const uint32_t* roff, const uint32_t* tmap, uint32_t nrows, uint32_t ntiles,
                                 uint4* tdesc) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += stride) {
        const uint32_t r_lo = tmap[t], r_cap = min(tmap[t + 1], nrows - 1);
        tdesc[t] = make_uint4(r_lo, r_cap - r_lo + 1, roff[r_lo], 0);
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

// graph of vertex v for a warp walking consecutive vertices: lane 0 searches
// for the warp's first vertex, every lane walks forward from there (a warp
// spans few graphs), falling back to a search after 32 steps (runs of empty graphs)
__device__ __forceinline__ uint32_t graph_of_warp(const uint32_t* gvbase, uint32_t ngraphs, uint32_t v,
                                                  uint32_t v0, int lane) {
    // v0: used from lane 0, the warp's lowest vertex
    uint32_t g = 0;
    if (lane == 0) g = graph_of(gvbase, ngraphs, v0);
    g = __shfl_sync(FULL, g, 0);
    for (int steps = 0; g + 1 < ngraphs && gvbase[g + 1] <= v; steps++) {
        if (steps == 32) return graph_of(gvbase, ngraphs, v);
        g++;
    }
    return g;
}

__global__ void k_union_setup(const uint32_t* gvbase, const uint32_t* ebase, const uint32_t* const* offs,
                              uint32_t ngraphs, uint32_t nvert, uint32_t* start, uint32_t* gid, uint32_t* len0) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const uint32_t nr = (nvert + 31) & ~31u;  // whole warps iterate together
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nr; v += stride) {
        const uint32_t vv = min(v, nvert - 1);
        const uint32_t g = graph_of_warp(gvbase, ngraphs, vv, vv, lane);  // lane 0's vertex starts the warp
        if (v >= nvert) continue;
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

__global__ void k_to_local_batch(const uint32_t* mate_u, const uint32_t* gvbase, const uint32_t* gid,
                                 uint32_t* const* dst, unsigned long long* matched2, uint32_t nvert) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const uint32_t nr = (nvert + 31) & ~31u;  // whole warps iterate together
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < nr; v += stride) {
        const bool live = v < nvert;
        uint32_t x = NIL, g = NIL;
        if (live) {
            g = gid[v];
            const uint32_t vb = gvbase[g];
            x = mate_u[v];
            uint32_t* d = dst[g];
            if (d) d[v - vb] = (x == NIL) ? NIL : x - vb;
        }
        // matched vertices per graph, one atomic per graph present in the warp
        const uint32_t hit = __ballot_sync(FULL, live && x != NIL);
        const uint32_t peers = __match_any_sync(FULL, g) & hit;
        if (matched2 && live && x != NIL && lane == __ffs(peers) - 1)
            atomicAdd(&matched2[g], (unsigned long long)__popc(peers));
    }
}
// ---------------------------------------------------------------- exclusive scan (set-up and contraction)
// A block scans a tile of 4096 words in two launches (tile sums, then the tiles'
// prefixes applied), recursing on the tile sums.  Thread t holds four chunks of
// four consecutive words, chunk c at tile offset 1024 c + 4 t, so every warp
// load and store moves 512 contiguous bytes; one block scan runs over the four
// chunk sums of every thread at once.  Unaligned arrays take scalar accesses.
constexpr int SCAN_THREADS = 256, SCAN_CHUNKS = 4, SCAN_TILE = SCAN_THREADS * 4 * SCAN_CHUNKS;

template <bool VEC>
__device__ __forceinline__ uint4 scan_load4(const uint32_t* in, uint64_t i, uint32_t count) {
    if (VEC && i + 4 <= count) return *reinterpret_cast<const uint4*>(in + i);
    uint4 v;
    v.x = i < count ? in[i] : 0u;
    v.y = i + 1 < count ? in[i + 1] : 0u;
    v.z = i + 2 < count ? in[i + 2] : 0u;
    v.w = i + 3 < count ? in[i + 3] : 0u;
    return v;
}

template <bool VEC>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* in, uint32_t count, uint32_t* sums) {
    __shared__ uint32_t tmp[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
    uint4 v[SCAN_CHUNKS];
#pragma unroll
    for (int c = 0; c < SCAN_CHUNKS; c++) v[c] = scan_load4<VEC>(in, base + 1024 * c, count);
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < SCAN_CHUNKS; c++) x += v[c].x + v[c].y + v[c].z + v[c].w;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if (lane == 0) tmp[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += tmp[w];
        sums[blockIdx.x] = t;
    }
}

template <bool VEC>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const uint32_t* in, uint32_t count,
                                                             const uint32_t* offsets, uint32_t* out) {
    __shared__ uint32_t tmp[SCAN_CHUNKS][SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + 4 * threadIdx.x;
    uint4 v[SCAN_CHUNKS];
    uint32_t incl[SCAN_CHUNKS], own[SCAN_CHUNKS];
#pragma unroll
    for (int c = 0; c < SCAN_CHUNKS; c++) {
        v[c] = scan_load4<VEC>(in, base + 1024 * c, count);
        own[c] = v[c].x + v[c].y + v[c].z + v[c].w;
        incl[c] = warp_incl_scan(own[c], lane);
        if (lane == 31) tmp[c][warp] = incl[c];
    }
    __syncthreads();
    // chunk c starts after every earlier chunk of the tile; within it, after the
    // earlier warps and lanes
    uint32_t run = offsets ? offsets[blockIdx.x] : 0u;
#pragma unroll
    for (int c = 0; c < SCAN_CHUNKS; c++) {
        uint32_t before = 0, total = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) {
            const uint32_t t = tmp[c][w];
            before += w < warp ? t : 0u;
            total += t;
        }
        uint4 o;
        o.x = run + before + incl[c] - own[c];
        o.y = o.x + v[c].x;
        o.z = o.y + v[c].y;
        o.w = o.z + v[c].z;
        const uint64_t i = base + 1024 * c;
        if (VEC && i + 4 <= count) {
            *reinterpret_cast<uint4*>(out + i) = o;
        } else {
            if (i < count) out[i] = o.x;
            if (i + 1 < count) out[i + 1] = o.y;
            if (i + 2 < count) out[i + 2] = o.z;
            if (i + 3 < count) out[i + 3] = o.w;
        }
        run += total;
    }
}

size_t exclusive_scan_tmp_words(uint32_t count) {
    size_t words = 0;
    uint64_t c = count;
    while (c > SCAN_TILE) {
        c = (c + SCAN_TILE - 1) / SCAN_TILE;
        words += 2 * ((c + 3) & ~3ull) + 4;  // block sums and their scan at this level, 16-byte aligned
    }
    return words + 4;
}

int launch_exclusive_scan(void* stream, const uint32_t* in, uint32_t* out, uint32_t count, uint32_t* tmp,
                          size_t tmp_words) {
    cudaStream_t s = (cudaStream_t)stream;
    if (count == 0) return 0;
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    const uint32_t blocks = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (blocks == 1) {
        if (vec) k_scan_apply<true><<<1, SCAN_THREADS, 0, s>>>(in, count, nullptr, out);
        else k_scan_apply<false><<<1, SCAN_THREADS, 0, s>>>(in, count, nullptr, out);
        return (int)cudaGetLastError();
    }
    const size_t bw = ((size_t)blocks + 3) & ~(size_t)3;
    if (tmp_words < 2 * bw + 4) return (int)cudaErrorInvalidValue;
    uint32_t* sums = tmp;
    uint32_t* sums_scan = tmp + bw;
    if (vec) k_scan_reduce<true><<<blocks, SCAN_THREADS, 0, s>>>(in, count, sums);
    else k_scan_reduce<false><<<blocks, SCAN_THREADS, 0, s>>>(in, count, sums);
    int e = launch_exclusive_scan(stream, sums, sums_scan, blocks, tmp + 2 * bw, tmp_words - 2 * bw);
    if (e) return e;
    if (vec) k_scan_apply<true><<<blocks, SCAN_THREADS, 0, s>>>(in, count, sums_scan, out);
    else k_scan_apply<false><<<blocks, SCAN_THREADS, 0, s>>>(in, count, sums_scan, out);
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

// the vertex pass fits 4 CTAs per SM (launch bounds); 0 or more takes that
static uint32_t vertex_grid(const LaunchCfg& c) {
    const uint32_t per = (c.vertex_ctas_per_sm == 0 || c.vertex_ctas_per_sm > LM_VMINB) ? (uint32_t)LM_VMINB
                                                                                    : c.vertex_ctas_per_sm;
    return (uint32_t)current_sms() * per;
}

int launch_vertex(void* stream, const VertexArgs* dargs, const LaunchCfg& cfg) {
    // a fixed grid: the pass iterates its rows block-strided (row counts live on the device)
    k_vertex<<<vertex_grid(cfg), VT, 0, (cudaStream_t)stream>>>(dargs);
    return (int)cudaGetLastError();
}

template <bool I, bool C, bool RN>
static uint32_t sweep_grid(const LaunchCfg& cfg) {
    static int blocks_per_sm = 0;
    if (!blocks_per_sm) {
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep<I, C, RN>, ST, 0);
        blocks_per_sm = per > 0 ? per : 1;
    }
    int per = blocks_per_sm;
    if (cfg.sweep_ctas_per_sm && (int)cfg.sweep_ctas_per_sm < per) per = (int)cfg.sweep_ctas_per_sm;
    return (uint32_t)(current_sms() * per);
}

template <bool I, bool C>
static int launch_sweep_t(void* stream, const SweepArgs* dargs, const LaunchCfg& cfg) {
    if (cfg.renew) k_sweep<I, C, true><<<sweep_grid<I, C, true>(cfg), ST, 0, (cudaStream_t)stream>>>(dargs);
    else k_sweep<I, C, false><<<sweep_grid<I, C, false>(cfg), ST, 0, (cudaStream_t)stream>>>(dargs);
    return (int)cudaGetLastError();
}
static int round0_blocks_per_sm() {
    static int per = 0;
    if (!per) {
        cudaError_t e = cudaFuncSetAttribute(k_round0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(R0Smem));
        if (e != cudaSuccess) return -(int)e;
        int p = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, k_round0, R0T, sizeof(R0Smem));
        if (e != cudaSuccess) return -(int)e;
        per = p > 0 ? p : 1;
    }
    return per;
}
// persistent: as many CTAs as fit, tiles strided over the grid
static int round0_grid(uint32_t* grid) {
    const int per = round0_blocks_per_sm();
    if (per < 0) return -per;
    *grid = (uint32_t)(current_sms() * per);
    return 0;
}
int launch_round0(void* stream, const Round0Args* d) {
    uint32_t grid = 0;
    const int e = round0_grid(&grid);
    if (e) return e;
    k_round0<<<grid, R0T, sizeof(R0Smem), (cudaStream_t)stream>>>(d);
    return (int)cudaGetLastError();
}
static uint32_t round0_cut_grid() { return (uint32_t)current_sms() * 2; }
int launch_round0_cut(void* stream, const Round0Args* d) {
    k_round0_cut<<<round0_cut_grid(), 256, 0, (cudaStream_t)stream>>>(d);
    return (int)cudaGetLastError();
}
int launch_sweep_cand(void* stream, const SweepArgs* d, const LaunchCfg& c) {
    if (c.renew) return (int)cudaErrorInvalidValue;  // round 0 keeps the default order: never needed
    return launch_sweep_t<true, false>(stream, d, c);
}
int launch_sweep_input(void* stream, const SweepArgs* d, const LaunchCfg& c) { return launch_sweep_t<true, true>(stream, d, c); }
int launch_sweep_live(void* stream, const SweepArgs* d, const LaunchCfg& c) { return launch_sweep_t<false, true>(stream, d, c); }

int launch_build_degrees(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n,
                         uint32_t m, uint32_t* deg, uint32_t* err) {
    k_build_degrees<<<grid_for(m, 256), 256, 0, (cudaStream_t)stream>>>(eu, ev, w, n, m, deg, err);
    return (int)cudaGetLastError();
}
size_t build_fill_tmp_words(uint32_t n, uint32_t m) {
    (void)n;
    const uint64_t tiles = ((uint64_t)m + BF_TILE - 1) / BF_TILE;
    return (size_t)4 * m + 2 * (BF_NB * tiles + 4) + 8;  // the records (16 B each), counts, their prefix
}
uint32_t build_fill_scan_count(uint32_t n, uint32_t m) {
    (void)n;
    return (uint32_t)(BF_NB * (((uint64_t)m + BF_TILE - 1) / BF_TILE));
}
int launch_build_fill(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n, uint32_t m,
                      uint32_t* cursor, uint32_t* nbr, uint64_t* pk, uint64_t* edges, uint32_t* eword, uint32_t* tmp,
                      uint32_t* scan_tmp, size_t scan_words, uint32_t* err) {
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0) return 0;
    if (!tmp) return (int)cudaErrorInvalidValue;
    uint32_t shift = 0;  // bucket = v >> shift, below 256
    while (((uint64_t)(n - 1) >> shift) > BF_NB - 1) shift++;
    const uint32_t tiles = (uint32_t)(((uint64_t)m + BF_TILE - 1) / BF_TILE);
    uint4* vrec = reinterpret_cast<uint4*>(tmp);           // 16-byte aligned (the caller's carve)
    uint32_t* hist = tmp + 4 * (size_t)m;
    uint32_t* offs = hist + ((BF_NB * (size_t)tiles + 4) & ~(size_t)3);
    k_build_vhist<<<tiles, BF_T, 0, s>>>(ev, m, shift, tiles, hist);
    if (int r = launch_exclusive_scan(stream, hist, offs, BF_NB * tiles, scan_tmp, scan_words)) return r;
    k_build_fill_u<<<tiles, BF_T, 0, s>>>(eu, ev, w, m, shift, tiles, offs, cursor, nbr, pk, edges, eword, vrec, err);
    k_build_fill_v<<<grid_for(m, 256), BF_T, 0, s>>>(vrec, m, cursor, nbr, pk, err);
    return (int)cudaGetLastError();
}
int launch_nonzero_flags(void* stream, const uint32_t* deg, uint32_t n, uint32_t* flags) {
    k_nonzero_flags<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(deg, n, flags);
    return (int)cudaGetLastError();
}
int launch_build_rows(void* stream, const uint32_t* deg, const uint32_t* rowidx_excl, const uint32_t* off,
                      uint32_t n, uint32_t nrows, uint32_t nent, uint32_t* vid0, uint32_t* rdeg0, uint32_t* roff) {
    k_build_rows<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(deg, rowidx_excl, off, n, nrows, nent, vid0,
                                                                     rdeg0, roff);
    return (int)cudaGetLastError();
}
int launch_build_tilemap(void* stream, const uint32_t* roff, uint32_t nrows, uint32_t nent, uint32_t* tmap,
                         uint32_t* rbits, uint4* tdesc) {
    k_build_tilemap<<<grid_for(nrows + 1, 256), 256, 0, (cudaStream_t)stream>>>(roff, nrows, nent, tmap, rbits);
    const uint32_t ntiles = (nent + TILE0 - 1) / TILE0;
    if (ntiles) k_build_tiledesc<<<grid_for(ntiles, 256), 256, 0, (cudaStream_t)stream>>>(roff, tmap, nrows, ntiles,
                                                                                         tdesc);
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
int launch_to_local_batch(void* stream, const uint32_t* mate_union, const uint32_t* gvbase, const uint32_t* gid,
                          uint32_t ngraphs, uint32_t* const* dst, unsigned long long* matched2, uint32_t nvert) {
    if (nvert == 0 || ngraphs == 0) return 0;
    k_to_local_batch<<<grid_for(nvert, 256), 256, 0, (cudaStream_t)stream>>>(mate_union, gvbase, gid, dst, matched2,
                                                                             nvert);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- device-driven loop
// Decides whether the conditional loop of a job graph runs another pair of
// rounds: not once the edge set is empty or an error was recorded; after the
// round cap or the job's time limit it records ERR_TIMEOUT and stops.
__global__ void k_loop_check(DevState* st, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0) return;
    unsigned int go = 1;
    if (ld_volatile_u32(&st->done) || ld_volatile_u32(&st->err)) go = 0;
    else if (ld_volatile_u32(&st->round) > ld_volatile_u32(&st->max_rounds) ||
             globaltimer_ns() - st->t0_ns > st->limit_ns) {
        set_err(st, ERR_TIMEOUT, ld_volatile_u32(&st->round));
        go = 0;
    } else if (*reinterpret_cast<volatile unsigned long long*>(&st->last_ent) < TAIL_ENT) {
        // few entries left: the tail kernel after the loop finishes the job
        st->tail = 1;
        st->tail_round = ld_volatile_u32(&st->round);
        go = 0;
    }
    cudaGraphSetConditional(h, go);
}

// The rounds that remain once few entries are live, in one CTA: the vertex pass
// and the sweep of rounds of both parities (the loop body's arguments) run as
// phases separated by block barriers, with no launch per round.  force = 1 (the
// profiled path) takes over unconditionally; otherwise only when the loop check
// handed over.  The round cap and the time limit hold as in the loop check.
template <bool RENEW>
__global__ void __launch_bounds__(ST, 1) k_tail(const JobArgs* __restrict__ A, uint32_t force) {
    __shared__ WarpRows<RENEW> s_rows[ST / 32];
    __shared__ WarpStage s_stage[ST / 32];
    __shared__ uint32_t s_go;
    DevState* st = A->v[2].st;
    if (threadIdx.x == 0) {
        if (force) {
            st->tail = 1;
            st->tail_round = ld_volatile_u32(&st->round);
        }
        s_go = ld_volatile_u32(&st->tail) && !ld_volatile_u32(&st->done) && !ld_volatile_u32(&st->err);
    }
    __syncthreads();
    if (!s_go) return;
    WarpRows<RENEW>& W = s_rows[threadIdx.x >> 5];
    WarpStage& S = s_stage[threadIdx.x >> 5];
    for (;;) {
        for (int k = 2; k < 4; k++) {
            vertex_pass(A->v[k], 0, 1);
            __syncthreads();
            sweep_pass<false, true, RENEW, true>(A->s[k], W, S, 0, 1);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_go = 1;
            if (ld_volatile_u32(&st->done) || ld_volatile_u32(&st->err)) s_go = 0;
            else if (ld_volatile_u32(&st->round) > ld_volatile_u32(&st->max_rounds) ||
                     globaltimer_ns() - st->t0_ns > st->limit_ns) {
                set_err(st, ERR_TIMEOUT, ld_volatile_u32(&st->round));
                s_go = 0;
            }
        }
        __syncthreads();
        if (!s_go) break;
    }
}

int launch_tail(void* stream, const JobArgs* dargs, const LaunchCfg& cfg) {
    if (cfg.renew) k_tail<true><<<1, ST, 0, (cudaStream_t)stream>>>(dargs, 1u);
    else k_tail<false><<<1, ST, 0, (cudaStream_t)stream>>>(dargs, 1u);
    return (int)cudaGetLastError();
}

static cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, cudaGraphNode_t dep, void* func, dim3 grid,
                              dim3 block, void** params, unsigned smem = 0) {
    cudaKernelNodeParams kp{};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = smem;
    kp.kernelParams = params;
    return cudaGraphAddKernelNode(node, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

// init -> round-0 candidate tiles (+ cut rows) -> round-0 match -> round-0
// compaction from the input arrays -> round 1 -> while (live) { two rounds }
int build_job_graph(const JobArgs* dargs, DevState* st, const LaunchCfg& cfg, void** exec_out) {
    *exec_out = nullptr;
    uint32_t rgrid = 0;
    if (int pe = round0_grid(&rgrid)) return pe;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return (int)e;
    cudaGraphNode_t prev = nullptr, node = nullptr;
    // kernel parameters: one pointer to the arguments in device memory
    const InitArgs* p_init = &dargs->init;
    const Round0Args* pr = &dargs->r0;
    const VertexArgs* pv[4] = {&dargs->v[0], &dargs->v[1], &dargs->v[2], &dargs->v[3]};
    const SweepArgs* ps[4] = {&dargs->s[0], &dargs->s[1], &dargs->s[2], &dargs->s[3]};
    void* init_params[1] = {&p_init};
    void* rparams[1] = {&pr};
    void* vparams[4][1], *sparams[4][1];
    for (int k = 0; k < 4; k++) {
        vparams[k][0] = &pv[k];
        sparams[k][0] = &ps[k];
    }
    const dim3 vgrid(vertex_grid(cfg)), vblock(VT), sblock(ST), rblock(R0T), cgrid(round0_cut_grid());
    const bool rn = cfg.renew;
    const dim3 lgrid(rn ? sweep_grid<false, true, true>(cfg) : sweep_grid<false, true, false>(cfg));
    const dim3 igrid(rn ? sweep_grid<true, true, true>(cfg) : sweep_grid<true, true, false>(cfg));
    void* const k_input = rn ? (void*)k_sweep<true, true, true> : (void*)k_sweep<true, true, false>;
    void* const k_live = rn ? (void*)k_sweep<false, true, true> : (void*)k_sweep<false, true, false>;
    do {
        if ((e = add_kernel(g, &node, prev, (void*)k_init, dim3(current_sms() * 16), dim3(256), init_params))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_round0, dim3(rgrid), rblock, rparams, sizeof(R0Smem)))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_round0_cut, cgrid, dim3(256), rparams))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_vertex, vgrid, vblock, vparams[0]))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, k_input, igrid, sblock, sparams[0]))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, (void*)k_vertex, vgrid, vblock, vparams[1]))) break;
        prev = node;
        if ((e = add_kernel(g, &node, prev, k_live, lgrid, sblock, sparams[1]))) break;
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
            if ((e = add_kernel(body, &bn, bp, k_live, lgrid, sblock, sparams[k]))) break;
            bp = bn;
        }
        if (e) break;
        void* cparams[2] = {&st, &h};
        if ((e = add_kernel(body, &bn, bp, (void*)k_loop_check, dim3(1), dim3(32), cparams))) break;
        // after the loop: the one-CTA tail (returns at once unless the loop check handed over)
        const JobArgs* pd = dargs;
        uint32_t no_force = 0;
        void* tparams[2] = {&pd, &no_force};
        void* const k_t = rn ? (void*)k_tail<true> : (void*)k_tail<false>;
        prev = node;
        if ((e = add_kernel(g, &node, prev, k_t, dim3(1), dim3(ST), tparams))) break;
        cudaGraphExec_t ex = nullptr;
        if ((e = cudaGraphInstantiate(&ex, g, 0))) break;
        *exec_out = ex;
    } while (0);
    cudaGraphDestroy(g);
    return (int)e;
}

static uint32_t ec_grid() { return (uint32_t)current_sms() * 8; }

int launch_edge_round(void* stream, const EdgeArgs* d, int phase) {
    const cudaStream_t s = (cudaStream_t)stream;
    switch (phase) {
        case 0: k_ec_offer<<<ec_grid(), EC_T, 0, s>>>(d); break;
        case 1: k_ec_match<<<ec_grid(), EC_T, 0, s>>>(d); break;
        case 2: k_ec_compact<<<ec_grid(), EC_T, 0, s>>>(d); break;
        default: k_ec_close<<<1, 32, 0, s>>>(d); break;
    }
    return (int)cudaGetLastError();
}

// init -> while (live) { offer, match, compact, check }
int build_edge_graph(const InitArgs* init, const EdgeArgs* dargs, DevState* /*st*/, void** exec_out) {
    *exec_out = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return (int)e;
    const InitArgs* p_init = init;
    const EdgeArgs* p_a = dargs;
    void* init_params[1] = {&p_init};
    void* params[1] = {&p_a};
    cudaGraphNode_t node = nullptr;
    do {
        if ((e = add_kernel(g, &node, nullptr, (void*)k_init, dim3(current_sms() * 16), dim3(256), init_params))) break;
        cudaGraphNode_t prev = node;
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
        cudaGraphNode_t bn = nullptr, bp = nullptr;
        const dim3 grid(ec_grid()), block(EC_T);
        if ((e = add_kernel(body, &bn, bp, (void*)k_ec_offer, grid, block, params))) break;
        bp = bn;
        if ((e = add_kernel(body, &bn, bp, (void*)k_ec_match, grid, block, params))) break;
        bp = bn;
        if ((e = add_kernel(body, &bn, bp, (void*)k_ec_compact, grid, block, params))) break;
        bp = bn;
        void* cparams[2] = {&p_a, &h};
        if ((e = add_kernel(body, &bn, bp, (void*)k_ec_check, dim3(1), dim3(32), cparams))) break;
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

// ---------------------------------------------------------------- small graphs without allocation
// lm_match_small_noalloc: local max for one small graph whose edge list is
// already on the device, run by one CTA whose only scratch is the static
// array below (no allocation at call time).  Each round every live edge
// offers its key to both ends, an edge that is the heaviest offer at both ends
// is matched, and edges with a matched end leave (Sec. 2, the phases of local
// max, with the same order K as the main path).
constexpr uint32_t NA_MAX_N = LM_NOALLOC_MAX_N, NA_MAX_M = LM_NOALLOC_MAX_M;
struct NaScratch {
    unsigned long long best[NA_MAX_N];   // heaviest offer at each vertex in the current round
    uint32_t live[2][NA_MAX_M];          // live edge ids, alternating between rounds
    uint8_t dead[NA_MAX_N];              // matched
};
static_assert(sizeof(NaScratch) == LM_NOALLOC_SCRATCH_BYTES, "scratch size as documented");
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NaScratch)];

constexpr int NA_T = 1024;
__global__ void __launch_bounds__(NA_T, 1) k_match_small(uint32_t n, uint32_t m, const uint32_t* __restrict__ eu,
                                                         const uint32_t* __restrict__ ev, const float* __restrict__ w,
                                                         uint32_t k0, uint32_t k1, uint32_t* mate, uint32_t* status,
                                                         NaScratch* sc) {
    __shared__ uint32_t s_cnt[2], s_err;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        s_cnt[0] = 0;
        s_cnt[1] = 0;
        s_err = 0;
    }
    for (uint32_t v = tid; v < n; v += NA_T) {
        mate[v] = NIL;
        sc->best[v] = 0;
        sc->dead[v] = 0;
    }
    __syncthreads();
    for (uint32_t e = tid; e < m; e += NA_T) {
        const uint32_t u = eu[e], v = ev[e], wb = __float_as_uint(w[e]);
        const bool nan = ((wb & 0x7F800000u) == 0x7F800000u) && (wb & 0x007FFFFFu);
        if (u >= n || v >= n || u == v || nan) {
            atomicOr(&s_err, 1u);
            continue;
        }
        sc->live[0][atomicAdd(&s_cnt[0], 1u)] = e;
    }
    __syncthreads();
    uint32_t cur = 0, count = s_err ? 0u : s_cnt[0];
    auto key = [&](uint32_t e) -> unsigned long long {
        return ((unsigned long long)ord_of_bits(__float_as_uint(w[e])) << 32) | perm_seed(e, k0, k1);
    };
    for (uint32_t round = 0; count > 0; round++) {
        if (round > m) {  // every round matches at least one edge
            if (tid == 0) s_err |= 2u;
            break;
        }
        for (uint32_t i = tid; i < count; i += NA_T) {
            const uint32_t e = __ldcg(&sc->live[cur][i]);
            const unsigned long long K = key(e);
            atomicMax(&sc->best[eu[e]], K);
            atomicMax(&sc->best[ev[e]], K);
        }
        if (tid == 0) s_cnt[cur ^ 1u] = 0;
        __syncthreads();
        for (uint32_t i = tid; i < count; i += NA_T) {
            const uint32_t e = __ldcg(&sc->live[cur][i]);
            const uint32_t u = eu[e], v = ev[e];
            const unsigned long long K = key(e);
            // read at L2, where the atomics of this round landed
            if (__ldcg(&sc->best[u]) == K && __ldcg(&sc->best[v]) == K) {
                mate[u] = v;
                mate[v] = u;
                sc->dead[u] = 1;
                sc->dead[v] = 1;
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < count; i += NA_T) {
            const uint32_t e = __ldcg(&sc->live[cur][i]);
            const uint32_t u = eu[e], v = ev[e];
            sc->best[u] = 0;
            sc->best[v] = 0;
            if (!__ldcg(&sc->dead[u]) && !__ldcg(&sc->dead[v]))
                sc->live[cur ^ 1u][atomicAdd(&s_cnt[cur ^ 1u], 1u)] = e;
        }
        __syncthreads();
        count = s_cnt[cur ^ 1u];
        cur ^= 1u;
        __syncthreads();
    }
    __syncthreads();
    // a round cap that tripped leaves no partial result behind: every vertex unmatched
    if (s_err & 2u)
        for (uint32_t v = tid; v < n; v += NA_T) mate[v] = NIL;
    if (tid == 0) *status = s_err;
}

}  // namespace lm

// The scratch's address on each device, looked up once with that device current.
namespace {
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
void* g_na_ptr[NA_MAX_DEVICES] = {};
}  // namespace

extern "C" int lm_match_small_noalloc(uint32_t n, uint32_t m, const uint32_t* eu, const uint32_t* ev,
                                      const float* w, uint64_t seed, uint32_t* mate, uint32_t* status,
                                      void* stream) {
    if (n > LM_NOALLOC_MAX_N || m > LM_NOALLOC_MAX_M) return LM_EINVAL;
    if (!status || (n > 0 && !mate) || (m > 0 && (!eu || !ev || !w))) return LM_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LM_ECUDA;
    }
    if (dev < 0 || dev >= NA_MAX_DEVICES) return LM_EINVAL;
    // every array must be global memory of the current device: a pointer into host
    // memory or into another GPU would be dereferenced by the kernel as it is
    const void* arrays[5] = {eu, ev, w, mate, status};
    const bool needed[5] = {m > 0, m > 0, m > 0, n > 0, true};
    for (int i = 0; i < 5; i++) {
        if (!needed[i]) continue;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, arrays[i]) != cudaSuccess) {
            cudaGetLastError();
            return LM_EINVAL;
        }
        if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
            return LM_EINVAL;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, lm::g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return LM_ECUDA;
            }
            g_na_ptr[dev] = p;
        }
        scratch = g_na_ptr[dev];
    }
    const uint64_t z = lm::splitmix64_first(seed);
    lm::k_match_small<<<1, lm::NA_T, 0, (cudaStream_t)stream>>>(n, m, eu, ev, w, (uint32_t)z, (uint32_t)(z >> 32),
                                                               mate, status, static_cast<lm::NaScratch*>(scratch));
    if (cudaGetLastError() != cudaSuccess) return LM_ECUDA;
    return LM_OK;
}
