// Contraction of a matching: the step that multilevel graph partitioning
// repeats on maximal matchings (Sec. 1 names it as the main use of the
// matching).  Reading: a matched pair becomes one coarse vertex and an
// unmatched vertex stays alone; coarse ids number the representatives (the
// unmatched vertices and the smaller end of each pair) in vertex order; a
// coarse vertex weighs the sum of its members; edges inside a pair vanish;
// the original edges between two coarse vertices become one coarse edge,
// placed and oriented as the first of them in the input order, whose weight
// is their sum (accumulated in double, rounded once to float32).
//
// Device steps (all of them here): representatives and their prefix ranks;
// the coarse map and vertex weights; every crossing edge inserts its unordered
// coarse pair into an open-addressing table (64-bit key, linear probing): the
// edge that creates a slot stores itself as the pair's leader and its weight
// as the sum with plain stores, and an edge that finds its pair already there
// marks itself; in the next kernel only those marked edges lower the leader
// (the smallest edge index) and add their weight with atomics (most pairs have
// one edge and need none); leader flags over the edges and their prefix ranks
// give each coarse edge its place; the leaders write the coarse edges.
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/lm.h"
#include "lm_internal.h"

namespace lm {

namespace {

constexpr uint32_t CT = 256;
constexpr uint32_t SLOT_DUP = 0x80000000u;  // slot_of: the pair was already in the table
constexpr uint32_t C_ERR_MATE = 1u, C_ERR_EDGE = 2u, C_ERR_TABLE = 4u;

__device__ __forceinline__ uint64_t pair_hash(uint64_t k) {
    // SplitMix64's output mix (Steele, Lea, Flood 2014)
    k = (k ^ (k >> 30)) * 0xBF58476D1CE4E5B9ull;
    k = (k ^ (k >> 27)) * 0x94D049BB133111EBull;
    return k ^ (k >> 31);
}

__global__ void k_c_rep(const uint32_t* __restrict__ mate, uint32_t n, uint32_t* __restrict__ flag,
                        uint32_t* __restrict__ err) {
    for (uint32_t v = blockIdx.x * CT + threadIdx.x; v < n; v += gridDim.x * CT) {
        const uint32_t u = mate[v];
        bool rep = true;
        if (u != NIL) {
            if (u >= n || u == v || mate[u] != v) { atomicOr(err, C_ERR_MATE); rep = false; }
            else rep = v < u;
        }
        flag[v] = rep ? 1u : 0u;
    }
}

__global__ void k_c_map(const uint32_t* __restrict__ mate, uint32_t n, const uint32_t* __restrict__ rank,
                        const uint32_t* __restrict__ vw, uint32_t* __restrict__ cmap, uint32_t* __restrict__ cvw) {
    for (uint32_t v = blockIdx.x * CT + threadIdx.x; v < n; v += gridDim.x * CT) {
        uint32_t u = mate[v];
        if (u >= n) u = v;  // unmatched (an invalid mate was flagged by k_c_rep)
        const uint32_t c = rank[u < v ? u : v];
        cmap[v] = c;
        atomicAdd(&cvw[c], vw ? vw[v] : 1u);
    }
}

__global__ void k_c_insert(const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                           const float* __restrict__ w, uint32_t m, uint32_t n, const uint32_t* __restrict__ cmap,
                           uint32_t tslots, PairSlot* __restrict__ table, uint32_t* __restrict__ slot_of,
                           uint32_t* __restrict__ err) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        slot_of[e] = NIL;
        const uint32_t a = eu[e], b = ev[e];
        if (a >= n || b >= n) { atomicOr(err, C_ERR_EDGE); continue; }
        const uint32_t c = cmap[a], d = cmap[b];
        if (c == d) continue;  // inside a matched pair
        // key + 1: zero marks an empty slot
        const unsigned long long key = ((((unsigned long long)min(c, d)) << 32) | max(c, d)) + 1ull;
        // slot: the hash's high half scaled to the table (multiply-shift), then linear probing
        uint32_t h = (uint32_t)(((pair_hash(key) >> 32) * (unsigned long long)tslots) >> 32);
        bool placed = false, created = false;
        for (uint32_t probe = 0; probe < tslots; probe++) {
            const unsigned long long old = atomicCAS(&table[h].key, 0ull, key);
            if (old == 0ull || old == key) {
                placed = true;
                created = old == 0ull;
                break;
            }
            h = (h + 1u == tslots) ? 0u : h + 1u;
        }
        if (!placed) { atomicOr(err, C_ERR_TABLE); continue; }
        if (created) {
            // the slot's creator: leader and sum so far (others add theirs in the next kernel)
            table[h].lead = e;
            table[h].sum = (double)w[e];
            slot_of[e] = h;
        } else {
            slot_of[e] = h | SLOT_DUP;
        }
    }
}

// edges whose pair was already in the table: lower the leader, add the weight
__global__ void k_c_merge(const float* __restrict__ w, uint32_t m, PairSlot* __restrict__ table,
                          uint32_t* __restrict__ slot_of) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        const uint32_t h = slot_of[e];
        if (h == NIL || !(h & SLOT_DUP)) continue;
        const uint32_t hs = h & ~SLOT_DUP;
        atomicMin(&table[hs].lead, e);
        atomicAdd(&table[hs].sum, (double)w[e]);
        slot_of[e] = hs;
    }
}

// empty slots: key 0, leader NIL, sum 0 (one 32-byte store per slot)
__global__ void k_c_clear(PairSlot* __restrict__ table, uint32_t slots) {
    for (uint32_t i = blockIdx.x * CT + threadIdx.x; i < slots; i += gridDim.x * CT) {
        PairSlot z;
        z.key = 0ull;
        z.lead = NIL;
        z.pad = 0;
        z.sum = 0.0;
        z.pad2 = 0.0;
        table[i] = z;
    }
}

__global__ void k_c_lead(uint32_t m, const uint32_t* __restrict__ slot_of, const PairSlot* __restrict__ table,
                         uint32_t* __restrict__ isl) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        const uint32_t h = slot_of[e];
        isl[e] = (h != NIL && table[h].lead == e) ? 1u : 0u;
    }
}

__global__ void k_c_emit(uint32_t m, const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                         const uint32_t* __restrict__ cmap, const uint32_t* __restrict__ slot_of,
                         const PairSlot* __restrict__ table, const uint32_t* __restrict__ isl,
                         const uint32_t* __restrict__ pos, uint32_t* __restrict__ ceu, uint32_t* __restrict__ cev,
                         float* __restrict__ cw) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        if (!isl[e]) continue;
        const uint32_t p = pos[e];
        ceu[p] = cmap[eu[e]];
        cev[p] = cmap[ev[e]];
        cw[p] = (float)table[slot_of[e]].sum;
    }
}

uint32_t grid_for(uint64_t count) {
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t b = (count + CT - 1) / CT;
    const uint64_t cap = (uint64_t)device_sm_count(dev) * 16;
    return (uint32_t)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

// table slots: two per edge (load factor at most one half: linear probing stays short;
// 1.25 per edge measured 30% slower on R-MAT 23), at least 1024
int contract_table_slots(uint32_t m, uint32_t* slots) {
    const uint64_t t = 2ull * m + 1024;
    if (t >= SLOT_DUP) return (int)cudaErrorInvalidValue;  // slot indices keep bit 31 free
    *slots = (uint32_t)t;
    return 0;
}

int launch_contract(void* stream, const ContractArgs& c) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c.err, 0, sizeof(uint32_t), s))) return (int)e;
    if ((e = cudaMemsetAsync(c.flag + c.n, 0, sizeof(uint32_t), s))) return (int)e;
    if ((e = cudaMemsetAsync(c.cvw, 0, (size_t)c.n * sizeof(uint32_t), s))) return (int)e;
    if (c.m) k_c_clear<<<grid_for(c.tslots), CT, 0, s>>>(c.table, c.tslots);
    if ((e = cudaMemsetAsync(c.isl + c.m, 0, sizeof(uint32_t), s))) return (int)e;
    k_c_rep<<<grid_for(c.n), CT, 0, s>>>(c.mate, c.n, c.flag, c.err);
    if (int r = launch_exclusive_scan(s, c.flag, c.rank, c.n + 1, c.scan_tmp, c.scan_words)) return r;
    k_c_map<<<grid_for(c.n), CT, 0, s>>>(c.mate, c.n, c.rank, c.vw, c.cmap, c.cvw);
    if (c.m) {
        k_c_insert<<<grid_for(c.m), CT, 0, s>>>(c.eu, c.ev, c.w, c.m, c.n, c.cmap, c.tslots, c.table,
                                                 c.slot_of, c.err);
        k_c_merge<<<grid_for(c.m), CT, 0, s>>>(c.w, c.m, c.table, c.slot_of);
        k_c_lead<<<grid_for(c.m), CT, 0, s>>>(c.m, c.slot_of, c.table, c.isl);
    }
    if (int r = launch_exclusive_scan(s, c.isl, c.pos, c.m + 1, c.scan_tmp, c.scan_words)) return r;
    if (c.m)
        k_c_emit<<<grid_for(c.m), CT, 0, s>>>(c.m, c.eu, c.ev, c.cmap, c.slot_of, c.table, c.isl, c.pos, c.ceu,
                                               c.cev, c.cw);
    return (int)cudaGetLastError();
}

}  // namespace lm
