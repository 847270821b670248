// Contraction of a matching: the step that multilevel graph partitioning
// repeats on maximal matchings (Sec. 1 names it as the main use of the
// matching).  Reading: a matched pair becomes one coarse vertex and an
// unmatched vertex stays alone; coarse ids number the representatives (the
// unmatched vertices and the smaller end of each pair) in vertex order; a
// coarse vertex weighs the sum of its members; edges inside a pair vanish;
// the original edges between two coarse vertices become one coarse edge,
// placed and oriented as the first of them in the input order, whose weight
// is their sum (accumulated in double in input order, rounded once to float32).
//
// Device steps (all of them here): representatives and their prefix ranks;
// the coarse map and vertex weights; every edge, in input order, gets its
// unordered coarse pair as a key (edges inside a pair a key above all pairs,
// so that they end up last); a stable LSD radix sort
// (8-bit digits over the key's significant bits) groups equal pairs with their
// edges still in input order; each group's first edge is its leader and the
// group's weight sum is taken over its edges in order; leader flags over the
// edges (the crossing flags with every non-leader cleared) and their prefix
// ranks give each coarse edge its place; the leaders write the coarse edges.
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/lm.h"
#include "lm_internal.h"

namespace lm {

namespace {

constexpr uint32_t CT = 256;
constexpr uint32_t C_ERR_MATE = 1u, C_ERR_EDGE = 2u;

uint32_t grid_for(uint64_t count) {
    int dev = 0;
    cudaGetDevice(&dev);
    const uint64_t b = (count + CT - 1) / CT;
    const uint64_t cap = (uint64_t)device_sm_count(dev) * 16;
    return (uint32_t)(b < 1 ? 1 : (b > cap ? cap : b));
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

// every edge in input order, keyed by its unordered coarse pair
// min(c, d) << bits | max(c, d); an edge inside a pair (or with an endpoint >= n)
// gets the key 2^(2 bits) - 1, above every pair's, so the sort puts it at the end.
// cross[e] = 1 for the edges between two coarse vertices (they are counted in
// *ncross), 0 for the others.
__global__ void k_c_keys(const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev, uint32_t m, uint32_t n,
                         const uint32_t* __restrict__ cmap, uint32_t bits, unsigned long long* __restrict__ key,
                         uint32_t* __restrict__ val, uint32_t* __restrict__ cross, uint32_t* __restrict__ ncross,
                         uint32_t* __restrict__ err) {
    const unsigned long long none = (1ull << (2 * bits)) - 1ull;
    uint32_t mine = 0;
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        const uint32_t a = eu[e], b = ev[e];
        unsigned long long k = none;
        uint32_t x = 0;
        if (a >= n || b >= n) {
            atomicOr(err, C_ERR_EDGE);
        } else {
            const uint32_t c = cmap[a], d = cmap[b];
            if (c != d) {
                k = ((unsigned long long)min(c, d) << bits) | max(c, d);
                x = 1;
            }
        }
        key[e] = k;
        val[e] = e;
        cross[e] = x;
        mine += x;
    }
    // one atomic per warp on the count
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(ncross, mine);
}

// ---- stable LSD radix sort of (key, value) pairs, 8 bits per pass ----------
// A block takes RS_TILE consecutive items.  Pass part 1 counts the block's
// digits; a scan over (digit, block) gives every block the output offset of
// each digit; part 2 ranks the block's items stably (warp by warp, 32 items
// at a time in input order: lanes with the same digit by a match, earlier
// rounds and warps by shared counters) and scatters them.
constexpr uint32_t RS_T = 256, RS_I = 8, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32;

__global__ void __launch_bounds__(RS_T) k_rs_hist(const unsigned long long* __restrict__ key, uint32_t cnt,
                                                  uint32_t shift, uint32_t nblk, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * RS_TILE;
    for (uint32_t i = threadIdx.x; i < RS_TILE; i += RS_T) {
        const uint32_t q = base + i;
        if (q < cnt) atomicAdd(&h[(uint32_t)(key[q] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];  // digit-major for the scan
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const unsigned long long* __restrict__ key_in,
                                                     const uint32_t* __restrict__ val_in, uint32_t cnt, uint32_t shift,
                                                     uint32_t nblk, const uint32_t* __restrict__ offs,
                                                     unsigned long long* __restrict__ key_out,
                                                     uint32_t* __restrict__ val_out) {
    __shared__ uint32_t wcnt[RS_W][256];  // items of each digit seen so far by each warp
    __shared__ uint32_t wpre[RS_W][256];  // exclusive prefix over warps (plus the digit's block start)
    __shared__ uint32_t dstart[256];      // block-local start of each digit
    __shared__ unsigned long long sk[RS_TILE];
    __shared__ uint32_t sv[RS_TILE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t i = threadIdx.x; i < RS_W * 256; i += RS_T) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    // warp w owns items [w * 32 RS_I, (w + 1) * 32 RS_I) of the tile, 32 per round in order
    const uint32_t tile0 = blockIdx.x * RS_TILE;
    const uint32_t base = tile0 + warp * 32 * RS_I;
    const uint32_t nin = cnt > tile0 ? min(RS_TILE, cnt - tile0) : 0u;
    const uint32_t lt = (1u << lane) - 1u;
    unsigned long long k[RS_I];
    uint32_t v[RS_I], d[RS_I], r[RS_I];
#pragma unroll
    for (int j = 0; j < (int)RS_I; j++) {
        const uint32_t q = base + j * 32 + lane;
        const bool ok = q < cnt;
        k[j] = ok ? key_in[q] : 0ull;
        v[j] = ok ? val_in[q] : 0u;
        d[j] = ok ? (uint32_t)(k[j] >> shift) & 0xFFu : 256u + lane;  // lanes past the end match nobody
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d[j]);
        r[j] = 0;
        if (ok) {
            const uint32_t before = wcnt[warp][d[j]];
            r[j] = before + __popc(peers & lt);
            __syncwarp(peers);
            if ((peers >> lane) == 1u) wcnt[warp][d[j]] = before + __popc(peers);  // the group's last lane
        }
        __syncwarp();
    }
    __syncthreads();
    {
        const uint32_t dg = threadIdx.x;  // one digit per thread: its total, then its block-local start
        uint32_t run = 0;
        for (int w = 0; w < (int)RS_W; w++) run += wcnt[w][dg];
        // exclusive scan of the 256 digit totals across the block
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ uint32_t wsum[RS_W];
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; w++) before += wsum[w];
        const uint32_t start = before + x - run;
        dstart[dg] = start;
        uint32_t acc = start;
        for (int w = 0; w < (int)RS_W; w++) {
            wpre[w][dg] = acc;
            acc += wcnt[w][dg];
        }
    }
    __syncthreads();
    // the tile in digit order in shared memory ...
#pragma unroll
    for (int j = 0; j < (int)RS_I; j++) {
        const uint32_t q = base + j * 32 + lane;
        if (q >= cnt) continue;
        const uint32_t p = wpre[warp][d[j]] + r[j];
        sk[p] = k[j];
        sv[p] = v[j];
    }
    __syncthreads();
    // ... then written out: consecutive threads take consecutive items, which within
    // a digit land on consecutive addresses
    for (uint32_t p = threadIdx.x; p < nin; p += RS_T) {
        const unsigned long long kk = sk[p];
        const uint32_t dg = (uint32_t)(kk >> shift) & 0xFFu;
        const uint32_t o = offs[dg * nblk + blockIdx.x] + (p - dstart[dg]);
        key_out[o] = kk;
        val_out[o] = sv[p];
    }
}

// groups in sorted order (runs of equal keys; a run's first item is its leader,
// the smallest edge index, since the sort is stable and the items entered in
// input order).  Almost every group is a single edge, so instead of marking
// the leaders (a scattered write per group) this clears the crossing flag of
// every other member, and marks the leaders of groups with several edges
// (a bit, and where their run starts).  The flags then say which edges lead.
__global__ void k_c_marks(const unsigned long long* __restrict__ key, const uint32_t* __restrict__ val, uint32_t cnt,
                          uint32_t* __restrict__ lead, uint32_t* __restrict__ multi, uint32_t* __restrict__ gref) {
    for (uint32_t i = blockIdx.x * CT + threadIdx.x; i < cnt; i += gridDim.x * CT) {
        const unsigned long long k = key[i];
        const uint32_t e = val[i];
        if (i > 0 && k == key[i - 1]) {
            lead[e] = 0u;
        } else if (i + 1 < cnt && key[i + 1] == k) {
            atomicOr(&multi[e >> 5], 1u << (e & 31));
            gref[e] = i;
        }
    }
}

// the leaders, in input order, write their coarse edge at their rank among the
// leaders; the weight is the group's sum over its edges in input order (a single
// edge's own weight, which double and back leaves unchanged)
__global__ void k_c_emit(uint32_t m, const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                         const float* __restrict__ w, const uint32_t* __restrict__ cmap,
                         const uint32_t* __restrict__ lead, const uint32_t* __restrict__ multi,
                         const uint32_t* __restrict__ pos, const uint32_t* __restrict__ gref,
                         const unsigned long long* __restrict__ key, const uint32_t* __restrict__ val, uint32_t cnt,
                         uint32_t* __restrict__ ceu, uint32_t* __restrict__ cev, float* __restrict__ cw) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        if (!lead[e]) continue;
        const uint32_t p = pos[e];
        float we = w[e];
        if ((__ldg(&multi[e >> 5]) >> (e & 31)) & 1u) {
            const uint32_t i0 = gref[e];
            const unsigned long long k = key[i0];
            double sum = 0.0;
            for (uint32_t i = i0; i < cnt && key[i] == k; i++) sum += (double)w[val[i]];
            we = (float)sum;
        }
        ceu[p] = cmap[eu[e]];
        cev[p] = cmap[ev[e]];
        cw[p] = we;
    }
}

uint32_t bits_for(uint32_t x) {  // bits to write 0 .. x
    uint32_t b = 1;
    while (b < 32 && (x >> b)) b++;
    return b;
}

}  // namespace

size_t contract_sort_tmp_words(uint32_t m) {
    const uint64_t nblk = ((uint64_t)m + RS_TILE - 1) / RS_TILE;
    return (size_t)(256 * nblk + 1);
}

int launch_contract(void* stream, const ContractArgs& c, uint32_t* mc_host_slot) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c.err, 0, sizeof(uint32_t), s))) return (int)e;
    if ((e = cudaMemsetAsync(c.flag + c.n, 0, sizeof(uint32_t), s))) return (int)e;
    if ((e = cudaMemsetAsync(c.cvw, 0, (size_t)c.n * sizeof(uint32_t), s))) return (int)e;
    k_c_rep<<<grid_for(c.n), CT, 0, s>>>(c.mate, c.n, c.flag, c.err);
    if (int r = launch_exclusive_scan(s, c.flag, c.rank, c.n + 1, c.scan_tmp, c.scan_words)) return r;
    k_c_map<<<grid_for(c.n), CT, 0, s>>>(c.mate, c.n, c.rank, c.vw, c.cmap, c.cvw);
    if (c.m == 0) return (int)cudaGetLastError();
    // the coarse vertex count decides the key's width: read it on the host
    if ((e = cudaMemcpyAsync(mc_host_slot + 1, c.rank + c.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s))) return (int)e;
    if ((e = cudaStreamSynchronize(s))) return (int)e;
    const uint32_t nc = mc_host_slot[1];
    const uint32_t bits = bits_for(nc);  // coarse ids 0 .. nc - 1 and the pair key's top value stay apart
    // every edge keyed in input order; the stable sort keeps input order among equal keys
    // and puts the edges inside pairs last, after the mc crossing edges
    if ((e = cudaMemsetAsync(c.cross + c.m, 0, sizeof(uint32_t), s))) return (int)e;
    if ((e = cudaMemsetAsync(c.cpos, 0, sizeof(uint32_t), s))) return (int)e;
    k_c_keys<<<grid_for(c.m), CT, 0, s>>>(c.eu, c.ev, c.m, c.n, c.cmap, bits, c.key[0], c.val[0], c.cross, c.cpos,
                                          c.err);
    if ((e = cudaMemcpyAsync(mc_host_slot, c.cpos, sizeof(uint32_t), cudaMemcpyDeviceToHost, s))) return (int)e;
    if ((e = cudaStreamSynchronize(s))) return (int)e;
    const uint32_t mc = mc_host_slot[0];
    // radix passes over the key's 2 * bits significant bits
    int cur = 0;
    const uint32_t ns = mc < c.m ? c.m : mc;  // the crossing edges and, past them, the ones inside pairs
    if (mc > 1 || (mc && ns > mc)) {
        const uint32_t nblk = (ns + RS_TILE - 1) / RS_TILE;
        for (uint32_t shift = 0; shift < 2 * bits; shift += 8) {
            k_rs_hist<<<nblk, RS_T, 0, s>>>(c.key[cur], ns, shift, nblk, c.hist);
            if (int r = launch_exclusive_scan(s, c.hist, c.hoff, 256 * nblk, c.scan_tmp, c.scan_words)) return r;
            k_rs_scatter<<<nblk, RS_T, 0, s>>>(c.key[cur], c.val[cur], ns, shift, nblk, c.hoff, c.key[cur ^ 1],
                                               c.val[cur ^ 1]);
            cur ^= 1;
        }
    }
    // the crossing flags become the leader flags: other members are cleared
    if ((e = cudaMemsetAsync(c.multi, 0, ((size_t)c.m / 32 + 2) * sizeof(uint32_t), s))) return (int)e;
    if (mc) k_c_marks<<<grid_for(mc), CT, 0, s>>>(c.key[cur], c.val[cur], mc, c.cross, c.multi, c.gref);
    if (int r = launch_exclusive_scan(s, c.cross, c.pos, c.m + 1, c.scan_tmp, c.scan_words)) return r;
    k_c_emit<<<grid_for(c.m), CT, 0, s>>>(c.m, c.eu, c.ev, c.w, c.cmap, c.cross, c.multi, c.pos, c.gref, c.key[cur],
                                          c.val[cur], mc, c.ceu, c.cev, c.cw);
    return (int)cudaGetLastError();
}

}  // namespace lm
