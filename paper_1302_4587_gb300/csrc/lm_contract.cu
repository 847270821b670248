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
// the coarse map and vertex weights; the crossing edges, compacted in input
// order, get their unordered coarse pair as a key; a stable LSD radix sort
// (8-bit digits over the key's significant bits) groups equal pairs with their
// edges still in input order; each group's first edge is its leader and the
// group's weight sum is taken over its edges in order; leader flags over the
// edges and their prefix ranks give each coarse edge its place; the leaders
// write the coarse edges.
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

// crossing[e] = 1 when the edge joins two coarse vertices (endpoints validated)
__global__ void k_c_cross(const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev, uint32_t m, uint32_t n,
                          const uint32_t* __restrict__ cmap, uint32_t* __restrict__ cross, uint32_t* __restrict__ err) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        const uint32_t a = eu[e], b = ev[e];
        uint32_t x = 0;
        if (a >= n || b >= n) atomicOr(err, C_ERR_EDGE);
        else x = cmap[a] != cmap[b] ? 1u : 0u;
        cross[e] = x;
    }
}

// the crossing edges in input order: key = min(c, d) << bits | max(c, d), value = e
__global__ void k_c_keys(const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev, uint32_t m,
                         const uint32_t* __restrict__ cmap, const uint32_t* __restrict__ cross,
                         const uint32_t* __restrict__ cpos, uint32_t bits, unsigned long long* __restrict__ key,
                         uint32_t* __restrict__ val) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        if (!cross[e]) continue;
        const uint32_t c = cmap[eu[e]], d = cmap[ev[e]];
        const uint32_t p = cpos[e];
        key[p] = ((unsigned long long)min(c, d) << bits) | max(c, d);
        val[p] = e;
    }
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

// group heads in sorted order: the first item of every run of equal keys; the
// head's value is the group's leader (the smallest edge index: the sort is
// stable and the items entered in input order)
__global__ void k_c_heads(const unsigned long long* __restrict__ key, const uint32_t* __restrict__ val, uint32_t cnt,
                          uint32_t* __restrict__ isl, uint32_t* __restrict__ gref) {
    for (uint32_t i = blockIdx.x * CT + threadIdx.x; i < cnt; i += gridDim.x * CT) {
        if (i > 0 && key[i] == key[i - 1]) continue;
        const uint32_t e = val[i];
        isl[e] = 1u;
        gref[e] = i;
    }
}

// the leaders write their coarse edge at their rank among the leaders; the weight
// is the group's sum over its edges in input order
__global__ void k_c_emit(uint32_t m, const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                         const float* __restrict__ w, const uint32_t* __restrict__ cmap,
                         const uint32_t* __restrict__ isl, const uint32_t* __restrict__ pos,
                         const uint32_t* __restrict__ gref, const unsigned long long* __restrict__ key,
                         const uint32_t* __restrict__ val, uint32_t cnt, uint32_t* __restrict__ ceu,
                         uint32_t* __restrict__ cev, float* __restrict__ cw) {
    for (uint32_t e = blockIdx.x * CT + threadIdx.x; e < m; e += gridDim.x * CT) {
        if (!isl[e]) continue;
        const uint32_t p = pos[e], i0 = gref[e];
        const unsigned long long k = key[i0];
        double sum = 0.0;
        for (uint32_t i = i0; i < cnt && key[i] == k; i++) sum += (double)w[val[i]];
        ceu[p] = cmap[eu[e]];
        cev[p] = cmap[ev[e]];
        cw[p] = (float)sum;
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
    // crossing edges compacted in input order
    if ((e = cudaMemsetAsync(c.cross + c.m, 0, sizeof(uint32_t), s))) return (int)e;
    k_c_cross<<<grid_for(c.m), CT, 0, s>>>(c.eu, c.ev, c.m, c.n, c.cmap, c.cross, c.err);
    if (int r = launch_exclusive_scan(s, c.cross, c.cpos, c.m + 1, c.scan_tmp, c.scan_words)) return r;
    // the crossing count decides the sort's size: read it on the host
    if ((e = cudaMemcpyAsync(mc_host_slot, c.cpos + c.m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s))) return (int)e;
    if ((e = cudaMemcpyAsync(mc_host_slot + 1, c.rank + c.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s))) return (int)e;
    if ((e = cudaStreamSynchronize(s))) return (int)e;
    const uint32_t mc = mc_host_slot[0], nc = mc_host_slot[1];
    const uint32_t bits = bits_for(nc ? nc - 1 : 0);
    k_c_keys<<<grid_for(c.m), CT, 0, s>>>(c.eu, c.ev, c.m, c.cmap, c.cross, c.cpos, bits, c.key[0], c.val[0]);
    // radix passes over the key's 2 * bits significant bits
    int cur = 0;
    if (mc > 1) {
        const uint32_t nblk = (mc + RS_TILE - 1) / RS_TILE;
        for (uint32_t shift = 0; shift < 2 * bits; shift += 8) {
            k_rs_hist<<<nblk, RS_T, 0, s>>>(c.key[cur], mc, shift, nblk, c.hist);
            if (int r = launch_exclusive_scan(s, c.hist, c.hoff, 256 * nblk, c.scan_tmp, c.scan_words)) return r;
            k_rs_scatter<<<nblk, RS_T, 0, s>>>(c.key[cur], c.val[cur], mc, shift, nblk, c.hoff, c.key[cur ^ 1],
                                               c.val[cur ^ 1]);
            cur ^= 1;
        }
    }
    if ((e = cudaMemsetAsync(c.isl, 0, ((size_t)c.m + 1) * sizeof(uint32_t), s))) return (int)e;
    if (mc) k_c_heads<<<grid_for(mc), CT, 0, s>>>(c.key[cur], c.val[cur], mc, c.isl, c.gref);
    if (int r = launch_exclusive_scan(s, c.isl, c.pos, c.m + 1, c.scan_tmp, c.scan_words)) return r;
    k_c_emit<<<grid_for(c.m), CT, 0, s>>>(c.m, c.eu, c.ev, c.w, c.cmap, c.isl, c.pos, c.gref, c.key[cur], c.val[cur],
                                          mc, c.ceu, c.cev, c.cw);
    return (int)cudaGetLastError();
}

}  // namespace lm
