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
// the coarse map and vertex weights; every edge, in input order, gets a 32-bit
// hash of its unordered coarse pair as a key (edges inside a pair the key
// 0xFFFFFFFF; no pair's hash ends in the byte 0xFF, so that they end up last),
// and its coarse endpoints are stored.  A stable LSD radix sort by the low B
// bits of the hash (8-bit passes, as few as leave about 2048 edges to a
// bucket of equal low bits) brings each pair's edges into one bucket, still in
// input order.  Inside each bucket a shared-memory hash table finds the items
// whose full hash repeats; each such run (a group of several edges, or pairs
// whose hashes collide) is put in input order and walked: its groups' first
// edges lead, every later member loses its crossing bit, and a leader of
// several edges records the group's weight summed over its edges in order.
// An edge alone with its hash is alone in its group and leads it.  Buckets,
// runs too long or too mixed for that walk are taken out and sorted again by
// the pair itself.  Prefix counts of the remaining bits (the leaders) give
// each coarse edge its place, and the leaders write the coarse edges.
#include <cstdint>
#include <type_traits>
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

// the unordered coarse pair of an edge as a 64-bit word, min(c, d) << 32 | max(c, d)
__device__ __forceinline__ unsigned long long pair_word(uint32_t c, uint32_t d) {
    return ((unsigned long long)min(c, d) << 32) | max(c, d);
}
// 32-bit hash of a pair word (a 64-bit finaliser's upper half) whose low byte is never
// 0xFF: sorted by any number of low bytes, the pairs come before the edges inside a
// pair (key 0xFFFFFFFF)
__device__ __forceinline__ uint32_t pair_hash(unsigned long long x) {
    x ^= x >> 33;
    x *= 0xFF51AFD7ED558CCDull;
    x ^= x >> 33;
    x *= 0xC4CEB9FE1A85EC53ull;
    x ^= x >> 33;
    const uint32_t h = (uint32_t)(x >> 32);
    return (h & 0xFFu) == 0xFFu ? h ^ 1u : h;
}

// Edge kernels take four consecutive edges per thread (vector loads when the
// arrays are 16-byte aligned) and a warp 128 edges: four whole words of a bitmask
// over the edges, lanes 8q .. 8q+7 sharing word q.
template <bool VEC>
__device__ __forceinline__ uint4 load4(const uint32_t* a, uint64_t i, uint32_t count) {
    if (VEC && i + 4 <= count) return __ldg(reinterpret_cast<const uint4*>(a + i));
    uint4 v;
    v.x = i < count ? a[i] : 0u;
    v.y = i + 1 < count ? a[i + 1] : 0u;
    v.z = i + 2 < count ? a[i + 2] : 0u;
    v.w = i + 3 < count ? a[i + 3] : 0u;
    return v;
}
__device__ __forceinline__ uint32_t at(const uint4& v, int j) { return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w; }

// every edge in input order, keyed by a hash of its unordered coarse pair (equal
// pairs get equal keys); an edge inside a pair (or with an endpoint >= n) gets the
// key 0xFFFFFFFF, above every pair's, so the sort puts it at the end.  Bit e of
// cross: edge e joins two coarse vertices (counted in counts[0]); cpair: the
// coarse endpoints of every edge; hist: each tile's counts of the keys' low byte,
// the sort's first digit.  A warp takes 64 groups of four edges per step, their
// loads issued together.
template <bool VEC>
__global__ void __launch_bounds__(CT) k_c_keys(const uint32_t* __restrict__ eu, const uint32_t* __restrict__ ev,
                                               uint32_t m, uint32_t n, const uint32_t* __restrict__ cmap,
                                               uint32_t* __restrict__ key, uint32_t* __restrict__ cpair,
                                               uint32_t* __restrict__ cross, uint32_t* __restrict__ counts,
                                               uint32_t* __restrict__ hist, uint32_t* __restrict__ err) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t mine = 0;
    // a block takes the 4096 edges of one tile of the sort that follows (1024 groups
    // of four); g0: the warp's first group of a step (a multiple of 64, so of 8)
    for (uint32_t it = 0; it < 2; it++) {
        const uint64_t g0 = (uint64_t)blockIdx.x * 1024 + warp * 128 + it * 64;
        uint4 a[2], b[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const uint64_t e0 = 4 * (g0 + 32 * u + lane);
            a[u] = load4<VEC>(eu, e0, m);
            b[u] = load4<VEC>(ev, e0, m);
        }
        uint32_t cu[2][4], cv[2][4];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const uint64_t e0 = 4 * (g0 + 32 * u + lane);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t x = at(a[u], j), y = at(b[u], j);
                const bool ok = e0 + j < m && x < n && y < n;
                if (e0 + j < m && !ok) atomicOr(err, C_ERR_EDGE);
                cu[u][j] = ok ? cmap[x] : 0u;
                cv[u][j] = ok ? cmap[y] : 0u;
            }
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const uint64_t g = g0 + 32 * u + lane;
            const uint64_t e0 = 4 * g;
            uint32_t nib = 0, k[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                k[j] = 0xFFFFFFFFu;
                if (e0 + j >= m) continue;
                if (cu[u][j] != cv[u][j]) {
                    k[j] = pair_hash(pair_word(cu[u][j], cv[u][j]));
                    nib |= 1u << j;
                }
                atomicAdd(&h[k[j] & 0xFFu], 1u);  // the sort's first digit
            }
            if (e0 + 4 <= m) {  // key and cpair are 16-byte aligned scratch
                *reinterpret_cast<uint4*>(key + e0) = make_uint4(k[0], k[1], k[2], k[3]);
                *reinterpret_cast<uint4*>(cpair + 2 * e0) = make_uint4(cu[u][0], cv[u][0], cu[u][1], cv[u][1]);
                *reinterpret_cast<uint4*>(cpair + 2 * e0 + 4) = make_uint4(cu[u][2], cv[u][2], cu[u][3], cv[u][3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (e0 + j < m) {
                        key[e0 + j] = k[j];
                        cpair[2 * (e0 + j)] = cu[u][j];
                        cpair[2 * (e0 + j) + 1] = cv[u][j];
                    }
            }
            mine += __popc(nib);
            uint32_t w = nib << (4 * (g & 7));
            w |= __shfl_xor_sync(0xFFFFFFFFu, w, 1);
            w |= __shfl_xor_sync(0xFFFFFFFFu, w, 2);
            w |= __shfl_xor_sync(0xFFFFFFFFu, w, 4);
            if ((g & 7) == 0 && e0 < m) cross[g >> 3] = w;
        }
    }
    // one atomic per warp on the count
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, o);
    if (lane == 0 && mine) atomicAdd(&counts[0], mine);
    __syncthreads();
    hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];  // digit-major, as the sort's counts
}

// ---- buckets of the partial hash sort --------------------------------------
// The sort orders the items by the low B bits of their keys only, so a bucket
// (the items sharing those bits) holds every edge of each of its pairs, in input
// order.  A block takes the buckets that start in its chunk of BK_C sorted items.
// It reads a window of BK_W keys from the chunk's first bucket on into registers,
// enters the keys of its buckets in a shared-memory hash table with a count per
// key, and lists the items whose key repeats grouped by key.  Each such run (a
// group of several edges, or pairs whose hashes collide) is put back in input
// order and walked by one thread: with at most GR_PAIRS distinct pairs among at
// most GR_MAX items (the case on simple graphs, where a group has at most four
// edges) it finds the groups in registers -- a group's first edge leads it, every
// later member loses its crossing bit as soon as it is seen, and a leader of
// several edges gets its multi bit and the group's weight summed in double in
// input order once the run is known to fit.  A bucket that runs past the window
// is done in a second window that starts at it.  A bucket longer than a window,
// and any run that does not fit the walk, is flagged in ofl for the general path
// below: taken out in order with its pair as the key and sorted again by the pair
// (which clears the same bits again).
constexpr uint32_t GR_MAX = 64, GR_PAIRS = 4;
constexpr uint32_t BK_T = 512, BK_J = 12, BK_W = BK_T * BK_J, BK_C = 4096, BK_TS = 8192, BK_TS_BITS = 13;
constexpr uint32_t BK_AVG = 2048;  // the sort takes as few bytes as leave at most this many items to a bucket
constexpr uint32_t BK_EMPTY = 0xFFFFFFFFu;
static_assert(BK_TS == 1u << BK_TS_BITS && BK_TS / 16 == BK_T && BK_W < BK_TS && BK_W < 65536 && BK_C < BK_W,
              "table of at most 3/4 load, 16-bit counts and window indices, a chunk shorter than a window");

struct BkSmem {
    union {
        uint32_t tab[BK_TS];    // keys of the table (BK_EMPTY: free), linear probing; then
        uint32_t dl[BK_W];      // items of runs, slot << 16 | window index, grouped by slot
    };
    uint32_t cnt[BK_TS / 2];    // a 16-bit field per slot: its items, then where its run goes in dl
    uint32_t dupb[BK_TS / 32];  // slots whose key repeats
    uint32_t hand[BK_J * (BK_T / 32) + 1];  // each warp's last keys, and the key before the window
    uint32_t wsum[BK_T / 32];
    uint32_t first, lastp1, end, ndup;
};

__device__ __forceinline__ uint32_t bk_slot(uint32_t k) { return (k * 0x9E3779B1u) >> (32 - BK_TS_BITS); }

__device__ __forceinline__ unsigned long long upair(const uint32_t* __restrict__ cpair, uint32_t e) {
    const uint2 p = *reinterpret_cast<const uint2*>(cpair + 2 * (size_t)e);
    return ((unsigned long long)min(p.x, p.y) << 32) | max(p.x, p.y);
}

// One run of dl[i .. i + len) (window indices in input order), items at sorted
// positions ws + index: settled here, or flagged for the general path.
__device__ void bk_walk(const BkSmem& S, uint32_t i, uint32_t len, uint32_t ws, const uint32_t* __restrict__ val,
                        const uint32_t* __restrict__ cpair, const float* __restrict__ w, uint32_t* __restrict__ cross,
                        uint32_t* __restrict__ multi, uint32_t* __restrict__ gsum, uint32_t* __restrict__ ofl,
                        uint32_t* __restrict__ counts) {
    unsigned long long gp[GR_PAIRS];
    uint32_t gl[GR_PAIRS], gn[GR_PAIRS];
    double gs[GR_PAIRS];
    uint32_t ng = 0;
    bool over = len > GR_MAX;
    for (uint32_t j0 = 0; j0 < len && !over; j0 += 4) {
        uint32_t e[4];
        unsigned long long pj[4];
        float wj[4];
#pragma unroll
        for (uint32_t t = 0; t < 4; t++) e[t] = j0 + t < len ? val[ws + (S.dl[i + j0 + t] & 0xFFFFu)] : 0u;
#pragma unroll
        for (uint32_t t = 0; t < 4; t++) {
            pj[t] = j0 + t < len ? upair(cpair, e[t]) : 0ull;
            wj[t] = j0 + t < len ? w[e[t]] : 0.0f;
        }
#pragma unroll
        for (uint32_t t = 0; t < 4; t++) {
            if (j0 + t >= len || over) continue;
            bool found = false;
#pragma unroll
            for (uint32_t g = 0; g < GR_PAIRS; g++)
                if (!found && g < ng && gp[g] == pj[t]) {
                    gs[g] += (double)wj[t];
                    gn[g]++;
                    found = true;
                }
            // a later member of a group: not a leader, whatever the rest of the run
            // holds (a run left to the general path has the same bits cleared there)
            if (found) atomicAnd(&cross[e[t] >> 5], ~(1u << (e[t] & 31)));
            if (!found) {
                if (ng == GR_PAIRS) {
                    over = true;
                } else {
#pragma unroll
                    for (uint32_t g = 0; g < GR_PAIRS; g++)
                        if (g == ng) {
                            gp[g] = pj[t];
                            gl[g] = e[t];
                            gn[g] = 1;
                            gs[g] = (double)wj[t];
                        }
                    ng++;
                }
            }
        }
    }
    if (over) {
        for (uint32_t a = 0; a < len; a++) {
            const uint32_t p = ws + (S.dl[i + a] & 0xFFFFu);
            atomicOr(&ofl[p >> 5], 1u << (p & 31));
        }
        atomicAdd(&counts[1], len);
        return;
    }
#pragma unroll
    for (uint32_t g = 0; g < GR_PAIRS; g++)
        if (g < ng && gn[g] > 1) {
            atomicOr(&multi[gl[g] >> 5], 1u << (gl[g] & 31));
            gsum[gl[g]] = __float_as_uint((float)gs[g]);
        }
}

// key: the sorted keys of the cnt crossing items (sorted by the bits in mask);
// val: their edge indices
__global__ void __launch_bounds__(BK_T, 2)
    k_c_buckets(const uint32_t* __restrict__ key, const uint32_t* __restrict__ val, uint32_t cnt, uint32_t mask,
                const uint32_t* __restrict__ cpair, const float* __restrict__ w, uint32_t* __restrict__ cross,
                uint32_t* __restrict__ multi, uint32_t* __restrict__ gsum, uint32_t* __restrict__ ofl,
                uint32_t* __restrict__ counts) {
    extern __shared__ __align__(16) unsigned char bk_raw[];
    BkSmem& S = *reinterpret_cast<BkSmem*>(bk_raw);
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // (cnt < 2^31: every index below fits in 32 bits)
    const uint32_t c0 = blockIdx.x * BK_C;
    const uint32_t cend = min(cnt, c0 + BK_C);  // this block's buckets start in [c0, cend)
    uint32_t ws = c0;                           // the window: sorted items ws .. ws + BK_W - 1
    for (;;) {
        // item q of the window (thread q % BK_T, slot q / BK_T) ...
        uint32_t k[BK_J];
#pragma unroll
        for (int j = 0; j < (int)BK_J; j++) {
            const uint32_t p = ws + j * BK_T + tid;
            k[j] = p < cnt ? key[p] : BK_EMPTY;
        }
        for (uint32_t i = tid; i < BK_TS / 4; i += BK_T)
            reinterpret_cast<uint4*>(S.tab)[i] = make_uint4(BK_EMPTY, BK_EMPTY, BK_EMPTY, BK_EMPTY);
        for (uint32_t i = tid; i < BK_TS / 8; i += BK_T) reinterpret_cast<uint4*>(S.cnt)[i] = make_uint4(0, 0, 0, 0);
        if (tid == 0) {
            S.first = ~0u;
            S.lastp1 = 0;
            S.end = ~0u;
        }
        // ... starts a bucket when its key's low bits differ from the previous item's:
        // the first and last bucket starts in the chunk, and the first one after it
        // (each warp's last lane hands its keys to the next warp's first lane)
        const uint32_t chunk_q = cend > ws ? cend - ws : 0u;
        if (lane == 31)
#pragma unroll
            for (int j = 0; j < (int)BK_J; j++) S.hand[j * (BK_T / 32) + warp] = k[j];
        if (tid == 0) S.hand[BK_J * (BK_T / 32)] = ws > 0 ? key[ws - 1] : 0u;
        __syncthreads();
        uint32_t f = ~0u, l = 0, e = ~0u;
#pragma unroll
        for (int j = 0; j < (int)BK_J; j++) {
            const uint32_t q = j * BK_T + tid;
            const uint32_t p = ws + q;
            uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, k[j], 1);
            if (lane == 0)
                prev = S.hand[warp > 0 ? j * (BK_T / 32) + warp - 1 : j > 0 ? j * (BK_T / 32) - 1 : BK_J * (BK_T / 32)];
            if (p < cnt && (p == 0 || ((k[j] ^ prev) & mask) != 0)) {
                if (q < chunk_q) {
                    f = min(f, q);
                    l = max(l, q + 1);
                } else {
                    e = min(e, q);
                }
            }
        }
        f = __reduce_min_sync(0xFFFFFFFFu, f);
        l = __reduce_max_sync(0xFFFFFFFFu, l);
        e = __reduce_min_sync(0xFFFFFFFFu, e);
        if (lane == 0) {
            if (f != ~0u) atomicMin(&S.first, f);
            if (l) atomicMax(&S.lastp1, l);
            if (e != ~0u) atomicMin(&S.end, e);
        }
        __syncthreads();
        const uint32_t s = S.first, last = S.lastp1 - 1u;
        uint32_t end = S.end;
        if (ws + BK_W >= cnt) end = min(end, cnt - ws);
        if (s == ~0u) return;  // no bucket starts in this block's chunk
        // the buckets done in this window: [lo, hi)
        uint32_t lo = s, hi = s;
        bool again = false;
        if (end != ~0u) {
            hi = end;
        } else if (last > s) {
            hi = last;  // the last one runs past the window: a window of its own
            again = true;
        } else if (s > 0) {
            again = true;  // the only one runs past the window: a window of its own
        } else {
            // a bucket longer than a window: all of it to the general path
            const uint32_t bv = key[ws] & mask;
            uint32_t mine = 0;
            for (uint32_t p = ws + tid;; p += BK_T) {
                const bool in = p < cnt && (key[p] & mask) == bv;
                if (!__syncthreads_or(in)) break;
                if (in) {
                    atomicOr(&ofl[p >> 5], 1u << (p & 31));
                    mine++;
                }
            }
            mine = __reduce_add_sync(0xFFFFFFFFu, mine);
            if (lane == 0 && mine) atomicAdd(&counts[1], mine);
            return;
        }
        // every item of [lo, hi) into the table; its slot kept in 16 bits of sp
        uint32_t sp[BK_J / 2];
#pragma unroll
        for (int j = 0; j < (int)BK_J; j++) {
            const uint32_t q = j * BK_T + tid;
            uint32_t sl = 0;
            if (q >= lo && q < hi) {
                sl = bk_slot(k[j]);
                // (at most BK_W < BK_TS keys: a free slot or the key is always found)
                for (uint32_t probe = 0; probe < BK_TS; probe++) {
                    const uint32_t old = atomicCAS(&S.tab[sl], BK_EMPTY, k[j]);
                    if (old == BK_EMPTY || old == k[j]) break;
                    sl = (sl + 1) & (BK_TS - 1);
                }
                atomicAdd(&S.cnt[sl >> 1], 1u << (16 * (sl & 1)));
            }
            if (j & 1) sp[j >> 1] |= sl << 16;
            else sp[j >> 1] = sl;
        }
        __syncthreads();
        // slots of two or more items, and where each one's run starts in dl (thread t:
        // slots 16 t .. 16 t + 15, cnt words 8 t .. 8 t + 7)
        {
            uint4* cq = reinterpret_cast<uint4*>(S.cnt) + 2 * tid;
            uint32_t tot = 0, bits = 0;
#pragma unroll
            for (int v = 0; v < 2; v++) {
                const uint4 x = cq[v];
                const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int h = 0; h < 8; h++) {
                    const uint32_t c = (wv[h >> 1] >> (16 * (h & 1))) & 0xFFFFu;
                    if (c >= 2) {
                        tot += c;
                        bits |= 1u << (8 * v + h);
                    }
                }
            }
            uint32_t x = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= (uint32_t)o) x += y;
            }
            if (lane == 31) S.wsum[warp] = x;
            __syncthreads();
            uint32_t run = x - tot;
            for (uint32_t v = 0; v < warp; v++) run += S.wsum[v];
#pragma unroll
            for (int v = 0; v < 2; v++) {
                if (!((bits >> (8 * v)) & 0xFFu)) continue;
                const uint4 x4 = cq[v];
                uint32_t wv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int h = 0; h < 8; h++) {
                    if (!((bits >> (8 * v + h)) & 1u)) continue;
                    const uint32_t sh = 16 * (h & 1);
                    const uint32_t c = (wv[h >> 1] >> sh) & 0xFFFFu;
                    wv[h >> 1] = (wv[h >> 1] & ~(0xFFFFu << sh)) | (run << sh);
                    run += c;
                }
                cq[v] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
            reinterpret_cast<uint16_t*>(S.dupb)[tid] = (uint16_t)bits;  // bit 16 t + h: slot 16 t + h
            if (tid == BK_T - 1) S.ndup = run;
        }
        __syncthreads();
        // the items of repeated keys into dl, grouped by slot
#pragma unroll
        for (int j = 0; j < (int)BK_J; j++) {
            const uint32_t q = j * BK_T + tid;
            if (q >= lo && q < hi) {
                const uint32_t sl = (sp[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
                if ((S.dupb[sl >> 5] >> (sl & 31)) & 1u) {
                    const uint32_t sh = 16 * (sl & 1);
                    const uint32_t pos = (atomicAdd(&S.cnt[sl >> 1], 1u << sh) >> sh) & 0xFFFFu;
                    S.dl[pos] = (sl << 16) | q;
                }
            }
        }
        __syncthreads();
        // each run by the thread that holds its first entry: back in input order
        // (insertion sort on the window index; its entries share their slot bits, which
        // is all that other threads read of them), then walked
        const uint32_t nd = S.ndup;
        for (uint32_t i = tid; i < nd; i += BK_T) {
            const uint32_t sl = S.dl[i] >> 16;
            if (i > 0 && (S.dl[i - 1] >> 16) == sl) continue;
            uint32_t len = 1;
            while (i + len < nd && (S.dl[i + len] >> 16) == sl) len++;
            if (len <= GR_MAX)
                for (uint32_t a = 1; a < len; a++) {
                    const uint32_t y = S.dl[i + a];
                    uint32_t b = a;
                    for (; b > 0 && S.dl[i + b - 1] > y; b--) S.dl[i + b] = S.dl[i + b - 1];
                    S.dl[i + b] = y;
                }
            bk_walk(S, i, len, ws, val, cpair, w, cross, multi, gsum, ofl, counts);
        }
        if (!again) return;
        __syncthreads();  // (dl and the table are free again)
        ws += hi > s ? hi : s;
    }
}

// The general path: the flagged items, a tile of 4096 per block, thread t holding
// chunks c = 0..3 of four items at tile offset 1024 c + 4 t.  One launch counts
// them per tile; after a scan of the counts the second takes them out in order.
constexpr uint32_t RN_TILE = 4096;

// bit j: item i + j is flagged (i a multiple of 4)
__device__ __forceinline__ uint32_t run_bits(const uint32_t* __restrict__ ofl, uint64_t i, uint32_t cnt) {
    return i < cnt ? (ofl[i >> 5] >> (i & 31)) & 0xFu : 0u;
}

__global__ void __launch_bounds__(CT) k_c_runs_count(const uint32_t* __restrict__ ofl, uint32_t cnt,
                                                     uint32_t* __restrict__ tcount) {
    __shared__ uint32_t ws[CT / 32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * RN_TILE + 4 * threadIdx.x;
    uint32_t x = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) x += __popc(run_bits(ofl, base + 1024 * c, cnt));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if (lane == 0) ws[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)(CT / 32); w++) t += ws[w];
        tcount[blockIdx.x] = t;
    }
}

// the flagged items in sorted order (so a pair's edges keep their input order), with
// (min, max) of their coarse pair as the key of a second sort; counts[3] = how many.
// The tile's run items are listed in shared memory first, so that the gathers of
// their pairs spread over all threads.
__global__ void __launch_bounds__(CT) k_c_runs_take(const uint32_t* __restrict__ ofl, const uint32_t* __restrict__ val,
                                                    uint32_t cnt, const uint32_t* __restrict__ toffs,
                                                    const uint32_t* __restrict__ cpair, uint32_t bits,
                                                    unsigned long long* __restrict__ skey,
                                                    uint32_t* __restrict__ sval, uint32_t* __restrict__ counts) {
    __shared__ uint32_t ws[4][CT / 32];
    __shared__ uint32_t list[RN_TILE];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t tile0 = (uint64_t)blockIdx.x * RN_TILE;
    const uint64_t base = tile0 + 4 * threadIdx.x;
    uint32_t f[4], incl[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        f[c] = run_bits(ofl, base + 1024 * c, cnt);
        uint32_t x = __popc(f[c]);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        incl[c] = x;
        if (lane == 31) ws[c][warp] = x;
    }
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        uint32_t before = 0, total = 0;
        for (uint32_t w = 0; w < CT / 32; w++) {
            before += w < warp ? ws[c][w] : 0u;
            total += ws[c][w];
        }
        uint32_t q = run + before + incl[c] - __popc(f[c]);
        for (uint32_t bl = f[c]; bl; bl &= bl - 1) list[q++] = 1024 * c + 4 * threadIdx.x + __ffs(bl) - 1;
        run += total;
    }
    __syncthreads();
    const uint32_t off = toffs[blockIdx.x];
    for (uint32_t q = threadIdx.x; q < run; q += CT) {
        const uint32_t e = val[tile0 + list[q]];
        const uint2 cp = *reinterpret_cast<const uint2*>(cpair + 2 * (size_t)e);
        const uint32_t x = cp.x, y = cp.y;
        skey[off + q] = ((unsigned long long)min(x, y) << bits) | max(x, y);  // coarse ids take `bits` bits
        sval[off + q] = e;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) counts[3] = off + run;
}

// ---- stable LSD radix sort of (key, value) pairs, 8 bits per pass ----------
// A pass is three launches.  The first counts each tile's digits; an exclusive
// scan over (digit, tile) then gives every tile the output position of its first
// item of each digit; the third ranks each tile's items stably (warp by warp, 32
// items at a time in input order: lanes with the same digit from one ballot per
// digit bit, earlier rounds and warps by shared counters), puts the tile in digit
// order in shared memory and writes it out.  No block waits on another.
constexpr uint32_t RS_T = 256, RS_I = 16, RS_TILE = RS_T * RS_I, RS_W = RS_T / 32;

template <class K>
struct RsSmem {
    uint32_t wcnt[RS_W][256];  // items of each digit seen so far by each warp, then where the warp's start
    uint32_t gofs[256];        // output position of the tile's first item of each digit, minus its tile start
    uint32_t wsum[RS_W];
    K sk[RS_TILE];
    uint32_t sv[RS_TILE];
};

// digit counts of every tile, digit-major (hist[d * tiles + t]) for the scan
template <class K>
__global__ void __launch_bounds__(RS_T) k_rs_hist(const K* __restrict__ key, uint32_t cnt, uint32_t shift,
                                                  uint32_t tiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RS_W][256];
    for (uint32_t i = threadIdx.x; i < RS_W * 256; i += RS_T) (&h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t base = blockIdx.x * RS_TILE + threadIdx.x;
    K k[RS_I];
#pragma unroll
    for (int j = 0; j < (int)RS_I; j++) {
        const uint32_t q = base + j * RS_T;
        k[j] = q < cnt ? key[q] : (K)0;
    }
#pragma unroll
    for (int j = 0; j < (int)RS_I; j++)
        if (base + j * RS_T < cnt) atomicAdd(&h[warp][(uint32_t)(k[j] >> shift) & 0xFFu], 1u);
    __syncthreads();
    uint32_t x = 0;
#pragma unroll
    for (int w = 0; w < (int)RS_W; w++) x += h[w][threadIdx.x];
    hist[threadIdx.x * tiles + blockIdx.x] = x;
}

// val_in NULL: the values are the items' indices
template <class K>
__global__ void __launch_bounds__(RS_T, sizeof(K) == 4 ? 3 : 2)
    k_rs_scatter(const K* __restrict__ key_in, const uint32_t* __restrict__ val_in, uint32_t cnt, uint32_t shift,
                 uint32_t tiles, const uint32_t* __restrict__ offs, K* __restrict__ key_out,
                 uint32_t* __restrict__ val_out) {
    extern __shared__ __align__(16) unsigned char rs_raw[];
    RsSmem<K>& S = *reinterpret_cast<RsSmem<K>*>(rs_raw);
    auto& wcnt = S.wcnt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t tile = blockIdx.x, dg = threadIdx.x;  // (one digit per thread below)
    const uint32_t gstart = offs[dg * tiles + tile];
    for (uint32_t i = threadIdx.x; i < RS_W * 256; i += RS_T) (&wcnt[0][0])[i] = 0;
    // warp w owns items [w * 32 RS_I, (w + 1) * 32 RS_I) of the tile, 32 per round in order
    const uint32_t tile0 = tile * RS_TILE;
    const uint32_t base = tile0 + warp * 32 * RS_I;
    const uint32_t nin = cnt > tile0 ? min(RS_TILE, cnt - tile0) : 0u;
    K k[RS_I];
    uint32_t v[RS_I], r[RS_I];
#pragma unroll
    for (int j = 0; j < (int)RS_I; j++) {
        const uint32_t q = base + j * 32 + lane;
        const bool ok = q < cnt;
        k[j] = ok ? key_in[q] : (K)0;
        v[j] = ok ? (val_in ? val_in[q] : q) : 0u;  // no values: each item's own index
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < (int)RS_I; j++) {
        const bool ok = base + j * 32 + lane < cnt;
        const uint32_t d = (uint32_t)(k[j] >> shift) & 0xFFu;
        // the lanes holding the same digit, from one ballot per digit bit (lanes past
        // the end match nobody)
        uint32_t peers = __ballot_sync(0xFFFFFFFFu, ok);
#pragma unroll
        for (int b = 0; b < 8; b++) {
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
        // the whole warp reads, then each digit's last lane writes: no branch splits
        // the warp by digit
        const uint32_t before = ok ? wcnt[warp][d] : 0u;
        r[j] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers >> lane) == 1u) wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        uint32_t run = 0;
        for (int w = 0; w < (int)RS_W; w++) run += wcnt[w][dg];
        // exclusive scan of the 256 digit totals across the tile
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) S.wsum[warp] = x;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; w++) before += S.wsum[w];
        const uint32_t dst = before + x - run;
        uint32_t acc = dst;
        for (int w = 0; w < (int)RS_W; w++) {
            const uint32_t c = wcnt[w][dg];
            wcnt[w][dg] = acc;
            acc += c;
        }
        S.gofs[dg] = gstart - dst;
    }
    __syncthreads();
    // the tile in digit order in shared memory ...
#pragma unroll
    for (int j = 0; j < (int)RS_I; j++) {
        if (base + j * 32 + lane >= cnt) continue;
        const uint32_t p = wcnt[warp][(uint32_t)(k[j] >> shift) & 0xFFu] + r[j];
        S.sk[p] = k[j];
        S.sv[p] = v[j];
    }
    __syncthreads();
    // ... then written out: consecutive threads take consecutive items, which within
    // a digit land on consecutive addresses
    for (uint32_t p = threadIdx.x; p < nin; p += RS_T) {
        const K kk = S.sk[p];
        const uint32_t o = S.gofs[(uint32_t)(kk >> shift) & 0xFFu] + p;
        if (o < cnt) {
            key_out[o] = kk;
            val_out[o] = S.sv[p];
        }
    }
}

// groups in pair order (runs of equal keys; a run's first item is its leader, the
// smallest edge index, since the sort is stable and a pair's edges entered in
// input order).  Every other member loses its bit in cross; the leader of a
// group of several edges gets a bit in multi and, in gsum, the float32 bits of
// the group's weight: the sum in double over its edges in input order, rounded once.
__global__ void k_c_marks(const unsigned long long* __restrict__ key, const uint32_t* __restrict__ val, uint32_t cnt,
                          const float* __restrict__ w, uint32_t* __restrict__ cross, uint32_t* __restrict__ multi,
                          uint32_t* __restrict__ gsum) {
    for (uint32_t i = blockIdx.x * CT + threadIdx.x; i < cnt; i += gridDim.x * CT) {
        const unsigned long long k = key[i];
        const uint32_t e = val[i];
        if (i > 0 && k == key[i - 1]) {
            atomicAnd(&cross[e >> 5], ~(1u << (e & 31)));
        } else if (i + 1 < cnt && key[i + 1] == k) {
            double sum = (double)w[e];
            uint32_t j = i + 1;
            // members four at a time: their loads issue together, the additions stay in order
            for (bool more = true; more;) {
                uint32_t vj[4];
                bool in[4];
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    in[t] = j + t < cnt && key[j + t] == k;
                    vj[t] = in[t] ? val[j + t] : 0u;
                }
                float wj[4];
#pragma unroll
                for (int t = 0; t < 4; t++) wj[t] = in[t] ? w[vj[t]] : 0.0f;
#pragma unroll
                for (int t = 0; t < 4; t++)
                    if (in[t]) sum += (double)wj[t];
                more = in[3];
                j += 4;
            }
            atomicOr(&multi[e >> 5], 1u << (e & 31));
            gsum[e] = __float_as_uint((float)sum);
        }
    }
}

// leaders per word of cross (wlead[words] = 0, so that the scan's last entry is the total)
__global__ void k_c_wcount(const uint32_t* __restrict__ cross, uint32_t words, uint32_t* __restrict__ wlead) {
    for (uint32_t i = blockIdx.x * CT + threadIdx.x; i <= words; i += gridDim.x * CT)
        wlead[i] = i < words ? __popc(cross[i]) : 0u;
}

// the leaders, in input order, write their coarse edge at their rank among the
// leaders, with their group's weight (a single edge's own weight, which double and
// back leaves unchanged)
template <bool VEC>
__global__ void __launch_bounds__(CT) k_c_emit(uint32_t m, const uint32_t* __restrict__ cpair,
                                               const float* __restrict__ w, const uint32_t* __restrict__ cross,
                                               const uint32_t* __restrict__ wpos, const uint32_t* __restrict__ multi,
                                               const uint32_t* __restrict__ gsum, uint32_t* __restrict__ ceu,
                                               uint32_t* __restrict__ cev, float* __restrict__ cw) {
    // a block takes 1024 edges (32 words of cross) at a time; their leaders fill one
    // run of the output, staged here and written out contiguously
    __shared__ uint32_t su[4 * CT], sv2[4 * CT], sw[4 * CT];
    const uint32_t groups = (uint32_t)(((uint64_t)m + 3) / 4);
    const uint32_t words = (uint32_t)(((uint64_t)m + 31) / 32);
    const uint32_t* wb = reinterpret_cast<const uint32_t*>(w);
    for (uint32_t c0 = blockIdx.x * CT; c0 < groups; c0 += gridDim.x * CT) {
        const uint32_t g = c0 + threadIdx.x;
        const uint32_t w0 = c0 >> 3, w1 = min(w0 + CT / 8, words);
        const uint32_t obase = wpos[w0], ocount = wpos[w1] - obase;
        if (g < groups) {
            const uint64_t e0 = 4ull * g;
            // every load of the group at once (most edges lead); cpair is aligned scratch
            const uint32_t word = cross[g >> 3], wp = wpos[g >> 3], mw = __ldg(&multi[g >> 3]);
            const uint4 x = load4<VEC>(wb, e0, m);
            const uint4 p0 = load4<true>(cpair, 2 * e0, 2 * m), p1 = load4<true>(cpair, 2 * e0 + 4, 2 * m);
            const uint32_t sh = 4 * (g & 7);
            const uint32_t nib = (word >> sh) & 0xFu, mb = (mw >> sh) & 0xFu;
            uint32_t p = wp - obase + __popc(word & ((1u << sh) - 1u));
            const uint32_t cu[4] = {p0.x, p0.z, p1.x, p1.z}, cv[4] = {p0.y, p0.w, p1.y, p1.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (!((nib >> j) & 1u)) continue;
                su[p] = cu[j];
                sv2[p] = cv[j];
                sw[p] = ((mb >> j) & 1u) ? gsum[(uint32_t)e0 + j] : at(x, j);
                p++;
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < ocount; i += CT) {
            ceu[obase + i] = su[i];
            cev[obase + i] = sv2[i];
            cw[obase + i] = __uint_as_float(sw[i]);
        }
        __syncthreads();
    }
}

uint32_t bits_for(uint32_t x) {  // bits to write 0 .. x
    uint32_t b = 1;
    while (b < 32 && (x >> b)) b++;
    return b;
}

}  // namespace

size_t contract_sort_words(uint32_t m) {
    const uint64_t tiles = ((uint64_t)m + RS_TILE - 1) / RS_TILE;
    return (size_t)(2 * (256 * tiles + 4));
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
    if ((e = cudaFuncSetAttribute(k_rs_scatter<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(RsSmem<uint32_t>)))) return (int)e;
    if ((e = cudaFuncSetAttribute(k_rs_scatter<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sizeof(RsSmem<unsigned long long>)))) return (int)e;
    // stable sort by the low `bits` bits of the keys (8-bit digits), ping-ponging
    // between the two buffers; *cur tells which holds the result
    // (ident: the values are the items' indices, and v0 is not read)
    // (counted0: the first pass's per-tile digit counts are in place already)
    auto radix = [&](auto* k0, auto* k1, uint32_t* v0, uint32_t* v1, uint32_t cnt, uint32_t bits, bool ident,
                     bool counted0, int* cur) -> int {
        using K = typename std::remove_pointer<decltype(k0)>::type;
        K* kk[2] = {k0, k1};
        uint32_t* vv[2] = {v0, v1};
        *cur = 0;
        if (cnt < 2) return 0;
        const uint32_t tiles = (cnt + RS_TILE - 1) / RS_TILE;
        uint32_t* hist = c.shist;
        uint32_t* offs = c.shist + ((256 * (size_t)tiles + 4) & ~(size_t)3);
        for (uint32_t p = 0; p * 8 < bits; p++) {
            if (!(counted0 && p == 0)) k_rs_hist<K><<<tiles, RS_T, 0, s>>>(kk[*cur], cnt, 8 * p, tiles, hist);
            if (int r = launch_exclusive_scan(s, hist, offs, 256 * tiles, c.scan_tmp, c.scan_words)) return r;
            const uint32_t* vin = (ident && p == 0) ? nullptr : vv[*cur];
            k_rs_scatter<K><<<tiles, RS_T, sizeof(RsSmem<K>), s>>>(kk[*cur], vin, cnt, 8 * p, tiles, offs,
                                                                   kk[*cur ^ 1], vv[*cur ^ 1]);
            *cur ^= 1;
        }
        return (int)cudaGetLastError();
    };
    // 1. every edge keyed by its pair's hash in input order; the stable sort keeps input
    //    order among equal keys and puts the edges inside pairs last, after the mc crossing edges
    uint32_t* hk[2] = {reinterpret_cast<uint32_t*>(c.key[0]), reinterpret_cast<uint32_t*>(c.key[1])};
    const uint32_t words = (uint32_t)(((uint64_t)c.m + 31) / 32);
    const uint32_t egrid = grid_for(((uint64_t)c.m + 3) / 4);
    const bool vec = ((reinterpret_cast<uintptr_t>(c.eu) | reinterpret_cast<uintptr_t>(c.ev) |
                       reinterpret_cast<uintptr_t>(c.w)) & 15u) == 0;
    if ((e = cudaMemsetAsync(c.counts, 0, 8 * sizeof(uint32_t), s))) return (int)e;
    static_assert(RS_TILE == 4096 && CT == 256, "k_c_keys takes one tile of the sort per block");
    const uint32_t kgrid = (uint32_t)(((uint64_t)c.m + RS_TILE - 1) / RS_TILE);  // the sort's tiles
    if (vec)
        k_c_keys<true><<<kgrid, CT, 0, s>>>(c.eu, c.ev, c.m, c.n, c.cmap, hk[0], c.cpair, c.cross, c.counts, c.shist,
                                            c.err);
    else
        k_c_keys<false><<<kgrid, CT, 0, s>>>(c.eu, c.ev, c.m, c.n, c.cmap, hk[0], c.cpair, c.cross, c.counts, c.shist,
                                             c.err);
    if ((e = cudaMemcpyAsync(mc_host_slot, c.counts, sizeof(uint32_t), cudaMemcpyDeviceToHost, s))) return (int)e;
    if ((e = cudaMemcpyAsync(mc_host_slot + 1, c.rank + c.n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s))) return (int)e;
    if ((e = cudaStreamSynchronize(s))) return (int)e;
    const uint32_t mc = mc_host_slot[0], nc = mc_host_slot[1];
    // the sort's bits: as few bytes as leave at most BK_AVG crossing edges to a bucket
    uint32_t sbits = c.sort_bits;
    if (!sbits)
        for (sbits = 8; sbits < 32 && (uint64_t)mc > ((uint64_t)BK_AVG << sbits); sbits += 8) {
        }
    const uint32_t mask = sbits >= 32 ? ~0u : (1u << sbits) - 1u;
    int hc = 0;
    if (mc > 1)
        if (int r = radix(hk[0], hk[1], c.val[0], c.val[1], c.m, sbits, true, true, &hc)) return r;
    // 2. runs of equal hash (groups of several edges, and collisions): the crossing bits
    //    become the leader bits, every group member but the first cleared.  Runs with
    //    few pairs are settled by k_c_buckets; the rest are taken out in sorted order
    //    with their pair as the key, sorted again by the pair and marked.
    if ((e = cudaMemsetAsync(c.multi, 0, ((size_t)c.m / 32 + 2) * sizeof(uint32_t), s))) return (int)e;
    uint32_t nsub = 0;
    const uint32_t bits = bits_for(nc ? nc - 1 : 0);
    uint32_t* ofl = c.wlead;  // (free until the leaders are counted)
    if (mc > 1) {
        if ((e = cudaMemsetAsync(ofl, 0, ((size_t)mc / 32 + 2) * sizeof(uint32_t), s))) return (int)e;
        if ((e = cudaFuncSetAttribute(k_c_buckets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BkSmem))))
            return (int)e;
        if ((e = cudaFuncSetAttribute(k_c_buckets, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared)))
            return (int)e;
        k_c_buckets<<<(mc + BK_C - 1) / BK_C, BK_T, sizeof(BkSmem), s>>>(hk[hc], c.val[hc], mc, mask, c.cpair, c.w,
                                                                       c.cross, c.multi, c.gref, ofl, c.counts);
        if ((e = cudaMemcpyAsync(mc_host_slot + 2, c.counts + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)))
            return (int)e;
        if ((e = cudaStreamSynchronize(s))) return (int)e;
        if (mc_host_slot[2]) {
            const uint32_t tiles = (mc + RN_TILE - 1) / RN_TILE;
            uint32_t* toffs = c.tsum + ((size_t)c.m / RN_TILE + 2);
            k_c_runs_count<<<tiles, CT, 0, s>>>(ofl, mc, c.tsum);
            if (int r = launch_exclusive_scan(s, c.tsum, toffs, tiles, c.scan_tmp, c.scan_words)) return r;
            k_c_runs_take<<<tiles, CT, 0, s>>>(ofl, c.val[hc], mc, toffs, c.cpair, bits, c.key[hc ^ 1],
                                               c.val[hc ^ 1], c.counts);
            if ((e = cudaMemcpyAsync(mc_host_slot + 2, c.counts + 3, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)))
                return (int)e;
            if ((e = cudaStreamSynchronize(s))) return (int)e;
            nsub = mc_host_slot[2];
        }
    }
    // the subset's two buffers: the ones the hash sort did not end in, and, once the
    // subset is taken out, the ones it did
    unsigned long long* sk[2] = {c.key[hc ^ 1], c.key[hc]};
    uint32_t* sv[2] = {c.val[hc ^ 1], c.val[hc]};
    int cur = 0;
    if (nsub) {
        if (int r = radix(sk[0], sk[1], sv[0], sv[1], nsub, 2 * bits, false, false, &cur)) return r;
        k_c_marks<<<grid_for(nsub), CT, 0, s>>>(sk[cur], sv[cur], nsub, c.w, c.cross, c.multi, c.gref);
    }
    // 4. leaders ranked by words of the bitmask; the leaders write the coarse edges
    k_c_wcount<<<grid_for((uint64_t)words + 1), CT, 0, s>>>(c.cross, words, c.wlead);
    if (int r = launch_exclusive_scan(s, c.wlead, c.wpos, words + 1, c.scan_tmp, c.scan_words)) return r;
    if ((e = cudaMemcpyAsync(c.counts + 2, c.wpos + words, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)))
        return (int)e;
    if (mc) {
        if (vec)
            k_c_emit<true><<<egrid, CT, 0, s>>>(c.m, c.cpair, c.w, c.cross, c.wpos, c.multi, c.gref, c.ceu, c.cev,
                                                c.cw);
        else
            k_c_emit<false><<<egrid, CT, 0, s>>>(c.m, c.cpair, c.w, c.cross, c.wpos, c.multi, c.gref, c.ceu, c.cev,
                                                 c.cw);
    }
    return (int)cudaGetLastError();
}

}  // namespace lm
