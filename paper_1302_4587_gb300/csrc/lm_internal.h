// Internal declarations shared by the kernels (lm_kernels.cu) and the host
// driver (lm_api.cpp).  Not part of the public ABI (include/lm.h is).
#pragma once
#include <stdint.h>
#include <stddef.h>

#if defined(__CUDACC__)
#define LM_HD __host__ __device__ __forceinline__
#else
#define LM_HD inline
#endif

namespace lm {

constexpr uint32_t NIL = 0xFFFFFFFFu;

// One sweep tile = SWEEP_T consecutive adjacency entries, processed by one
// CTA of SWEEP_THREADS threads (each warp owns SWEEP_T / 32 / warps groups of
// 32 consecutive entries).
constexpr int SWEEP_T = 2048;
constexpr int SWEEP_THREADS = 256;
constexpr int SWEEP_WARPS = SWEEP_THREADS / 32;
constexpr int SWEEP_GROUPS = SWEEP_T / 32;              // 64
constexpr int SWEEP_GPW = SWEEP_GROUPS / SWEEP_WARPS;   // 8 groups per warp
constexpr int SWEEP_RPT = (SWEEP_T + 1 + SWEEP_THREADS - 1) / SWEEP_THREADS; // rows per thread in row scans

// error bits written to DevState::err by kernels
constexpr uint32_t ERR_TIMEOUT = 1u;    // look-back wait gave up
constexpr uint32_t ERR_BOUNDS = 2u;     // an index check failed (row / position / vertex)
constexpr uint32_t ERR_INPUT = 4u;      // device-side input validation failed

// ---------------------------------------------------------------------------
// Segmented aggregate carried between tiles of a sweep.
//
// A sweep walks the live adjacency entries in order.  Entries are grouped in
// rows (one row per live vertex); an entry "survives" when neither endpoint
// was matched.  For a contiguous run X of entries:
//   S   number of survivors in X
//   H   X contains the first entry of some row
//   HS  the head segment (entries of X before its first row start; all of X
//       when !H) has a survivor
//   TS  the tail segment (from the last row start in X to its end) has a
//       survivor; equals HS when !H
//   nr  rows that start inside X and have a survivor inside X (each such row
//       becomes one row of the compacted graph)
// combine(X, Y) describes X followed by Y; it is associative with identity
// agg_identity().  The exclusive prefix of a tile is the combination of all
// earlier tiles; the first tile starts a row, so a prefix has H set, its S is
// the output position of the tile's first survivor, its nr the number of
// compacted rows before the tile, and its TS says whether the row that
// continues into the tile already has a survivor.
constexpr uint32_t F_H = 1u, F_HS = 2u, F_TS = 4u;

struct Agg {
    uint32_t S, nr, f;
};

LM_HD Agg agg_identity() {
    Agg a;
    a.S = 0; a.nr = 0; a.f = 0;
    return a;
}

LM_HD Agg agg_combine(const Agg& X, const Agg& Y) {
    const bool xh = (X.f & F_H) != 0, yh = (Y.f & F_H) != 0;
    const bool xhs = (X.f & F_HS) != 0, yhs = (Y.f & F_HS) != 0;
    const bool xts = (X.f & F_TS) != 0, yts = (Y.f & F_TS) != 0;
    Agg r;
    r.S = X.S + Y.S;
    // Y's head continues X's tail row; if X has a row start, that row started
    // inside X and gets its first survivor in Y exactly when X's tail had none.
    r.nr = X.nr + Y.nr + ((xh && yhs && !xts) ? 1u : 0u);
    const bool h = xh || yh;
    const bool hs = xh ? xhs : (xhs || yhs);
    const bool ts = yh ? yts : (xts || yhs);
    r.f = (h ? F_H : 0u) | (hs ? F_HS : 0u) | (ts ? F_TS : 0u);
    return r;
}

LM_HD void kv_max(uint64_t& k, uint32_t& u, uint64_t k2, uint32_t u2) {
    if (k2 > k) { k = k2; u = u2; }
}

// Partial maxima of one tile, for rows cut by tile boundaries: the heaviest
// surviving key (0 = none) and its neighbour in the head segment and in the
// tail segment (tail = head when the tile has no row start).
struct alignas(16) Part {
    uint64_t hk, tk;
    uint32_t hu, tu, pad0, pad1;
};

// ---------------------------------------------------------------------------
// Device-side control block (one per context workspace).
struct DevState {
    uint32_t cnt[2][2];       // [buffer][0 = live entries, 1 = live rows] of each ping-pong buffer
    uint32_t tile_ctr;        // dynamic tile counter of the running sweep
    uint32_t exit_ctr;        // CTAs of the running sweep that have finished
    uint32_t epoch;           // sweep generation (tags look-back records)
    uint32_t err;             // ERR_* bits
    uint32_t err_info;        // first failing index (debug aid)
    uint32_t rounds;          // rounds completed when the edge set became empty
    unsigned long long matched2;  // matched vertices (= 2 |M|)
    uint64_t ring_m[64];      // live edges at the start of round r
    uint64_t ring_n[64];      // live rows at the start of round r
};

// One input graph as a source segment of a sweep (the graph's own CSR).
struct SegDesc {
    const uint32_t* off;      // [nrows + 1] row offsets (rows = vertices with degree > 0)
    const uint32_t* vid;      // [nrows] local vertex id of each row
    const uint32_t* nbr;      // [nent] local neighbour id of each entry
    const uint32_t* eid;      // [nent] edge id of each entry
    const uint32_t* ordw;     // [nent] ord(weight) of each entry
    const uint32_t* tilemap;  // [ntiles + 1] row containing entry t*SWEEP_T; [ntiles] = nrows
    uint32_t nrows, nent, vbase, k0, k1, tile_begin, ntiles, pad;
};

// Arguments of a sweep launch.
struct SweepArgs {
    // INPUT source
    const SegDesc* segs;
    uint32_t nsegs, ntiles_in;
    // LIVE source (compacted arrays of the previous round)
    const uint64_t* in_key;
    const uint32_t* in_nbr;
    const uint32_t* in_off;
    const uint32_t* in_vid;
    const uint32_t* in_tilemap;
    uint32_t in_buf;          // which DevState::cnt buffer describes the live source
    // outputs (COMPACT mode)
    uint64_t* out_key;
    uint32_t* out_nbr;
    uint32_t* out_off;
    uint32_t* out_vid;
    uint32_t out_buf;         // DevState::cnt buffer that receives the new counts
    uint32_t out_cap;         // capacity of out_key / out_nbr (entries)
    uint32_t out_rows_cap;    // capacity of out_vid (rows); out_off holds one more
    uint32_t round;           // round index of this sweep (stats)
    const uint32_t* prefix_in;  // optional (S, N) the first tile starts from (appending sweeps); NULL = 0
    // vertex state
    uint32_t* cnbr;           // [N] chosen neighbour of each vertex (written for the next round)
    const uint8_t* dead;      // [N] 1 = matched
    uint32_t nvert;           // N (bounds checks)
    // look-back storage: one 16-byte descriptor per tile {status, S, nr, flags}
    // (status = generation << 2 | 1 aggregate / 2 inclusive prefix) and the
    // tile's partial maxima
    uint32_t* lb_desc;        // [lb_cap * 4]
    Part* lb_part;            // [lb_cap]
    uint32_t lb_cap;          // tiles that fit
    DevState* st;
};

struct VertexArgs {
    // LIVE rows (round >= 1) or a vertex range (round 0)
    const uint32_t* off;
    const uint32_t* vid;
    uint32_t in_buf;          // DevState::cnt buffer with the live row / entry counts
    uint32_t vbegin, vcount;  // round 0: vertices [vbegin, vbegin + vcount) are scanned
    uint32_t nvert;           // total vertices of the vertex arrays (bounds)
    // optional per-graph round counters (batched form): graph g owns vertices
    // [gvbase[g], gvbase[g+1]); grounds[g] = max(round + 1) over its matches
    const uint32_t* gvbase;
    uint32_t ngraphs, round;
    uint32_t* grounds;
    uint32_t* cnbr;
    uint8_t* dead;
    uint32_t* mate;
    uint32_t* tilemap;        // LIVE: tile map of the live entries for the coming sweep
    uint32_t tilemap_cap;
    DevState* st;
};

// ---------------------------------------------------------------------------
// Host-callable launchers (defined in lm_kernels.cu).  All return a
// cudaError_t value as int.
// mate (if non-null) and cnbr := NIL, dead := 0 for n vertices; st (if non-null) is reset for a new match
int launch_init(void* stream, uint32_t* mate, uint32_t* cnbr, uint8_t* dead, uint32_t n, DevState* st);
int launch_sweep_input_cand(void* stream, const SweepArgs& a, int grid);
int launch_sweep_input_compact(void* stream, const SweepArgs& a, int grid);
int launch_sweep_live(void* stream, const SweepArgs& a, int grid);
int launch_vertex_all(void* stream, const VertexArgs& a, int grid);
int launch_vertex_live(void* stream, const VertexArgs& a, int grid);
int sweep_grid(int device);   // persistent grid size for sweeps (SMs x resident CTAs)
int vertex_grid(int device);

// graph construction
int launch_build_degrees(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n,
                         uint32_t m, uint32_t* deg, uint32_t* err);
int launch_exclusive_scan(void* stream, const uint32_t* in, uint32_t* out, uint32_t count, uint32_t* tmp,
                          size_t tmp_words);
size_t exclusive_scan_tmp_words(uint32_t count);
int launch_build_fill(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t m,
                      const uint32_t* rowstart_all, uint32_t* cursor, uint32_t* nbr, uint32_t* eid,
                      uint32_t* ordw);
int launch_build_rows(void* stream, const uint32_t* deg, const uint32_t* rowidx_excl, const uint32_t* off_all,
                      uint32_t n, uint32_t nrows, uint32_t nent, uint32_t* off0, uint32_t* vid0);
int launch_build_tilemap(void* stream, const uint32_t* off0, uint32_t nrows, uint32_t nent, uint32_t* tilemap);
int launch_nonzero_flags(void* stream, const uint32_t* deg, uint32_t n, uint32_t* flags);
// out[v] = local id of mate_global[vbase + v] (v < n); *matched2 += matched vertices (if non-null)
int launch_to_local(void* stream, const uint32_t* mate_global, uint32_t vbase, uint32_t n, uint32_t* out,
                    unsigned long long* matched2);
// union results -> per-graph local ids: graph g owns union vertices [gvbase[g], gvbase[g+1]) and its
// result goes to dst[g] (device pointer, n_g entries); matched2[g] += matched vertices of g
int launch_to_local_batch(void* stream, const uint32_t* mate_union, const uint32_t* gvbase, uint32_t ngraphs,
                          uint32_t* const* dst, unsigned long long* matched2, uint32_t nvert);
// live rows per request: row i of the union belongs to graph g (by gvbase); rows_per[g] += 1
int launch_rows_per_graph(void* stream, const uint32_t* vid, const DevState* st, uint32_t buf,
                          const uint32_t* gvbase, uint32_t ngraphs, uint32_t* rows_per, int grid);

}  // namespace lm
