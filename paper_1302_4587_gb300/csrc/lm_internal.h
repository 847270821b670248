// Internal declarations shared by the kernels (lm_kernels.cu, lm_contract.cu) and
// the host code (lm_api.cpp, lm_serve.cpp).  Not part of the public ABI (include/lm.h is).
//
// Layout of one matching job (one graph, or the disjoint union of a batch):
//   * vertices live in a union id space [0, N); graph g owns [vbase_g, vbase_g + n_g)
//   * adjacency entries live in a union entry space; vertex v's row occupies
//     [start[v], start[v] + deg(v)) -- the graph's own CSR range, shifted by the
//     graph's entry base.  The row never moves: in every round its surviving
//     entries are compacted to the front of the same range of the other
//     ping-pong buffer, and len[round & 1][v] says how many there are.
//   * a round works from two task lists built by the vertex pass:
//       R  rows with 1..RMAX live entries (a warp takes 32 rows and walks
//          their entries as one flattened sequence)
//       C  chunks of up to CHUNK entries of longer rows (one warp per chunk)
//   * a row keeps only the heaviest surviving key; the neighbour over that
//     edge is recovered from the key itself: its low half is perm_seed(e),
//     which is inverted to the edge index e, whose record holds both ends.
#pragma once
#include <stdint.h>
#include <stddef.h>

#include <vector_types.h>

#if defined(__CUDACC__)
#define LM_HD __host__ __device__ __forceinline__
#else
#define LM_HD inline
#endif

namespace lm {

constexpr uint32_t NIL = 0xFFFFFFFFu;

// Task sizes of the sweep.  A warp walks a sweep's task list at a rate set by
// memory latency, so the longest task bounds the sweep's tail: rows of up to
// LM_RMAX live entries are batched (at most 32 rows, and a batch ends where
// its entries cross a multiple of 1 << LM_BATCH_SHIFT, so no batch holds much
// more than LM_RMAX + that many entries); longer rows are cut into chunks of
// LM_CHUNK entries.  Measured best on R-MAT scales 21 and 23 (1024 / 512 / 1024).
#ifndef LM_CHUNK
#define LM_CHUNK 1024
#endif
#ifndef LM_RMAX
#define LM_RMAX 1024
#endif
#ifndef LM_BATCH_SHIFT
#define LM_BATCH_SHIFT 9
#endif
constexpr uint32_t CHUNK = LM_CHUNK;        // long rows are split into chunks of this size
#ifndef LM_TILE0
#define LM_TILE0 1024
#endif
constexpr uint32_t TILE0 = LM_TILE0;        // round 0 streams the input adjacency in tiles of this many entries
constexpr uint32_t RMAX = LM_RMAX;          // rows up to this length are batched 32 to a warp

// error bits written to DevState::err by kernels
constexpr uint32_t ERR_TIMEOUT = 1u;    // a bounded device wait gave up
constexpr uint32_t ERR_BOUNDS = 2u;     // an index check failed (vertex / entry / list)
constexpr uint32_t ERR_INPUT = 4u;      // device-side input validation failed

LM_HD void kv_max(uint64_t& k, uint32_t& u, uint64_t k2, uint32_t u2) {
    if (k2 > k) { k = k2; u = u2; }
}

// Task lists of one round: R holds (vertex, live length) pairs, C holds
// (vertex, chunk index) pairs; a row's chunks are consecutive in C.  R is cut
// into batches of consecutive rows (at most 32, see LaunchCfg::batch_shift):
// bit 31 of a row's length word marks the first row of a batch, and B lists
// the R index of every batch's first row, in no particular order.
constexpr uint32_t BATCH_START = 0x80000000u;
constexpr uint32_t R_LEN_KNOWN = 0x80000000u;  // vertex pass, internal: the length came with the entry
struct Lists {
    uint2* R;
    uint2* C;
    uint32_t* B;
    uint32_t capR, capC;      // B holds at most capR entries
    uint32_t* cnt;            // device counters {nR, nC, nB}
};

// Device-side control block (one per engine).
struct DevState {
    uint32_t lcnt[4][4];      // counters {nR, nC, nB, -} of the four list sets
    uint32_t exit_v, exit_s;  // CTAs of the running vertex pass / sweep that have finished
    uint32_t task[4];         // task counters of the sweeps that follow a vertex pass
    uint32_t err;             // ERR_* bits
    uint32_t err_info;        // first failing index (debug aid)
    uint32_t rounds;          // set to r by the vertex pass of round r that found no live row
    uint32_t done;            // 1 once the edge set is empty
    uint32_t live_rows;       // live rows seen by the running vertex pass
    uint32_t round;           // next round of the device-driven loop
    uint32_t max_rounds;      // the device-driven loop stops (ERR_TIMEOUT) beyond this round ...
    uint32_t err_any;         // ERR_* bits of every job since the host last cleared them
    unsigned long long t0_ns; // ... or limit_ns after the job started
    unsigned long long limit_ns;
    unsigned long long live_ent;   // live entries seen by the running vertex pass
    unsigned long long matched2;   // matched vertices (= 2 |M|)
    unsigned long long last_ent;   // live entries the last vertex pass saw (its round's)
    uint32_t tail;            // 1: the remaining rounds run in the one-CTA tail kernel
    uint32_t tail_round;      // the round the tail kernel took over at
    uint64_t ring_m[64];      // live edges at the start of round r
    uint64_t ring_n[64];      // live vertices at the start of round r
};

// Arrays of one graph: round 0 reads its adjacency entries, every round
// recovers candidate neighbours from its edge records.
struct SegIn {
    const uint32_t* nbr;      // [2m] neighbour (local id) of each entry of the graph's CSR
    const uint64_t* pk;       // [2m] ord(weight) << 32 | edge index, per entry
    const uint64_t* edges;    // [m] edge records: eu | ev << 32 (local ids)
    const uint32_t* roff;     // [nrows + 1] entry offset of each row (rows = vertices with edges)
    const uint32_t* rvid;     // [nrows] local vertex id of each row
    const uint32_t* tmap;     // [ntiles + 1] row containing entry t * TILE0; [ntiles] = nrows
    const uint32_t* rbits;    // [ntiles * TILE0 / 32 + 8] bit j set: a row starts at entry j
    const uint4* tdesc;       // [ntiles] per round-0 tile: first row, rows touched, first row's offset
    uint32_t m;               // edges
    uint32_t nrows, nent;     // rows, entries (2m)
    uint32_t ntiles, tile_begin;  // round-0 tiles of the graph and the job-wide index of the first
    uint32_t ebase;           // union entry index of the graph's entry 0
    uint32_t vbase;           // union id of the graph's vertex 0
    uint32_t k0, k1;          // perm_seed keys of the graph's seed (round 0)
    uint64_t seed;            // the seed itself (renewed keys of later rounds)
};

// Launch parameters a context may tune (lm_set_tuning / lm_autotune): the
// sweep's task sizes and the CTAs per SM of the vertex pass and the sweep
// (0 = as many as fit).
struct LaunchCfg {
    uint32_t rmax = RMAX;
    uint32_t chunk_shift = 0;
    uint32_t sweep_ctas_per_sm = 0;
    uint32_t vertex_ctas_per_sm = 4;
    uint32_t batch_shift = LM_BATCH_SHIFT;  // 32: batches of 32 rows only
    bool renew = false;  // sweeps renew the order every round (LM_F_RENEW)
    uint32_t contract_bits = 0;  // bits of the contraction's hash sort (0: by size); no match graph uses it
    LaunchCfg() {
        while ((1u << chunk_shift) < CHUNK) chunk_shift++;
    }
    bool operator==(const LaunchCfg& o) const {
        return rmax == o.rmax && chunk_shift == o.chunk_shift && sweep_ctas_per_sm == o.sweep_ctas_per_sm &&
               vertex_ctas_per_sm == o.vertex_ctas_per_sm && batch_shift == o.batch_shift && renew == o.renew;
    }
    bool operator!=(const LaunchCfg& o) const { return !(*this == o); }
};

// Per-vertex arrays of a job (union ids).
struct VertexArrays {
    const uint32_t* start;    // [N] union entry index of each vertex's row
    uint32_t* len[2];         // [N] live length of each row, by round parity
    uint32_t* cnbr;           // [N] neighbour over the heaviest live edge (valid for live rows)
    uint32_t* dead;           // [N / 32 + 1] bit v set once v is matched (read through the read-only cache)
    uint32_t* mate;           // [N] result (union ids)
    uint32_t* bcnt;           // [N] chunks of a long row finished in the running sweep
    unsigned long long* bkey; // [N] heaviest surviving key of a long row (0 between sweeps)
    const uint32_t* gid;      // [N] graph of each vertex (NULL: single graph 0)
    uint32_t nvert;           // N
};

// Vertex pass: reads rows from `in` (or an explicit vertex list), checks the
// mutual choice (when match != 0), and files every live unmatched row into `out`.
struct VertexArgs {
    VertexArrays va;
    Lists in;                 // rows of the previous round (when vlist == NULL)
    uint32_t in_set;          // DevState::lcnt index of `in` (zeroed when the pass ends; 4 = none)
    const uint32_t* vlist;    // explicit rows (round 0): vertex ids
    uint32_t nvlist;
    uint32_t vlist_base;      // added to vlist entries (union id of the list's graph)
    const uint32_t* deg0;     // explicit rows: row length source (indexed like vlist), NULL = len_cur
    Lists out;
    uint32_t out_set;
    uint32_t par;             // round parity: lengths in va.len[par], next ones in va.len[par ^ 1]
    uint32_t round;
    uint32_t match;           // 0 = classification only (before the candidate sweep)
    uint32_t round_from_state; // 1: the round index is DevState::round (advanced by this pass)
    uint32_t* grounds;        // per-graph rounds: max(round + 1) over graphs with a live row, NULL = none
    uint32_t* glive;          // live unmatched rows per graph seen by this pass, NULL = none
    uint32_t rmax;            // rows of at most this many live entries go to R, longer ones to C
    uint32_t chunk_shift;     // chunks of a long row hold 1 << chunk_shift entries
    uint32_t batch_shift;     // a batch of R ends where its entries cross a multiple of
                              // 1 << batch_shift (32: after 32 rows only)
    DevState* st;
};

// Sweep over the tasks of `in`.
struct SweepArgs {
    VertexArrays va;
    Lists in;
    uint32_t in_set;
    uint32_t par;             // source lengths va.len[par]; next lengths va.len[par ^ 1]
    // LIVE source (rounds >= 1): buffers of the previous round
    const uint64_t* in_key;
    const uint32_t* in_nbr;
    // the graphs' own arrays (round 0 entries; every round: edge records)
    const SegIn* segs;
    uint32_t nsegs;
    uint32_t* task_ctr;       // dynamic task counter (zeroed by the preceding vertex pass)
    // destination (compacting sweeps)
    uint64_t* out_key;
    uint32_t* out_nbr;
    uint32_t ecap;            // entries in the union entry space
    uint32_t rmax, chunk_shift;  // as in VertexArgs
    DevState* st;
};

// Round-0 candidates over the graphs' own adjacency arrays in tiles of TILE0 entries.
struct Round0Args {
    VertexArrays va;
    const SegIn* segs;
    uint32_t nsegs, ntiles;   // graphs, tiles of all graphs
    DevState* st;
};

// Arguments of a whole job in device memory, for the device-driven loop:
// r0 finds the round-0 candidates, v[0] matches round 0 and files the open
// rows, s[0] compacts from the input arrays, v[1]/s[1] run round 1, and
// v[2]/s[2], v[3]/s[3] run rounds of parity 0 and 1.
struct InitArgs {
    uint32_t* mate;
    uint32_t* dead;           // the whole bitmap; bits [dbase, dbase + n) are cleared
    uint32_t dbase;
    uint32_t* bcnt;
    unsigned long long* bkey;
    uint32_t n;
    uint32_t max_rounds;
    unsigned long long limit_ns;  // the job's time limit (ERR_TIMEOUT once exceeded)
    DevState* st;
};
struct JobArgs {
    InitArgs init;
    Round0Args r0;            // round-0 candidates
    VertexArgs v[4];          // round 0, round 1, loop rounds of parity 0 and 1
    SweepArgs s[4];           // round-0 compaction, round 1, loop rounds of parity 0 and 1
};
// The edge-centric path (LM_F_EDGE_CENTRIC) of one graph: per round every live
// edge offers its key to both ends (atomic maximum), an edge that is the best
// offer at both ends is matched, and the others with no matched end are
// compacted into the next round's edge list.  Round r = DevState::round - 1.
struct EdgeArgs {
    const uint64_t* edges;       // [m] eu | ev << 32
    const uint32_t* eword;       // [m] ord(weight)
    uint32_t m, k0, k1, nvert;
    uint32_t* live[2];           // live edge ids by round parity (round 0: every edge, implicitly)
    uint32_t cap;                // capacity of each live list
    unsigned long long* best;    // [n] heaviest offer of the running round (zero between rounds)
    uint32_t* stamp;             // [n] round + 1 of the last offer (zero between rounds)
    uint32_t* dead;              // matched bits
    uint32_t* mate;
    DevState* st;
};

constexpr unsigned long long LOOP_LIMIT_NS = 120000000000ull;  // 120 s: the default time limit of a job
// once a round starts with fewer live entries than this, the rounds that remain
// run in one kernel of one CTA (no launch per round)
#ifndef LM_TAIL_ENT
#define LM_TAIL_ENT 4096
#endif
constexpr unsigned long long TAIL_ENT = LM_TAIL_ENT;

// ---------------------------------------------------------------------------
// Host-callable launchers (defined in lm_kernels.cu).  All return a
// cudaError_t value as int.
// kernel arguments are passed as pointers to device memory
int launch_init(void* stream, const InitArgs* dargs);
int launch_vertex(void* stream, const VertexArgs* dargs, const struct LaunchCfg& cfg);
int launch_sweep_cand(void* stream, const SweepArgs* dargs, const struct LaunchCfg& cfg);   // round 0, candidates only
int launch_sweep_input(void* stream, const SweepArgs* dargs, const struct LaunchCfg& cfg);  // round-0 compaction
int launch_sweep_live(void* stream, const SweepArgs* dargs, const struct LaunchCfg& cfg);   // rounds >= 1
int launch_round0(void* stream, const Round0Args* dargs);      // round-0 candidates in TMA-fed tiles
int launch_round0_cut(void* stream, const Round0Args* dargs);  // candidates of rows cut by tile boundaries
int device_sm_count(int device);
uint64_t splitmix64_first(uint64_t seed);  // lm_api.cpp
// executable graph that runs a whole job from its arguments in device memory
// (init, round 0, then a conditional loop of rounds until the device's done
// flag is set); returns a cudaError_t value
int build_job_graph(const JobArgs* dargs, DevState* st, const struct LaunchCfg& cfg, void** exec_out);
// the one-CTA tail of a job (profiled path): runs the remaining rounds from rounds 2 / 3's arguments
int launch_tail(void* stream, const JobArgs* dargs, const struct LaunchCfg& cfg);

// contraction of a matching (lm_contract): inputs, outputs and device scratch
struct ContractArgs {
    uint32_t n, m;
    const uint32_t *eu, *ev;
    const float* w;
    const uint32_t* vw;       // NULL = 1 per vertex
    const uint32_t* mate;
    uint32_t *cmap, *cvw, *ceu, *cev;
    float* cw;
    uint32_t* flag;           // [n + 1] representative flags
    uint32_t* rank;           // [n + 1] their exclusive prefix (rank[n] = coarse vertices)
    uint32_t* cross;          // [m / 32 + 2] bit e: edge e joins two coarse vertices, then: it leads its group
    uint32_t* counts;         // [8] crossing edges, items of runs left to the pair sort, coarse edges,
                              // items taken out for it
    uint32_t* cpair;          // [2 m] coarse endpoints of every edge, cmap[eu[e]] then cmap[ev[e]]
    unsigned long long* key[2];  // [m] coarse pair of each crossing edge (radix ping-pong)
    uint32_t* val[2];         // [m] its edge index
    uint32_t* shist;          // radix pass: [256 * tiles] per-tile digit counts, then their exclusive prefix
    uint32_t* multi;          // [m / 32 + 2] bit e: edge e leads a group of several edges
    uint32_t* wlead;          // [m / 32 + 2] flags of the sorted items left to the pair sort, then
                              // leaders per word of cross
    uint32_t* wpos;           // [m / 32 + 2] their exclusive prefix (wpos[words] = coarse edges)
    uint32_t* tsum;           // [2 * (m / 4096 + 2)] per-tile counts of run items and their prefix
    uint32_t* gref;           // [m] float32 bits of the weight of a group led by edge e (groups of several edges)
    uint32_t* scan_tmp;
    size_t scan_words;
    uint32_t* err;            // bit 1: mate is not a matching, 2: endpoint >= n
    uint32_t sort_bits;       // low bits of the hash the sort orders by (8, 16, 24, 32; 0: by size)
};
size_t contract_sort_words(uint32_t m);  // words of shist
// runs every step; mc_host_slot: 2 pinned words (crossing edges and coarse vertices
// are read back once, to size the sort); returns a cudaError_t value
int launch_contract(void* stream, const ContractArgs& c, uint32_t* mc_host_slot);
int launch_job_graph(void* exec, void* stream);
// edge-centric path: the job graph (init, then a conditional loop of rounds) and the
// per-round launches of the profiled path
int build_edge_graph(const InitArgs* init, const EdgeArgs* dargs, DevState* st, void** exec_out);
int launch_edge_round(void* stream, const EdgeArgs* dargs, int phase);  // phase 0 offer, 1 match, 2 compact, 3 close
void destroy_job_graph(void* exec);

// graph construction
int launch_build_degrees(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n,
                         uint32_t m, uint32_t* deg, uint32_t* err);
int launch_exclusive_scan(void* stream, const uint32_t* in, uint32_t* out, uint32_t count, uint32_t* tmp,
                          size_t tmp_words);
size_t exclusive_scan_tmp_words(uint32_t count);
// fill: tmp = build_fill_tmp_words(n, m) words of 16-byte aligned scratch; scan_tmp sized for
// exclusive scans of build_fill_scan_count(n, m) words
size_t build_fill_tmp_words(uint32_t n, uint32_t m);
uint32_t build_fill_scan_count(uint32_t n, uint32_t m);
int launch_build_fill(void* stream, const uint32_t* eu, const uint32_t* ev, const float* w, uint32_t n, uint32_t m,
                      uint32_t* cursor, uint32_t* nbr, uint64_t* pk, uint64_t* edges, uint32_t* eword, uint32_t* tmp,
                      uint32_t* scan_tmp, size_t scan_words, uint32_t* err);  // err |= 2 when a fill slot falls outside 2m
int launch_build_rows(void* stream, const uint32_t* deg, const uint32_t* rowidx_excl, const uint32_t* off,
                      uint32_t n, uint32_t nrows, uint32_t nent, uint32_t* vid0, uint32_t* rdeg0, uint32_t* roff);
int launch_build_tilemap(void* stream, const uint32_t* roff, uint32_t nrows, uint32_t nent, uint32_t* tmap,
                         uint32_t* rbits, uint4* tdesc);
int launch_nonzero_flags(void* stream, const uint32_t* deg, uint32_t n, uint32_t* flags);
// union set-up of a batch: for every graph g (vertices [gvbase[g], gvbase[g+1])):
// start[v] = ebase[g] + off_g[v - gvbase[g]], gid[v] = g, len0[v] = degree
int launch_union_setup(void* stream, const uint32_t* gvbase, const uint32_t* ebase, const uint32_t* const* offs,
                       uint32_t ngraphs, uint32_t nvert, uint32_t* start, uint32_t* gid, uint32_t* len0);
// serving: start[vbase + i] = ebase + off[i], gid[vbase + i] = slot for i < n
int launch_req_setup(void* stream, const uint32_t* off, uint32_t n, uint32_t vbase, uint32_t ebase, uint32_t slot,
                     uint32_t* start, uint32_t* gid);
// out[v] = local id of mate_global[vbase + v] (v < n); *matched2 += matched vertices (if non-null)
int launch_to_local(void* stream, const uint32_t* mate_global, uint32_t vbase, uint32_t n, uint32_t* out,
                    unsigned long long* matched2);
// union results -> per-graph local ids into dst[g] (device pointers; NULL = skip); matched2[g] += matched vertices
int launch_to_local_batch(void* stream, const uint32_t* mate_union, const uint32_t* gvbase, const uint32_t* gid,
                          uint32_t ngraphs, uint32_t* const* dst, unsigned long long* matched2, uint32_t nvert);

}  // namespace lm
