/*
 * Seeded synthetic graph generators.
 *
 * These produce the inputs that both the CUDA path and the oracle consume:
 * plain undirected edge lists (eu[i], ev[i], w[i]).  Nothing in this file
 * computes any part of the matching method (no edge order, no keys, no
 * matching); it only draws graphs.
 *
 * Randomness is counter based: the i-th draw of stream `s` is the i-th
 * output of SplitMix64 seeded with `s` (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), so every draw is a pure
 * function of (seed, index) and the large generators can run on several
 * threads while producing identical bytes.
 *
 * Workload shapes follow the paper's input families (Sec. 3): random graphs
 * with uniform [0,1) weights, a locality-heavy grid family standing in for the
 * geometric and sparse-matrix inputs, and a skewed R-MAT family (Chakrabarti,
 * Zhan, Faloutsos 2004) standing in for the large irregular graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (i >= 0) of SplitMix64 seeded with `seed`. */
uint64_t sx_at(uint64_t seed, uint64_t i) { return mix64(seed + (i + 1) * GAMMA); }

/* Derive an independent stream seed from (seed, tag). */
uint64_t sx_derive(uint64_t seed, uint64_t tag) { return sx_at(seed ^ (tag * 0xD1B54A32D192ED03ULL), tag); }

/* uniform double in [0,1) with 53 random bits */
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------ */
/* open-addressing set of canonical pairs (min<<32 | max)              */
typedef struct { uint64_t* slot; uint64_t mask; } pairset;

static int ps_init(pairset* s, uint64_t expect) {
    uint64_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    s->slot = (uint64_t*)malloc(cap * sizeof(uint64_t));
    if (!s->slot) return -1;
    memset(s->slot, 0xFF, cap * sizeof(uint64_t)); /* all-ones = empty (never a valid pair: min<max) */
    s->mask = cap - 1;
    return 0;
}
static void ps_free(pairset* s) { free(s->slot); s->slot = NULL; }
/* returns 1 if inserted, 0 if present */
static int ps_insert(pairset* s, uint64_t key) {
    uint64_t h = mix64(key) & s->mask;
    for (;;) {
        uint64_t v = s->slot[h];
        if (v == key) return 0;
        if (v == ~0ULL) { s->slot[h] = key; return 1; }
        h = (h + 1) & s->mask;
    }
}
static inline uint64_t canon(uint32_t a, uint32_t b) {
    return a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
}

/* ------------------------------------------------------------------ */
/* Erdos-Renyi G(n, m): m distinct non-loop unordered pairs drawn uniformly by
 * rejection; edge i is the i-th accepted pair, endpoints in drawn order.
 * Returns m, or -1 if m exceeds the number of pairs / on allocation failure. */
int64_t gen_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t* eu, uint32_t* ev) {
    if (n < 2 || m > (uint64_t)n * (n - 1) / 2) return m == 0 ? 0 : -1;
    pairset s;
    if (ps_init(&s, m)) return -1;
    uint64_t k = 0, i = 0;
    while (k < m) {
        uint64_t x = sx_at(seed, i++);
        uint32_t a = (uint32_t)(((x & 0xFFFFFFFFULL) * n) >> 32);
        uint32_t b = (uint32_t)(((x >> 32) * n) >> 32);
        if (a == b) continue;
        if (!ps_insert(&s, canon(a, b))) continue;
        eu[k] = a; ev[k] = b; k++;
    }
    ps_free(&s);
    return (int64_t)k;
}

/* 2D grid rows x cols with 4-neighbour edges (vertex id = r*cols + c), listed
 * row by row (right edge then down edge of each cell), followed by n_long
 * uniform random long-range pairs that are neither loops nor duplicates of
 * any earlier edge.  If n_vertices < rows*cols, only the first n_vertices
 * cells (row-major) exist and edges to missing cells are skipped; if
 * max_edges is smaller than the grid edge count, the list is cut there.
 * Returns the edge count, or -1 on allocation failure / capacity overflow. */
int64_t gen_grid(uint32_t rows, uint32_t cols, uint32_t n_vertices, uint64_t n_long,
                 uint64_t max_edges, uint64_t seed, uint32_t* eu, uint32_t* ev, uint64_t cap) {
    uint64_t n = n_vertices;
    if ((uint64_t)rows * cols < n) return -1;
    pairset s;
    if (ps_init(&s, 2 * n + n_long)) return -1;
    uint64_t k = 0;
    for (uint32_t r = 0; r < rows && k < max_edges; r++) {
        for (uint32_t c = 0; c < cols && k < max_edges; c++) {
            uint64_t v = (uint64_t)r * cols + c;
            if (v >= n) break;
            if (c + 1 < cols && v + 1 < n && k < max_edges) {
                if (k >= cap) { ps_free(&s); return -1; }
                eu[k] = (uint32_t)v; ev[k] = (uint32_t)(v + 1); ps_insert(&s, canon(eu[k], ev[k])); k++;
            }
            if (r + 1 < rows && v + cols < n && k < max_edges) {
                if (k >= cap) { ps_free(&s); return -1; }
                eu[k] = (uint32_t)v; ev[k] = (uint32_t)(v + cols); ps_insert(&s, canon(eu[k], ev[k])); k++;
            }
        }
    }
    uint64_t want = k + n_long;
    if (n < 2) want = k;
    if (want > cap) { ps_free(&s); return -1; }
    if (n >= 2 && want > n * (n - 1) / 2) want = n * (n - 1) / 2;
    uint64_t i = 0;
    while (k < want) {
        uint64_t x = sx_at(seed, i++);
        uint32_t a = (uint32_t)(((x & 0xFFFFFFFFULL) * n) >> 32);
        uint32_t b = (uint32_t)(((x >> 32) * n) >> 32);
        if (a == b) continue;
        if (!ps_insert(&s, canon(a, b))) continue;
        eu[k] = a; ev[k] = b; k++;
    }
    ps_free(&s);
    return (int64_t)k;
}

/* ------------------------------------------------------------------ */
/* Random geometric graph (Sec. 3's rgg family): n points uniform in the unit
 * square (point i from draws 2i and 2i+1), an edge between every two points
 * closer than `radius`.  Points are bucketed in k x k cells of side 1/k >=
 * radius; each pair is listed once, from its lower id, in id order and, for one
 * id, in cell-scan order.  Returns the edge count, or -1 when cap is too small
 * or on allocation failure. */
int64_t gen_rgg(uint32_t n, double radius, uint64_t seed, uint32_t* eu, uint32_t* ev, uint64_t cap) {
    if (n == 0) return 0;
    if (!(radius > 0.0)) return 0;
    uint32_t k = (uint32_t)(1.0 / radius);
    if (k < 1) k = 1;
    if (k > 65536) k = 65536;
    double* x = (double*)malloc((size_t)n * sizeof(double));
    double* y = (double*)malloc((size_t)n * sizeof(double));
    uint32_t* cell = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* start = (uint32_t*)calloc((size_t)k * k + 1, sizeof(uint32_t));
    uint32_t* order = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!x || !y || !cell || !start || !order) {
        free(x); free(y); free(cell); free(start); free(order);
        return -1;
    }
    for (uint32_t i = 0; i < n; i++) {
        x[i] = u01(sx_at(seed, 2ull * i));
        y[i] = u01(sx_at(seed, 2ull * i + 1));
        uint32_t cx = (uint32_t)(x[i] * k), cy = (uint32_t)(y[i] * k);
        if (cx >= k) cx = k - 1;
        if (cy >= k) cy = k - 1;
        cell[i] = cy * k + cx;
        start[cell[i] + 1]++;
    }
    for (uint64_t c = 0; c < (uint64_t)k * k; c++) start[c + 1] += start[c];
    {
        uint32_t* fill = (uint32_t*)malloc(((size_t)k * k + 1) * sizeof(uint32_t));
        if (!fill) { free(x); free(y); free(cell); free(start); free(order); return -1; }
        memcpy(fill, start, ((size_t)k * k + 1) * sizeof(uint32_t));
        for (uint32_t i = 0; i < n; i++) order[fill[cell[i]]++] = i;  /* ids ascending within a cell */
        free(fill);
    }
    const double r2 = radius * radius;
    uint64_t m = 0;
    int fail = 0;
    for (uint32_t i = 0; i < n && !fail; i++) {
        const int32_t cx = (int32_t)(cell[i] % k), cy = (int32_t)(cell[i] / k);
        for (int32_t dy = -1; dy <= 1 && !fail; dy++) {
            for (int32_t dx = -1; dx <= 1 && !fail; dx++) {
                const int32_t nx = cx + dx, ny = cy + dy;
                if (nx < 0 || ny < 0 || nx >= (int32_t)k || ny >= (int32_t)k) continue;
                const uint32_t c = (uint32_t)ny * k + (uint32_t)nx;
                for (uint32_t t = start[c]; t < start[c + 1]; t++) {
                    const uint32_t j = order[t];
                    if (j <= i) continue;
                    const double ddx = x[i] - x[j], ddy = y[i] - y[j];
                    if (ddx * ddx + ddy * ddy >= r2) continue;
                    if (m >= cap) { fail = 1; break; }
                    eu[m] = i;
                    ev[m] = j;
                    m++;
                }
            }
        }
    }
    free(x); free(y); free(cell); free(start); free(order);
    return fail ? -1 : (int64_t)m;
}

/* ------------------------------------------------------------------ */
/* R-MAT: one edge = `scale` quadrant choices with probabilities (a,b,c,d).
 * Draw j of edge e uses counter e*scale + j of the stream `seed`. */
static inline void rmat_edge(int scale, double a, double ab, double abc, uint64_t seed,
                             uint64_t e, uint32_t* pu, uint32_t* pv) {
    uint32_t u = 0, v = 0;
    for (int j = 0; j < scale; j++) {
        double x = u01(sx_at(seed, e * (uint64_t)scale + j));
        uint32_t bu = 0, bv = 0;
        if (x < a) { }
        else if (x < ab) { bv = 1; }
        else if (x < abc) { bu = 1; }
        else { bu = 1; bv = 1; }
        u = (u << 1) | bu;
        v = (v << 1) | bv;
    }
    *pu = u; *pv = v;
}

typedef struct {
    int scale; double a, ab, abc; uint64_t seed; const uint32_t* relabel;
    uint64_t e0, e1; uint64_t* out;
} rmat_job;

static void* rmat_worker(void* p) {
    rmat_job* J = (rmat_job*)p;
    for (uint64_t e = J->e0; e < J->e1; e++) {
        uint32_t u, v;
        rmat_edge(J->scale, J->a, J->ab, J->abc, J->seed, e, &u, &v);
        u = J->relabel[u]; v = J->relabel[v];
        J->out[e] = (u == v) ? ~0ULL : canon(u, v); /* loops become the all-ones sentinel */
    }
    return NULL;
}

/* LSD radix sort of 64-bit keys, 16-bit digits over the low `bits` bits */
static int radix_sort_u64(uint64_t* a, uint64_t n, int bits) {
    uint64_t* t = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* cnt = (uint64_t*)malloc(65536 * sizeof(uint64_t));
    if (!t || !cnt) { free(t); free(cnt); return -1; }
    uint64_t *src = a, *dst = t;
    for (int sh = 0; sh < bits; sh += 16) {
        memset(cnt, 0, 65536 * sizeof(uint64_t));
        for (uint64_t i = 0; i < n; i++) cnt[(src[i] >> sh) & 0xFFFF]++;
        uint64_t s = 0;
        for (int d = 0; d < 65536; d++) { uint64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (uint64_t i = 0; i < n; i++) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
        uint64_t* x = src; src = dst; dst = x;
    }
    if (src != a) memcpy(a, src, n * sizeof(uint64_t));
    free(t);
    free(cnt);
    return 0;
}

/* R-MAT graph with 2^scale vertices and n_gen generated edges; vertex ids are
 * relabelled by a seeded random permutation (Fisher-Yates over stream
 * derive(seed,1)); loops are dropped and duplicate undirected pairs removed.
 * Output edges are (min,max) pairs sorted ascending.  Returns the number of
 * distinct edges written (<= cap), or -1 on failure. */
int64_t gen_rmat(int scale, uint64_t n_gen, double a, double b, double c, uint64_t seed,
                 uint32_t* eu, uint32_t* ev, uint64_t cap, int nthreads) {
    if (scale < 1 || scale > 31) return -1;
    uint32_t nv = 1u << scale;
    uint32_t* relabel = (uint32_t*)malloc((size_t)nv * sizeof(uint32_t));
    uint64_t* keys = (uint64_t*)malloc((n_gen ? n_gen : 1) * sizeof(uint64_t));
    if (!relabel || !keys) { free(relabel); free(keys); return -1; }
    for (uint32_t i = 0; i < nv; i++) relabel[i] = i;
    uint64_t rs = sx_derive(seed, 1);
    for (uint32_t i = nv - 1; i > 0; i--) {
        uint32_t j = (uint32_t)(((sx_at(rs, nv - 1 - i) >> 32) * (uint64_t)(i + 1)) >> 32);
        uint32_t t = relabel[i]; relabel[i] = relabel[j]; relabel[j] = t;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    pthread_t th[64];
    rmat_job jobs[64];
    uint64_t es = sx_derive(seed, 2);
    for (int t = 0; t < nthreads; t++) {
        jobs[t].scale = scale; jobs[t].a = a; jobs[t].ab = a + b; jobs[t].abc = a + b + c;
        jobs[t].seed = es; jobs[t].relabel = relabel; jobs[t].out = keys;
        jobs[t].e0 = n_gen * t / nthreads; jobs[t].e1 = n_gen * (t + 1) / nthreads;
        if (pthread_create(&th[t], NULL, rmat_worker, &jobs[t])) { jobs[t].e1 = jobs[t].e0; rmat_worker(&jobs[t]); th[t] = 0; }
    }
    for (int t = 0; t < nthreads; t++) if (th[t]) pthread_join(th[t], NULL);
    free(relabel);
    /* drop loops (sentinel) before sorting */
    uint64_t k = 0;
    for (uint64_t i = 0; i < n_gen; i++) if (keys[i] != ~0ULL) keys[k++] = keys[i];
    if (radix_sort_u64(keys, k, 32 + scale)) { free(keys); return -1; }
    uint64_t out = 0;
    for (uint64_t i = 0; i < k; i++) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        if (out >= cap) { free(keys); return -1; }
        eu[out] = (uint32_t)(keys[i] >> 32); ev[out] = (uint32_t)keys[i]; out++;
    }
    free(keys);
    return (int64_t)out;
}

/* Small R-MAT for the mixed batch: scale = ceil(log2 n), ids >= n rejected,
 * draws continue until m distinct non-loop pairs exist or max_draws draws
 * were made.  Endpoints are in drawn order.  Returns the edge count. */
int64_t gen_rmat_small(uint32_t n, uint64_t m, double a, double b, double c, uint64_t seed,
                       uint64_t max_draws, uint32_t* eu, uint32_t* ev) {
    if (n < 2) return 0;
    int scale = 0;
    while ((1ULL << scale) < n) scale++;
    pairset s;
    if (ps_init(&s, m)) return -1;
    uint64_t k = 0;
    for (uint64_t e = 0; e < max_draws && k < m; e++) {
        uint32_t u, v;
        rmat_edge(scale, a, a + b, a + b + c, seed, e, &u, &v);
        if (u >= n || v >= n || u == v) continue;
        if (!ps_insert(&s, canon(u, v))) continue;
        eu[k] = u; ev[k] = v; k++;
    }
    ps_free(&s);
    return (int64_t)k;
}

/* Weights: w[i] = (draw_i >> 40) * 2^-24, exact in float32 and in [0,1);
 * unit != 0 gives all-ones weights instead. */
void gen_weights(uint64_t m, uint64_t seed, int unit, float* w) {
    for (uint64_t i = 0; i < m; i++)
        w[i] = unit ? 1.0f : (float)((double)(sx_at(seed, i) >> 40) * (1.0 / 16777216.0));
}

/* Fill out[i] = sx_at(seed, i) for i < count (parameter draws for the mixed
 * batch and the request stream are taken from these on the Python side). */
void gen_draws(uint64_t seed, uint64_t count, uint64_t* out) {
    for (uint64_t i = 0; i < count; i++) out[i] = sx_at(seed, i);
}
