/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously correct CPU code for what the local-max matching
 * path computes.  Only the tests, the smoke check and the benchmark's CPU
 * baseline and reference legs may load this file's library; the product path
 * never does.  It
 * shares no code with the CUDA library: the edge order, the permutation and
 * both matching algorithms below are written out here on their own.
 *
 * Functions and the passages they follow ("Efficient Parallel and External
 * Matching", Birn, Osipov, Sanders, Schulz, Sitchinava):
 *
 *   lmo_ord, lmo_perm, lmo_key   -- the strict total order on edges that
 *       replaces "weight, ties broken by random perturbation" (Sec. 1, the
 *       local max algorithm; Sec. 2, sequential model).  Reading: weight
 *       first, then a seeded bijective permutation of the edge index; the
 *       perturbation is drawn once per call and never renewed.
 *   lmo_greedy  -- the greedy algorithm of Sec. 3 (sort by decreasing
 *       weight, scan, take an edge when both ends are free).  For a strict
 *       total order fixed for the whole run, local max selects exactly this
 *       matching; this is the oracle for the GPU's mate[].
 *   lmo_seq_local_max -- the three-pass sequential local max of Sec. 2
 *       ("Sequential Model"), iteration by iteration, recording the live edge
 *       and live vertex counts at the start of every iteration;
 *       lmo_seq_local_max_renew the same with the perturbation renewed in
 *       every iteration (Sec. 2, the footnote to Lemma 1).
 *   lmo_brute_mwm -- maximum weight matching by exhaustive dynamic
 *       programming over vertex subsets (small n only), for the
 *       1/2-approximation property cited in Sec. 1.
 *   lmo_contract -- contraction of a matching, the step that multilevel
 *       graph partitioning repeats on maximal matchings (Sec. 1).  Reading
 *       (the paper names the use, not the operation): a matched pair
 *       becomes one coarse vertex and an unmatched vertex stays alone;
 *       coarse ids follow the smaller member's index; a coarse vertex
 *       weighs the sum of its members; edges inside a pair vanish; the
 *       original edges between two coarse vertices become one coarse edge,
 *       oriented and placed as the first of them in the input order, whose
 *       weight is their sum (taken in double, rounded to float32 once).
 *
 * Floating point: edge weights arrive as float32 (the input format); the
 * order only reinterprets their bits; sums of weights are taken in double.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LMO_NIL 0xFFFFFFFFu

/* ---- the order ------------------------------------------------------ */

/* Monotone map from non-NaN float32 to uint32: a < b  <=>  ord(a) < ord(b).
 * -0.0 is first made +0.0 so the two zeros compare equal, as floats do.
 * Non-negative floats get the sign bit set; negative floats are bit-inverted
 * so that larger magnitudes come first.  Every non-NaN float maps to a value
 * >= 0x007FFFFF (the image of -inf), so a key of 0 is below every edge. */
uint32_t lmo_ord(float w) {
    uint32_t b;
    memcpy(&b, &w, 4);
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

/* MurmurHash3 32-bit finaliser (Appleby, public domain): a bijection on 32 bits. */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* SplitMix64 (Steele, Lea, Flood 2014): first output for state `seed`. */
uint64_t lmo_splitmix64(uint64_t seed) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint32_t lmo_fmix32(uint32_t h) { return fmix32(h); }

/* perm_seed(e) = fmix32(fmix32(e ^ k0) ^ k1), (k0, k1) = low, high half of
 * SplitMix64(seed).  Each stage is a bijection, hence so is perm_seed. */
uint32_t lmo_perm(uint64_t seed, uint32_t e) {
    uint64_t z = lmo_splitmix64(seed);
    uint32_t k0 = (uint32_t)z, k1 = (uint32_t)(z >> 32);
    return fmix32(fmix32(e ^ k0) ^ k1);
}

/* inverse of x -> x * a (a odd) modulo 2^32, by Newton iteration */
static uint32_t inv_odd(uint32_t a) {
    uint32_t x = a;                 /* correct to 3 bits */
    for (int i = 0; i < 5; i++) x *= 2u - a * x;
    return x;
}
/* inverse of h ^= h >> s */
static uint32_t unxorshift(uint32_t h, int s) {
    uint32_t x = h;
    for (int k = s; k < 32; k += s) x = h ^ (x >> s);
    return x;
}
static uint32_t fmix32_inv(uint32_t h) {
    h = unxorshift(h, 16);
    h *= inv_odd(0xC2B2AE35u);
    h = unxorshift(h, 13);
    h *= inv_odd(0x85EBCA6Bu);
    h = unxorshift(h, 16);
    return h;
}
uint32_t lmo_perm_inv(uint64_t seed, uint32_t x) {
    uint64_t z = lmo_splitmix64(seed);
    uint32_t k0 = (uint32_t)z, k1 = (uint32_t)(z >> 32);
    return fmix32_inv(fmix32_inv(x) ^ k1) ^ k0;
}

/* K(e) = ord(w_e) * 2^32 + perm_seed(e): larger key = heavier edge. */
uint64_t lmo_key(float w, uint64_t seed, uint32_t e) {
    return ((uint64_t)lmo_ord(w) << 32) | lmo_perm(seed, e);
}

void lmo_keys(uint64_t m, const float* w, uint64_t seed, uint64_t* out) {
    for (uint64_t e = 0; e < m; e++) out[e] = lmo_key(w[e], seed, (uint32_t)e);
}

/* ---- greedy (Sec. 3) ------------------------------------------------ */

typedef struct { uint64_t key; uint32_t e; } kv;

static int by_key_desc(const void* a, const void* b) {
    uint64_t x = ((const kv*)a)->key, y = ((const kv*)b)->key;
    return x < y ? 1 : (x > y ? -1 : 0);
}

/* mate[v] = partner of v or LMO_NIL.  Returns the number of matched edges,
 * or -1 on allocation failure. */
int64_t lmo_greedy(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev,
                   const float* w, uint64_t seed, uint32_t* mate) {
    kv* order = (kv*)malloc((m ? m : 1) * sizeof(kv));
    if (!order) return -1;
    for (uint64_t e = 0; e < m; e++) { order[e].key = lmo_key(w[e], seed, (uint32_t)e); order[e].e = (uint32_t)e; }
    qsort(order, m, sizeof(kv), by_key_desc);
    for (uint32_t v = 0; v < n; v++) mate[v] = LMO_NIL;
    int64_t taken = 0;
    for (uint64_t i = 0; i < m; i++) {
        uint32_t e = order[i].e, a = eu[e], b = ev[e];
        if (mate[a] == LMO_NIL && mate[b] == LMO_NIL) { mate[a] = b; mate[b] = a; taken++; }
    }
    free(order);
    return taken;
}

/* ---- sequential local max (Sec. 2, "Sequential Model") -------------- */

/* Iterations run over the remaining edges.  Pass 1: each edge becomes the
 * candidate C[x] of an endpoint x when it beats the current candidate (C
 * starts as a dummy whose key, 0, is below every edge).  Pass 2: an edge that
 * is the candidate of both endpoints enters M.  Pass 3: edges with a matched
 * endpoint leave the graph; the others reset their endpoints' candidates to
 * the dummy.  round_m[r] / round_n[r] receive the live edge count and the live
 * vertex count (unmatched vertices with a remaining edge) at the start of
 * iteration r, for r < max_rounds.  Returns the number of iterations, or -1
 * on allocation failure. */
static int64_t seq_local_max(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev,
                             const float* w, uint64_t seed, int renew, uint32_t* mate,
                             uint64_t* round_m, uint64_t* round_n, uint64_t max_rounds);

int64_t lmo_seq_local_max(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev,
                          const float* w, uint64_t seed, uint32_t* mate,
                          uint64_t* round_m, uint64_t* round_n, uint64_t max_rounds) {
    return seq_local_max(n, m, eu, ev, w, seed, 0, mate, round_m, round_n, max_rounds);
}

/* The same algorithm with the random perturbation renewed in every iteration,
 * as the proof of Lemma 1 assumes (Sec. 2, its footnote): iteration r orders
 * the edges by (weight, perm of the r-th SplitMix64 output of the seed), i.e.
 * lmo_key(w, seed + r * golden_gamma, e); iteration 0 is the unrenewed order. */
int64_t lmo_seq_local_max_renew(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev,
                                const float* w, uint64_t seed, uint32_t* mate,
                                uint64_t* round_m, uint64_t* round_n, uint64_t max_rounds) {
    return seq_local_max(n, m, eu, ev, w, seed, 1, mate, round_m, round_n, max_rounds);
}

static int64_t seq_local_max(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev,
                             const float* w, uint64_t seed, int renew, uint32_t* mate,
                             uint64_t* round_m, uint64_t* round_n, uint64_t max_rounds) {
    uint64_t* key = (uint64_t*)malloc((m ? m : 1) * sizeof(uint64_t));
    uint32_t* live = (uint32_t*)malloc((m ? m : 1) * sizeof(uint32_t));
    uint64_t* cand = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));   /* key of C[v] */
    uint32_t* candE = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));  /* edge of C[v] */
    uint8_t* seen = (uint8_t*)malloc(n ? n : 1);
    if (!key || !live || !cand || !candE || !seen) {
        free(key); free(live); free(cand); free(candE); free(seen); return -1;
    }
    for (uint64_t e = 0; e < m; e++) { key[e] = lmo_key(w[e], seed, (uint32_t)e); live[e] = (uint32_t)e; }
    for (uint32_t v = 0; v < n; v++) { mate[v] = LMO_NIL; cand[v] = 0; candE[v] = LMO_NIL; }
    uint64_t nlive = m, rounds = 0;
    while (nlive > 0) {
        if (rounds < max_rounds) {
            memset(seen, 0, n);
            uint64_t nv = 0;
            for (uint64_t i = 0; i < nlive; i++) {
                uint32_t e = live[i];
                if (!seen[eu[e]]) { seen[eu[e]] = 1; nv++; }
                if (!seen[ev[e]]) { seen[ev[e]] = 1; nv++; }
            }
            round_m[rounds] = nlive;
            round_n[rounds] = nv;
        }
        /* renewed perturbation: this iteration's keys */
        if (renew && rounds > 0)
            for (uint64_t i = 0; i < nlive; i++)
                key[live[i]] = lmo_key(w[live[i]], seed + rounds * 0x9E3779B97F4A7C15ull, live[i]);
        /* pass 1 */
        for (uint64_t i = 0; i < nlive; i++) {
            uint32_t e = live[i];
            if (key[e] > cand[eu[e]]) { cand[eu[e]] = key[e]; candE[eu[e]] = e; }
            if (key[e] > cand[ev[e]]) { cand[ev[e]] = key[e]; candE[ev[e]] = e; }
        }
        /* pass 2 */
        for (uint64_t i = 0; i < nlive; i++) {
            uint32_t e = live[i];
            if (candE[eu[e]] == e && candE[ev[e]] == e) { mate[eu[e]] = ev[e]; mate[ev[e]] = eu[e]; }
        }
        /* pass 3 */
        uint64_t k = 0;
        for (uint64_t i = 0; i < nlive; i++) {
            uint32_t e = live[i];
            if (mate[eu[e]] != LMO_NIL || mate[ev[e]] != LMO_NIL) continue;
            cand[eu[e]] = 0; candE[eu[e]] = LMO_NIL;
            cand[ev[e]] = 0; candE[ev[e]] = LMO_NIL;
            live[k++] = e;
        }
        nlive = k;
        rounds++;
    }
    free(key); free(live); free(cand); free(candE); free(seen);
    return (int64_t)rounds;
}

/* ---- brute-force maximum weight matching ---------------------------- */

/* Exhaustive DP over vertex subsets: best(S) = max( best(S - {i}),
 * max over edges {i,j}, j in S of w + best(S - {i,j}) ), i = lowest
 * vertex of S.  n <= 22.  Parallel edges: all are tried.  Returns the
 * optimum weight (>= 0), or -1 on bad input / allocation failure. */
double lmo_brute_mwm(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev, const float* w) {
    if (n > 22) return -1.0;
    uint64_t states = 1ull << n;
    double* best = (double*)malloc(states * sizeof(double));
    if (!best) return -1.0;
    best[0] = 0.0;
    for (uint64_t S = 1; S < states; S++) {
        uint32_t i = 0;
        while (!((S >> i) & 1ull)) i++;
        uint64_t rest = S & ~(1ull << i);
        double b = best[rest];
        for (uint64_t e = 0; e < m; e++) {
            uint32_t a = eu[e], c = ev[e], j;
            if (a == i) j = c; else if (c == i) j = a; else continue;
            if (j == i || !((rest >> j) & 1ull)) continue;
            double cand = (double)w[e] + best[rest & ~(1ull << j)];
            if (cand > b) b = cand;
        }
        best[S] = b;
    }
    double r = best[states - 1];
    free(best);
    return r;
}


/* ---- contraction of a matching -------------------------------------- */

typedef struct { uint64_t pair; uint32_t e; } lmo_pe;

static int by_pair_then_edge(const void* a, const void* b) {
    const lmo_pe* x = (const lmo_pe*)a;
    const lmo_pe* y = (const lmo_pe*)b;
    if (x->pair != y->pair) return x->pair < y->pair ? -1 : 1;
    return x->e < y->e ? -1 : (x->e > y->e);
}

typedef struct { uint32_t lead, c, d; double sum; } lmo_ce;

static int by_leader(const void* a, const void* b) {
    const lmo_ce* x = (const lmo_ce*)a;
    const lmo_ce* y = (const lmo_ce*)b;
    return x->lead < y->lead ? -1 : (x->lead > y->lead);
}

/* mate: partner or LMO_NIL per vertex (must be a matching of the graph's
 * vertex set: mate[mate[v]] == v).  vw: vertex weights, NULL = 1 each.
 * Outputs: cmap[n] coarse id per vertex, cvw[n'] coarse vertex weights,
 * ceu / cev / cw [m'] coarse edges; *n_out = n', *m_out = m'.
 * Returns 0, -1 on allocation failure, -2 on an invalid mate or endpoint. */
int lmo_contract(uint32_t n, uint64_t m, const uint32_t* eu, const uint32_t* ev, const float* w,
                 const uint32_t* vw, const uint32_t* mate, uint32_t* cmap, uint32_t* cvw,
                 uint32_t* ceu, uint32_t* cev, float* cw, uint32_t* n_out, uint64_t* m_out) {
    for (uint32_t v = 0; v < n; v++) {
        const uint32_t u = mate[v];
        if (u == LMO_NIL) continue;
        if (u >= n || u == v || mate[u] != v) return -2;
    }
    for (uint64_t e = 0; e < m; e++)
        if (eu[e] >= n || ev[e] >= n) return -2;
    /* coarse ids: representatives (unmatched vertices and the smaller end of
       each matched pair) numbered in vertex order */
    uint32_t nc = 0;
    for (uint32_t v = 0; v < n; v++) {
        const uint32_t u = mate[v];
        if (u == LMO_NIL || v < u) cmap[v] = nc++;
    }
    for (uint32_t v = 0; v < n; v++) {
        const uint32_t u = mate[v];
        if (u != LMO_NIL && u < v) cmap[v] = cmap[u];
    }
    for (uint32_t c = 0; c < nc; c++) cvw[c] = 0;
    for (uint32_t v = 0; v < n; v++) cvw[cmap[v]] += vw ? vw[v] : 1u;
    /* crossing edges grouped by their unordered coarse pair, in edge order */
    lmo_pe* pe = (lmo_pe*)malloc((m ? m : 1) * sizeof(lmo_pe));
    lmo_ce* ce = (lmo_ce*)malloc((m ? m : 1) * sizeof(lmo_ce));
    if (!pe || !ce) { free(pe); free(ce); return -1; }
    uint64_t k = 0;
    for (uint64_t e = 0; e < m; e++) {
        const uint32_t c = cmap[eu[e]], d = cmap[ev[e]];
        if (c == d) continue;
        const uint32_t lo = c < d ? c : d, hi = c < d ? d : c;
        pe[k].pair = ((uint64_t)lo << 32) | hi;
        pe[k].e = (uint32_t)e;
        k++;
    }
    qsort(pe, k, sizeof(lmo_pe), by_pair_then_edge);
    uint64_t g = 0;
    for (uint64_t i = 0; i < k;) {
        uint64_t j = i;
        double sum = 0.0;
        while (j < k && pe[j].pair == pe[i].pair) { sum += (double)w[pe[j].e]; j++; }
        const uint32_t lead = pe[i].e;  /* the group's first edge in input order */
        ce[g].lead = lead;
        ce[g].c = cmap[eu[lead]];
        ce[g].d = cmap[ev[lead]];
        ce[g].sum = sum;
        g++;
        i = j;
    }
    qsort(ce, g, sizeof(lmo_ce), by_leader);
    for (uint64_t i = 0; i < g; i++) {
        ceu[i] = ce[i].c;
        cev[i] = ce[i].d;
        cw[i] = (float)ce[i].sum;
    }
    *n_out = nc;
    *m_out = g;
    free(pe);
    free(ce);
    return 0;
}
