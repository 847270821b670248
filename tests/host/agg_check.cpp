// Host check of the segmented aggregate carried between sweep tiles
// (lm::Agg / agg_combine in lm_internal.h): random entry sequences are cut
// into random tiles; the tile aggregates, folded with agg_combine in random
// bracketings, must give what a direct walk over the entries gives.
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <vector>
#include <random>
#include "lm_internal.h"

using namespace lm;

struct Ent { bool start; bool surv; uint64_t key; uint32_t nbr; };

// aggregate of entries [a, b) from the definitions
static Agg direct(const std::vector<Ent>& e, size_t a, size_t b) {
    Agg r = agg_identity();
    for (size_t i = a; i < b; i++) {
        if (e[i].surv) r.S++;
    }
    size_t first = b;
    for (size_t i = a; i < b; i++) if (e[i].start) { first = i; break; }
    r.h = first < b;
    for (size_t i = a; i < first; i++) if (e[i].surv) kv_max(r.hk, r.hu, e[i].key, e[i].nbr);
    if (!r.h) { r.tk = r.hk; r.tu = r.hu; }
    else {
        size_t last = first;
        for (size_t i = first; i < b; i++) if (e[i].start) last = i;
        for (size_t i = last; i < b; i++) if (e[i].surv) kv_max(r.tk, r.tu, e[i].key, e[i].nbr);
        // rows starting inside with a survivor inside
        for (size_t i = first; i < b;) {
            size_t j = i + 1;
            while (j < b && !e[j].start) j++;
            bool any = false;
            for (size_t k = i; k < j; k++) any |= e[k].surv;
            r.nr += any;
            i = j;
        }
    }
    return r;
}

static bool same(const Agg& x, const Agg& y) {
    return x.S == y.S && x.nr == y.nr && x.h == y.h && x.hk == y.hk && x.tk == y.tk &&
           (x.hk == 0 || x.hu == y.hu) && (x.tk == 0 || x.tu == y.tu);
}

static Agg fold(const std::vector<Agg>& v, size_t a, size_t b, std::mt19937_64& rng) {
    if (b - a == 1) return v[a];
    size_t mid = a + 1 + rng() % (b - a - 1);
    return agg_combine(fold(v, a, mid, rng), fold(v, mid, b, rng));
}

int main() {
    std::mt19937_64 rng(12345);
    int bad = 0;
    for (int iter = 0; iter < 20000; iter++) {
        size_t n = 1 + rng() % 60;
        std::vector<Ent> e(n);
        uint64_t key = 1;
        for (size_t i = 0; i < n; i++) {
            e[i].start = (i == 0) || (rng() % 4 == 0);
            e[i].surv = rng() % 3 != 0;
            key += 1 + rng() % 5;
            e[i].key = e[i].surv ? (rng() % 2 ? key : key * 7919u % 100003u + 1) : 0;
            e[i].nbr = (uint32_t)(rng() % 1000);
        }
        // unique keys among survivors (keys are unique per edge in the library)
        for (size_t i = 0; i < n; i++) if (e[i].surv) e[i].key = (e[i].key << 8) | i;
        // cut into tiles
        std::vector<size_t> cuts{0};
        for (size_t i = 1; i < n; i++) if (rng() % 5 == 0) cuts.push_back(i);
        cuts.push_back(n);
        std::vector<Agg> tiles;
        for (size_t t = 0; t + 1 < cuts.size(); t++) {
            Agg a = direct(e, cuts[t], cuts[t + 1]);
            tiles.push_back(a);
        }
        Agg all = direct(e, 0, n);
        for (int rep = 0; rep < 3; rep++) {
            Agg f = fold(tiles, 0, tiles.size(), rng);
            if (!same(f, all)) { bad++; break; }
        }
        // exclusive prefixes seen by each tile: the identity folded left to right
        Agg P = agg_identity();
        P.h = 1;
        for (size_t t = 0; t + 1 < cuts.size(); t++) {
            Agg d = direct(e, 0, cuts[t]);
            if (cuts[t] > 0) {
                if (P.S != d.S || P.nr != d.nr || P.tk != d.tk) { bad++; break; }
            }
            P = agg_combine(P, tiles[t]);
        }
        // identity laws
        for (auto& a : tiles) {
            if (!same(agg_combine(agg_identity(), a), a) || !same(agg_combine(a, agg_identity()), a)) { bad++; break; }
        }
    }
    if (bad) { printf("FAIL %d\n", bad); return 1; }
    printf("OK\n");
    return 0;
}
