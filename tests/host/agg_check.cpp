// Host check of the segmented aggregate carried between sweep tiles
// (lm::Agg / agg_combine in lm_internal.h): random entry sequences are cut
// into random tiles; the tile aggregates, folded with agg_combine in random
// bracketings, must give what a direct walk over the entries gives, and the
// running prefixes must give each tile's output position, compacted row
// count and "open row already has a survivor" flag.
#include <cstdio>
#include <cstdint>
#include <vector>
#include <random>
#include "lm_internal.h"

using namespace lm;

struct Ent { bool start; bool surv; };

// aggregate of entries [a, b) from the definitions
static Agg direct(const std::vector<Ent>& e, size_t a, size_t b) {
    Agg r = agg_identity();
    for (size_t i = a; i < b; i++) r.S += e[i].surv;
    size_t first = b;
    for (size_t i = a; i < b; i++) if (e[i].start) { first = i; break; }
    const bool h = first < b;
    bool hs = false, ts = false;
    for (size_t i = a; i < first; i++) hs |= e[i].surv;
    if (!h) ts = hs;
    else {
        size_t last = first;
        for (size_t i = first; i < b; i++) if (e[i].start) last = i;
        for (size_t i = last; i < b; i++) ts |= e[i].surv;
        for (size_t i = first; i < b;) {
            size_t j = i + 1;
            while (j < b && !e[j].start) j++;
            bool any = false;
            for (size_t k = i; k < j; k++) any |= e[k].surv;
            r.nr += any;
            i = j;
        }
    }
    r.f = (h ? F_H : 0u) | (hs ? F_HS : 0u) | (ts ? F_TS : 0u);
    return r;
}

static bool same(const Agg& x, const Agg& y) { return x.S == y.S && x.nr == y.nr && x.f == y.f; }

static Agg fold(const std::vector<Agg>& v, size_t a, size_t b, std::mt19937_64& rng) {
    if (b - a == 1) return v[a];
    size_t mid = a + 1 + rng() % (b - a - 1);
    return agg_combine(fold(v, a, mid, rng), fold(v, mid, b, rng));
}

int main() {
    std::mt19937_64 rng(12345);
    int bad = 0;
    for (int iter = 0; iter < 50000 && !bad; iter++) {
        size_t n = 1 + rng() % 70;
        std::vector<Ent> e(n);
        const int pstart = 2 + rng() % 6, psurv = 1 + rng() % 4;
        for (size_t i = 0; i < n; i++) {
            e[i].start = (i == 0) || (rng() % pstart == 0);
            e[i].surv = rng() % psurv == 0;
        }
        std::vector<size_t> cuts{0};
        for (size_t i = 1; i < n; i++) if (rng() % 5 == 0) cuts.push_back(i);
        cuts.push_back(n);
        std::vector<Agg> tiles;
        for (size_t t = 0; t + 1 < cuts.size(); t++) tiles.push_back(direct(e, cuts[t], cuts[t + 1]));
        const Agg all = direct(e, 0, n);
        for (int rep = 0; rep < 3; rep++)
            if (!same(fold(tiles, 0, tiles.size(), rng), all)) { bad = 1; break; }
        // running prefixes seen by each tile (the first tile starts from the empty prefix with H)
        Agg P = agg_identity();
        P.f = F_H;
        for (size_t t = 0; t + 1 < cuts.size(); t++) {
            if (cuts[t] > 0) {
                const Agg d = direct(e, 0, cuts[t]);
                // S, compacted rows so far, and whether the open row has a survivor
                if (P.S != d.S || P.nr != d.nr || ((P.f & F_TS) != 0) != ((d.f & F_TS) != 0)) { bad = 2; break; }
            }
            P = agg_combine(P, tiles[t]);
        }
        for (auto& a : tiles)
            if (!same(agg_combine(agg_identity(), a), a) || !same(agg_combine(a, agg_identity()), a)) { bad = 3; break; }
    }
    if (bad) { printf("FAIL %d\n", bad); return 1; }
    printf("OK\n");
    return 0;
}
