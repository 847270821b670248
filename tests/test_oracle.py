"""Pins for the oracle (CPU only).

The oracle is checked against things other than itself: published hash test
vectors, hand-worked matchings, the local-max characterisation checked edge by
edge, the literal sequential algorithm of Sec. 2, an exact maximum weight
matching, and properties the paper states (maximality, the 1/2-approximation,
geometric shrinking of the edge set)."""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import (NIL, dominated, is_matching, is_maximal, load_hand_cases,
                     load_hash_vectors)


# ---------------------------------------------------------------- the order

def test_splitmix64_published_vectors():
    seqs, _ = load_hash_vectors()
    for state, outs in seqs:
        s = state
        for want in outs:
            assert oracle.splitmix64(s) == want
            s = (s + 0x9E3779B97F4A7C15) & (2**64 - 1)


def test_fmix32_published_vectors():
    _, fm = load_hash_vectors()
    assert fm
    for x, want in fm:
        assert oracle.fmix32(x) == want


@pytest.mark.parametrize("seed", [0, 1, 101, 2**63 + 12345, 2**64 - 1])
def test_perm_is_a_bijection(seed):
    rng = np.random.default_rng(seed & 0xFFFF)
    xs = [0, 1, 2, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF] + rng.integers(0, 2**32, 2000).tolist()
    for x in xs:
        assert oracle.perm_inv(seed, oracle.perm(seed, x)) == x
        assert oracle.perm(seed, oracle.perm_inv(seed, x)) == x
    # injective on a window (no collisions among 4096 consecutive ids)
    vals = {oracle.perm(seed, e) for e in range(4096)}
    assert len(vals) == 4096


def test_perm_depends_on_seed():
    a = [oracle.perm(1, e) for e in range(64)]
    b = [oracle.perm(2, e) for e in range(64)]
    assert a != b


def test_ord_is_monotone_on_floats():
    rng = np.random.default_rng(7)
    specials = np.array([-np.inf, -3.4e38, -1.0, -1e-38, -1e-45, -0.0, 0.0, 1e-45, 1e-38,
                         0.5, 1.0, 3.4e38, np.inf], dtype=np.float32)
    xs = np.concatenate([specials, rng.standard_normal(300).astype(np.float32),
                         (rng.random(300) * 2 - 1).astype(np.float32) * np.float32(1e-40)])
    ords = [oracle.ord32(float(x)) for x in xs]
    for i in range(len(xs)):
        for j in range(0, len(xs), 7):
            a, b = xs[i], xs[j]
            assert (a < b) == (ords[i] < ords[j]), (a, b)
            assert (a == b) == (ords[i] == ords[j]), (a, b)
    # every key sits above the dummy key 0 (Sec. 2 starts candidates at a dummy edge)
    assert min(ords) == oracle.ord32(-np.inf) == 0x007FFFFF
    assert oracle.ord32(-0.0) == oracle.ord32(0.0)


def test_key_layout():
    # K(e) = ord(w) << 32 | perm(e): weight decides, the permutation breaks ties
    assert oracle.key(0.5, 9, 3) >> 32 == oracle.ord32(0.5)
    assert oracle.key(0.5, 9, 3) & 0xFFFFFFFF == oracle.perm(9, 3)
    assert oracle.key(0.75, 9, 0) > oracle.key(0.5, 9, 1)
    ks = oracle.keys(np.array([0.5, 0.75, -1.0], np.float32), 9)
    assert [int(k) for k in ks] == [oracle.key(0.5, 9, 0), oracle.key(0.75, 9, 1), oracle.key(-1.0, 9, 2)]


# ---------------------------------------------------------------- hand-worked cases

@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(case):
    for seed in (0, 101, 2**40 + 3):
        g = oracle.greedy(case["n"], case["eu"], case["ev"], case["w"], seed)
        assert g.tolist() == case["mate"].tolist()
        s, rounds, rm, rn = oracle.seq_local_max(case["n"], case["eu"], case["ev"], case["w"], seed)
        assert s.tolist() == case["mate"].tolist()
        assert rounds == case["rounds"]
        assert rm[0] == len(case["eu"])


def test_unit_triangle_takes_top_permuted_edge():
    eu = np.array([0, 1, 0], np.uint32)
    ev = np.array([1, 2, 2], np.uint32)
    w = np.ones(3, np.float32)
    for seed in range(20):
        top = max(range(3), key=lambda e: oracle.perm(seed, e))
        mate = oracle.greedy(3, eu, ev, w, seed)
        a, b = int(eu[top]), int(ev[top])
        assert mate[a] == b and mate[b] == a
        assert mate[3 - a - b] == NIL


def test_unit_even_cycle_follows_perm_order():
    # unit-weight 8-cycle: the first edge taken is the one with the largest
    # permuted id; the result is a perfect or near-perfect maximal matching
    n = 8
    eu = np.arange(n, dtype=np.uint32)
    ev = ((np.arange(n) + 1) % n).astype(np.uint32)
    w = np.ones(n, np.float32)
    for seed in range(10):
        mate = oracle.greedy(n, eu, ev, w, seed)
        top = max(range(n), key=lambda e: oracle.perm(seed, e))
        assert mate[eu[top]] == ev[top]
        assert is_matching(n, eu, ev, mate) and is_maximal(eu, ev, mate)
        assert dominated(eu, ev, oracle.keys(w, seed), mate)


def test_star_unit_weights_centre_takes_top_perm():
    n = 9
    eu = np.zeros(n - 1, np.uint32)
    ev = np.arange(1, n, dtype=np.uint32)
    w = np.ones(n - 1, np.float32)
    for seed in range(10):
        top = max(range(n - 1), key=lambda e: oracle.perm(seed, e))
        mate = oracle.greedy(n, eu, ev, w, seed)
        assert mate[0] == ev[top]
        assert (mate[1:] != NIL).sum() == 1


# ---------------------------------------------------------------- invariants and equivalence

def _small_graphs():
    out = []
    for seed in range(40):
        n = 2 + seed % 23
        m = (seed * 7) % 60
        kind = ("uniform", "unit", "few", "signed")[seed % 4]
        out.append(synth.pairs(n, m, seed, kind))
    out.append(synth.er(200, 900, 5))
    out.append(synth.er(200, 900, 5, unit=True))
    out.append(synth.grid(12, 9, seed=3))
    out.append(synth.grid(12, 9, seed=3, unit=True))
    return out


@pytest.mark.parametrize("g", _small_graphs(), ids=lambda g: g.name)
def test_greedy_equals_sequential_local_max(g):
    for seed in (0, 77):
        a = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
        b, rounds, rm, rn = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed)
        assert a.tolist() == b.tolist()
        assert is_matching(g.n, g.eu, g.ev, a)
        assert is_maximal(g.eu, g.ev, a)
        assert dominated(g.eu, g.ev, oracle.keys(g.w, seed), a)
        if g.m:
            assert rm[0] == g.m and (np.diff(rm.astype(np.int64)) < 0).all()
            assert (rn <= g.n).all()


def test_half_approximation_small_graphs():
    # Sec. 1: the local max / greedy family is a 1/2-approximation of maximum weight
    checked = 0
    for seed in range(120):
        n = 2 + seed % 11          # n <= 12
        m = 1 + (seed * 5) % 30
        g = synth.pairs(n, m, 1000 + seed, "few" if seed % 3 == 0 else "uniform")
        mate = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
        # weight of M: the heaviest (by key) edge between each matched pair
        ks = oracle.keys(g.w, seed)
        best = {}
        for i in range(g.m):
            a, b = int(g.eu[i]), int(g.ev[i])
            if mate[a] == b:
                p = (min(a, b), max(a, b))
                if p not in best or ks[i] > ks[best[p]]:
                    best[p] = i
        got = sum(float(g.w[i]) for i in best.values())
        opt = oracle.brute_mwm(g.n, g.eu, g.ev, g.w)
        assert got >= 0.5 * opt - 1e-9
        assert got <= opt + 1e-9
        checked += 1
    assert checked == 120


def test_brute_mwm_known_values():
    # path of weights 1,3,2 -> 3 ; path 3,1,2 -> 5 ; a 4-cycle 1,1,1,1 -> 2
    f = lambda eu, ev, w: oracle.brute_mwm(4, np.array(eu, np.uint32), np.array(ev, np.uint32),
                                           np.array(w, np.float32))
    assert f([0, 1, 2], [1, 2, 3], [1, 3, 2]) == 3.0
    assert f([0, 1, 2], [1, 2, 3], [3, 1, 2]) == 5.0
    assert f([0, 1, 2, 3], [1, 2, 3, 0], [1, 1, 1, 1]) == 2.0
    # greedy is only 1/2-optimal here: path 1,1.01... -> greedy 1.01... vs optimum 2
    assert f([0, 1, 2], [1, 2, 3], [1, 1.5, 1]) == 2.0


def test_round_count_is_logarithmic_on_generated_graphs():
    # Sec. 2: with random weights the edge set shrinks geometrically
    for g in (synth.er(), synth.grid(64, 64, seed=2), synth.rmat(scale=12, seed=3)):
        _, rounds, rm, _ = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, 101)
        assert rounds <= 3 * math.ceil(math.log2(g.m + 1)) + 4, (g.name, rounds)


def test_unit_weight_rounds_remove_at_least_half():
    # Lemma (unit weights): each iteration removes at least half the edges in
    # expectation; in practice about a quarter survives (Sec. 2 footnote).
    g = synth.er(20000, 100000, 8, unit=True)
    _, rounds, rm, _ = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, 5)
    rm = rm.astype(np.float64)
    surv = rm[1:].sum() / rm[:-1].sum()
    assert surv < 0.5
    assert rm[1] / rm[0] < 0.5


def test_monotone_path_needs_linear_rounds():
    n = 41
    eu = np.arange(n - 1, dtype=np.uint32)
    ev = eu + 1
    w = (np.arange(n - 1) + 1).astype(np.float32)
    mate, rounds, rm, _ = oracle.seq_local_max(n, eu, ev, w, 3)
    assert rounds == math.ceil((n - 1) / 2)
    assert mate.tolist() == oracle.greedy(n, eu, ev, w, 3).tolist()


# ---------------------------------------------------------------- the checks have teeth

def test_checks_reject_planted_mistakes():
    """Plant a mistake in a copy of the oracle's answer (ascending instead of
    descending order; a dropped edge) and make sure the checks catch it."""
    g = synth.er(300, 1500, 11)
    seed = 4
    ks = oracle.keys(g.w, seed)
    good = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
    assert dominated(g.eu, g.ev, ks, good)
    # wrong sort direction: greedy on negated weights
    bad = oracle.greedy(g.n, g.eu, g.ev, -g.w, seed)
    assert is_matching(g.n, g.eu, g.ev, bad) and is_maximal(g.eu, g.ev, bad)
    assert not dominated(g.eu, g.ev, ks, bad)
    # a dropped matched edge breaks maximality
    v = int(np.nonzero(good != NIL)[0][0])
    dropped = good.copy()
    dropped[dropped[v]] = NIL
    dropped[v] = NIL
    assert not is_maximal(g.eu, g.ev, dropped)
    # a wrong tie-break (seed) changes the unit-weight answer
    gu = synth.er(300, 1500, 11, unit=True)
    a = oracle.greedy(gu.n, gu.eu, gu.ev, gu.w, 1)
    assert not dominated(gu.eu, gu.ev, oracle.keys(gu.w, 2), a)


# ---- the renewed perturbation (Sec. 2, the footnote to Lemma 1) -------------

def test_renewed_order_changes_nothing_when_weights_are_distinct():
    # ties never reach the permutation, so renewing it cannot change the result:
    # renewed local max = unrenewed local max = greedy (two independent algorithms)
    for seed in (1, 2, 3):
        g0 = synth.er(3000, 12000, seed=40 + seed)
        w = (np.random.default_rng(seed).permutation(g0.m) + 1).astype(np.float32)  # distinct weights
        g = synth.Graph(g0.n, g0.eu, g0.ev, w, "distinct")
        assert len(np.unique(g.w)) == g.m
        a, ra, ma, na = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed, renew=True)
        b, rb, mb, nb = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed)
        assert np.array_equal(a, b) and np.array_equal(a, oracle.greedy(g.n, g.eu, g.ev, g.w, seed))
        assert ra == rb and np.array_equal(ma, mb) and np.array_equal(na, nb)


def test_renewed_order_on_unit_weights():
    diff = 0
    for seed in range(6):
        g = synth.er(2000, 8000, seed=50 + seed, unit=True)
        a, ra, ma, _ = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed, renew=True)
        b, _, mb, _ = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed)
        assert is_matching(g.n, g.eu, g.ev, a) and is_maximal(g.eu, g.ev, a)
        # iteration 0 uses the unrenewed order: the first two live counts agree
        assert ma[0] == mb[0] and ma[1] == mb[1]
        diff += int(not np.array_equal(a, b))
        # Lemma 1 (renewed noise): at least half of the edges leave per iteration in
        # expectation; with this many edges every early iteration does so
        for r in range(min(3, ra - 1)):
            assert ma[r + 1] <= ma[r] / 2 + 3 * np.sqrt(ma[r])
    assert diff > 0  # renewal does change unit-weight results
