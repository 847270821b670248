"""Pins of the oracle's contraction of a matching (the step multilevel graph
partitioning repeats on maximal matchings, Sec. 1): hand-worked cases,
closed forms (an empty matching is the identity), invariants on random
graphs, brute force on tiny inputs (leader edge and pair set recomputed from
scratch, weights summed in exact rational arithmetic)."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

NIL = 0xFFFFFFFF


def _mate(n, pairs):
    m = np.full(n, NIL, np.uint32)
    for a, b in pairs:
        m[a], m[b] = b, a
    return m


def test_path_of_two_pairs():
    # path 0-1-2-3, pairs {0,1}, {2,3}: one crossing edge (1,2) joins the two coarse vertices
    cmap, cvw, ceu, cev, cw = oracle.contract(4, [0, 1, 2], [1, 2, 3], [1.0, 3.0, 2.0], _mate(4, [(0, 1), (2, 3)]))
    assert cmap.tolist() == [0, 0, 1, 1] and cvw.tolist() == [2, 2]
    assert ceu.tolist() == [0] and cev.tolist() == [1] and cw.tolist() == [3.0]


def test_triangle_merges_two_edges():
    # triangle, edges e0=(2,0) w=1.5, e1=(1,2) w=2.25, e2=(0,1) w=4; pair {0,1} -> coarse 0, vertex 2 -> coarse 1.
    # e0 and e1 both join the coarse vertices: one edge, placed and oriented as e0 (2 -> 0 becomes 1 -> 0)
    cmap, cvw, ceu, cev, cw = oracle.contract(3, [2, 1, 0], [0, 2, 1], [1.5, 2.25, 4.0], _mate(3, [(0, 1)]))
    assert cmap.tolist() == [0, 0, 1] and cvw.tolist() == [2, 1]
    assert ceu.tolist() == [1] and cev.tolist() == [0] and cw.tolist() == [3.75]


def test_k4_perfect_matching():
    # K4 with pairs {0,2}, {1,3}: the four crossing edges 0-1, 0-3, 1-2, 2-3 become one edge of weight 1+2+4+8
    eu = [0, 0, 0, 1, 1, 2]
    ev = [1, 2, 3, 2, 3, 3]
    w = [1.0, 16.0, 2.0, 4.0, 32.0, 8.0]
    cmap, cvw, ceu, cev, cw = oracle.contract(4, eu, ev, w, _mate(4, [(0, 2), (1, 3)]))
    assert cmap.tolist() == [0, 1, 0, 1] and cvw.tolist() == [2, 2]
    assert ceu.tolist() == [0] and cev.tolist() == [1] and cw.tolist() == [15.0]


def test_star_and_isolated_vertices():
    # star centre 0 with leaves 1..4, centre matched to leaf 3; vertex 5 isolated; vertex weights given
    eu, ev, w = [0, 0, 0, 0], [1, 2, 3, 4], [1.0, 2.0, 3.0, 4.0]
    vw = [10, 1, 2, 3, 4, 7]
    cmap, cvw, ceu, cev, cw = oracle.contract(6, eu, ev, w, _mate(6, [(0, 3)]), vw)
    assert cmap.tolist() == [0, 1, 2, 0, 3, 4]
    assert cvw.tolist() == [13, 1, 2, 4, 7]
    assert list(zip(ceu.tolist(), cev.tolist(), cw.tolist())) == [(0, 1, 1.0), (0, 2, 2.0), (0, 3, 4.0)]


def test_empty_matching_is_the_identity():
    g = synth.er(500, 2000, seed=3)
    cmap, cvw, ceu, cev, cw = oracle.contract(g.n, g.eu, g.ev, g.w, np.full(g.n, NIL, np.uint32))
    assert np.array_equal(cmap, np.arange(g.n)) and (cvw == 1).all()
    assert np.array_equal(ceu, g.eu) and np.array_equal(cev, g.ev) and np.array_equal(cw, g.w)


def test_invalid_matchings_are_rejected():
    with pytest.raises(ValueError):
        oracle.contract(3, [0], [1], [1.0], np.array([1, 2, NIL], np.uint32))   # not symmetric
    with pytest.raises(ValueError):
        oracle.contract(3, [0], [1], [1.0], np.array([5, NIL, NIL], np.uint32))  # out of range
    with pytest.raises(ValueError):
        oracle.contract(3, [0], [7], [1.0], np.full(3, NIL, np.uint32))          # endpoint out of range


def _brute(n, eu, ev, w, mate, vw=None):
    """From scratch, O(m * m'): representatives, pairs, leaders, exact sums."""
    rep = [v if mate[v] == NIL else min(v, int(mate[v])) for v in range(n)]
    reps = sorted(set(rep))
    cid = {r: i for i, r in enumerate(reps)}
    cmap = [cid[rep[v]] for v in range(n)]
    cvw = [0] * len(reps)
    for v in range(n):
        cvw[cmap[v]] += 1 if vw is None else int(vw[v])
    groups = {}
    for e in range(len(eu)):
        c, d = cmap[int(eu[e])], cmap[int(ev[e])]
        if c != d:
            groups.setdefault(frozenset((c, d)), []).append(e)
    edges = []
    for es in groups.values():
        lead = min(es)
        exact = sum(Fraction(float(np.float32(w[e]))) for e in es)
        edges.append((lead, cmap[int(eu[lead])], cmap[int(ev[lead])], np.float32(float(exact))))
    edges.sort()
    return cmap, cvw, edges


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_on_small_graphs(seed):
    # weights on the generator's 2^-24 grid: double sums are exact, so float32(double sum) =
    # float32(exact sum) when the exact sum is representable to within float rounding
    g = synth.er(60, 200, seed=40 + seed, unit=(seed % 3 == 0))
    mate = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
    vw = (np.arange(g.n) % 5 + 1).astype(np.uint32)
    cmap, cvw, ceu, cev, cw = oracle.contract(g.n, g.eu, g.ev, g.w, mate, vw)
    bmap, bvw, bedges = _brute(g.n, g.eu, g.ev, g.w, mate, vw)
    assert cmap.tolist() == bmap and cvw.tolist() == bvw
    assert list(zip(ceu.tolist(), cev.tolist())) == [(c, d) for _, c, d, _ in bedges]
    assert cw.tolist() == [float(x) for _, _, _, x in bedges]


@pytest.mark.parametrize("which", ["er", "grid", "rmat"])
def test_invariants(which):
    g = {"er": lambda: synth.er(20_000, 100_000, seed=5),
         "grid": lambda: synth.grid(128, 128, 0.05, seed=6),
         "rmat": lambda: synth.rmat(scale=14, edge_factor=16, seed=7)}[which]()
    mate = oracle.greedy(g.n, g.eu, g.ev, g.w, 11)
    M = int((mate != NIL).sum()) // 2
    cmap, cvw, ceu, cev, cw = oracle.contract(g.n, g.eu, g.ev, g.w, mate)
    assert cvw.shape[0] == g.n - M and int(cvw.sum()) == g.n
    assert (ceu != cev).all()
    lo, hi = np.minimum(ceu, cev).astype(np.uint64), np.maximum(ceu, cev).astype(np.uint64)
    pairs = (lo << np.uint64(32)) | hi
    assert np.unique(pairs).shape[0] == pairs.shape[0]
    cu, cv = cmap[g.eu], cmap[g.ev]
    cross = cu != cv
    want = np.unique((np.minimum(cu, cv)[cross].astype(np.uint64) << np.uint64(32)) | np.maximum(cu, cv)[cross])
    assert np.array_equal(np.sort(pairs), want)
    # weight conservation: the coarse weights carry the crossing weight (float32 rounding per edge)
    tot = float(np.sum(g.w[cross].astype(np.float64)))
    assert abs(float(np.sum(cw.astype(np.float64))) - tot) <= 1e-6 * max(1.0, tot)
    # coarse edges appear in the order of their first original edge
    first = {}
    for e in np.nonzero(cross)[0]:
        k = (int(min(cu[e], cv[e])) << 32) | int(max(cu[e], cv[e]))
        first.setdefault(k, int(e))
    leads = [first[int(k)] for k in pairs]
    assert leads == sorted(leads)


def test_multilevel():
    g = synth.rmat(scale=13, edge_factor=16, seed=9)
    n, eu, ev, w, vw = g.n, g.eu, g.ev, g.w, np.ones(g.n, np.uint32)
    for level in range(4):
        mate = oracle.greedy(n, eu, ev, w, 100 + level)
        M = int((mate != NIL).sum()) // 2
        cmap, cvw, ceu, cev, cw = oracle.contract(n, eu, ev, w, mate, vw)
        # every level keeps the total vertex weight, loses one vertex and at least one edge per matched pair
        assert M > 0 and int(cvw.sum()) == g.n and cvw.shape[0] == n - M and ceu.shape[0] <= eu.shape[0] - M
        n, eu, ev, w, vw = cvw.shape[0], ceu, cev, cw, cvw
