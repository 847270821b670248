"""The edge-centric path (LM_F_EDGE_CENTRIC: the Combining CRCW formulation of
Sec. 2, atomic maxima per edge instead of segmented maxima per row) through the
C ABI: mate[] bit-exact with the oracle and the per-round live edge and vertex
counts equal to the sequential algorithm's, on both launch paths."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import NIL, Lm
from helpers import load_hand_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[False, True], ids=["graph", "stream"])
def ec(request):
    c = Lm(profile=request.param, edge_centric=True)
    yield c
    c.close()


def _check(L, g, seed):
    mate, st = L.match(g, seed)
    want = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
    assert np.array_equal(mate, want), g.name
    assert st["matched"] == int((want != NIL).sum()) // 2
    if g.m:
        _, r, rm, rn = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed)
        assert st["rounds"] == r
        k = min(r, 64)
        assert st["round_m"][:k] == [int(x) for x in rm[:k]]
        assert st["round_n"][:k] == [int(x) for x in rn[:k]]


@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(ec, case):
    g = synth.Graph(case["n"], case["eu"], case["ev"], case["w"], case["name"])
    for seed in (0, 101):
        mate, st = ec.match(g, seed)
        assert mate.tolist() == case["mate"].tolist()
        assert st["rounds"] == case["rounds"]
        _check(ec, g, seed)


@pytest.mark.parametrize("which", ["er", "er_unit", "grid", "rmat", "hubs", "path"])
def test_workloads(ec, which):
    if which == "er":
        g, seed = synth.er(10_000, 50_000, seed=1), 101
    elif which == "er_unit":
        g, seed = synth.er(10_000, 50_000, seed=1, unit=True), 101
    elif which == "grid":
        g, seed = synth.grid(256, 256, 0.05, seed=2), 102
    elif which == "rmat":
        g, seed = synth.rmat(scale=14, edge_factor=16, seed=3), 103
    elif which == "hubs":
        n = 20_000
        eu = np.concatenate([np.zeros(9000, np.uint32), np.ones(9000, np.uint32)])
        ev = np.concatenate([np.arange(2, 9002, dtype=np.uint32), np.arange(9002, 18002, dtype=np.uint32)])
        g, seed = synth.Graph(n, eu, ev, synth.weights(eu.shape[0], 4), "two_hubs"), 4
    else:
        n = 2001
        eu = np.arange(n - 1, dtype=np.uint32)
        g, seed = synth.Graph(n, eu, eu + 1, (np.arange(n - 1) + 1).astype(np.float32), "mono_path"), 1
    _check(ec, g, seed)


def test_edgeless_graph(ec):
    g = synth.Graph(9, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32), "edgeless")
    mate, st = ec.match(g, 1)
    assert (mate == NIL).all() and st["rounds"] == 0


def test_same_result_as_the_segmented_path():
    seg, edge = Lm(), Lm(edge_centric=True)
    try:
        g = synth.rmat(scale=16, edge_factor=16, seed=8)
        a, sa = seg.match(g, 77)
        b, sb = edge.match(g, 77)
        assert np.array_equal(a, b)
        assert (sa["rounds"], sa["round_m"], sa["round_n"]) == (sb["rounds"], sb["round_m"], sb["round_n"])
    finally:
        seg.close()
        edge.close()
