"""The perturbation renewed in every round (LM_F_RENEW; the footnote to Lemma 1
in Sec. 2): round r orders edges by weight, ties broken by the seeded
permutation of the r-th SplitMix64 output.  mate[], the number of rounds and
the per-round live edge and vertex counts equal the oracle's sequential local
max with renewal, on both launch paths, alone and batched; with distinct
weights the order does not depend on the permutation, so the result is the
greedy matching."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import NIL, Lm

pytestmark = pytest.mark.gpu

RMAX, CHUNK, TILE = 1024, 1024, 1024


@pytest.fixture(scope="module", params=[False, True], ids=["graph", "stream"])
def rn(request):
    c = Lm(profile=request.param, renew=True)
    yield c
    c.close()


def _want(g, seed):
    return oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed, renew=True)


def _check(L, g, seed):
    mate, st = L.match(g, seed)
    want, r, rm, rn_ = _want(g, seed)
    assert np.array_equal(mate, want), g.name
    assert st["matched"] == int((want != NIL).sum()) // 2
    assert st["rounds"] == r, (g.name, st["rounds"], r)
    k = min(r, 64)
    assert st["round_m"][:k] == [int(x) for x in rm[:k]]
    assert st["round_n"][:k] == [int(x) for x in rn_[:k]]
    return mate


def _unit_stars(sizes):
    eu, ev, base, centres = [], [], 0, []
    for k in sizes:
        centres.append(base)
        eu.append(np.full(k, base, np.uint32))
        ev.append(np.arange(base + 1, base + k + 1, dtype=np.uint32))
        base += k + 1
    c = np.array(centres, np.uint32)
    eu.append(c[:-1])
    ev.append(c[1:])
    eu, ev = np.concatenate(eu), np.concatenate(ev)
    return synth.Graph(base, eu, ev, np.ones(eu.shape[0], np.float32), "unit_stars")


@pytest.mark.parametrize("which", ["er_unit", "grid_unit", "rmat_unit", "two_weights", "stars"])
def test_tied_weights(rn, which):
    if which == "er_unit":
        g, seeds = synth.er(10_000, 50_000, seed=1, unit=True), (1, 101)
    elif which == "grid_unit":
        g, seeds = synth.grid(256, 256, 0.05, seed=2, unit=True), (2, 3)
    elif which == "rmat_unit":
        g0 = synth.rmat(scale=14, edge_factor=16, seed=3)
        g, seeds = synth.Graph(g0.n, g0.eu, g0.ev, np.ones(g0.m, np.float32), "rmat14_unit"), (5,)
    elif which == "two_weights":
        g0 = synth.er(20_000, 120_000, seed=9)
        w = np.where(g0.w < 0.5, 1.0, 2.0).astype(np.float32)
        g, seeds = synth.Graph(g0.n, g0.eu, g0.ev, w, "er_two_weights"), (7,)
    else:
        # rows around the short-row limit, the chunk size and the tile size, all ties
        g, seeds = _unit_stars([RMAX - 1, RMAX, RMAX + 1, CHUNK, CHUNK + 1, 2 * CHUNK + 1, TILE + 1, 3 * TILE]), (4, 8)
    for seed in seeds:
        _check(rn, g, seed)


def test_renewal_changes_tied_results(rn):
    g = synth.er(4000, 20_000, seed=11, unit=True)
    d = Lm()
    try:
        differ = 0
        for seed in range(1, 6):
            a = _check(rn, g, seed)
            b, _ = d.match(g, seed)
            assert np.array_equal(b, oracle.greedy(g.n, g.eu, g.ev, g.w, seed))
            differ += int(not np.array_equal(a, b))
        assert differ > 0
    finally:
        d.close()


def test_distinct_weights_give_the_greedy_matching(rn):
    n, m = 30_000, 150_000
    g0 = synth.er(n, m, seed=12)
    # distinct weights: a random permutation of 1..m (exact in float32)
    w = (synth.draws(13, m).argsort().argsort() + 1).astype(np.float32)
    g = synth.Graph(n, g0.eu, g0.ev, w, "er_distinct")
    mate = _check(rn, g, 21)
    assert np.array_equal(mate, oracle.greedy(g.n, g.eu, g.ev, g.w, 21))


def test_batch(rn):
    lm = rn.lm
    gs = [synth.er(3000 + 500 * i, 12_000 + 3000 * i, seed=30 + i, unit=True) for i in range(5)]
    gs.append(_unit_stars([RMAX + 1, CHUNK + 1, 5]))
    hs = [rn.graph(g) for g in gs]
    try:
        seeds = [100 + i for i in range(len(gs))]
        mates = [rn.torch.empty(g.n, dtype=rn.torch.int32, device="cuda") for g in gs]
        out, stats = lm.lm_batch_match(rn.ctx, hs, seeds, mates, stats=True)
        for g, s, mt, st in zip(gs, seeds, out, stats):
            want, r, _, _ = _want(g, s)
            got = mt.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want), g.name
            assert st["rounds"] == r
    finally:
        for h in hs:
            lm.lm_graph_destroy(h)


def test_tuning_keeps_the_order(rn):
    lm = rn.lm
    keep = lm.lm_get_tuning(rn.ctx)
    try:
        lm.lm_set_tuning(rn.ctx, rmax=64, chunk=1024)
        _check(rn, synth.er(8000, 60_000, seed=14, unit=True), 3)
    finally:
        lm.lm_set_tuning(rn.ctx, **{k: keep[k] for k in ("rmax", "chunk", "sweep_ctas_per_sm", "vertex_ctas_per_sm",
                                                          "batch")})


def test_serving_and_edge_centric_refuse_renewal(rn):
    lm = rn.lm
    g = synth.er(100, 300, seed=15, unit=True)
    h = rn.graph(g)
    try:
        mate = rn.torch.empty(g.n, dtype=rn.torch.int32, device="cuda")
        with pytest.raises(lm.LmError) as ei:
            lm.lm_submit(rn.ctx, h, 1, mate)
        assert ei.value.code == lm.LM_EINVAL
    finally:
        lm.lm_graph_destroy(h)
    with pytest.raises(lm.LmError) as ei:
        lm.lm_create(0, None, flags=lm.LM_F_RENEW | lm.LM_F_EDGE_CENTRIC)
    assert ei.value.code == lm.LM_EINVAL
