"""Asynchronous matches (LM_F_ASYNC): lm_match returns once the match is queued
on the context's stream; after lm_sync every result equals the oracle's, also
when many matches are queued back to back (argument staging reused), mixed
with synchronous batched calls, and when the workspace has to grow.  Host
results and statistics are refused on such a context, as are the flag
combinations it cannot honour."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def actx():
    import torch
    import paper_1302_4587_gb300 as lm
    torch.cuda.init()
    c = lm.lm_create(0, None, flags=lm.LM_F_ASYNC)
    yield lm, torch, c
    lm.lm_destroy(c)


def _dev(torch, lm, ctx, g):
    eu = torch.from_numpy(g.eu.view(np.int32)).cuda()
    ev = torch.from_numpy(g.ev.view(np.int32)).cuda()
    w = torch.from_numpy(g.w).cuda()
    return lm.lm_graph_create(ctx, g.n, eu, ev, w)


def _graphs():
    return [synth.er(10_000, 50_000, seed=1), synth.grid(128, 128, 0.05, seed=2, unit=True),
            synth.rmat(scale=14, edge_factor=16, seed=3), synth.er(300, 1200, seed=4, unit=True),
            synth.Graph(7, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32), "edgeless")]


def test_queued_matches_equal_the_oracle(actx):
    lm, torch, ctx = actx
    gs = _graphs()
    hs = [_dev(torch, lm, ctx, g) for g in gs]
    try:
        jobs = []
        for rep in range(3):
            for i, (g, h) in enumerate(zip(gs, hs)):
                seed = 100 * rep + i
                mate = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")[: g.n]
                lm.lm_match(ctx, h, seed, mate)
                jobs.append((g, seed, mate))
        lm.lm_sync(ctx)
        for g, seed, mate in jobs:
            assert np.array_equal(to_u32(mate), oracle.greedy(g.n, g.eu, g.ev, g.w, seed)), (g.name, seed)
    finally:
        for h in hs:
            lm.lm_graph_destroy(h)


def test_many_queued_matches_of_one_graph(actx):
    lm, torch, ctx = actx
    g = synth.er(4000, 20_000, seed=5, unit=True)
    h = _dev(torch, lm, ctx, g)
    try:
        mates = [torch.empty(g.n, dtype=torch.int32, device="cuda") for _ in range(32)]
        for s, m in enumerate(mates):
            lm.lm_match(ctx, h, s, m)
        lm.lm_sync(ctx)
        for s, m in enumerate(mates):
            assert np.array_equal(to_u32(m), oracle.greedy(g.n, g.eu, g.ev, g.w, s)), s
    finally:
        lm.lm_graph_destroy(h)


def test_mixed_with_batches_and_growth(actx):
    lm, torch, ctx = actx
    small, big = synth.er(2000, 8000, seed=6), synth.rmat(scale=16, edge_factor=16, seed=7)
    hs, hb = _dev(torch, lm, ctx, small), _dev(torch, lm, ctx, big)
    try:
        m1 = torch.empty(small.n, dtype=torch.int32, device="cuda")
        lm.lm_match(ctx, hs, 11, m1)
        mb = [torch.empty(small.n, dtype=torch.int32, device="cuda"), torch.empty(big.n, dtype=torch.int32, device="cuda")]
        lm.lm_batch_match(ctx, [hs, hb], [12, 13], mb)  # synchronous
        m2 = torch.empty(big.n, dtype=torch.int32, device="cuda")
        lm.lm_match(ctx, hb, 14, m2)  # may grow the workspace
        lm.lm_sync(ctx)
        assert np.array_equal(to_u32(m1), oracle.greedy(small.n, small.eu, small.ev, small.w, 11))
        assert np.array_equal(to_u32(mb[0]), oracle.greedy(small.n, small.eu, small.ev, small.w, 12))
        assert np.array_equal(to_u32(mb[1]), oracle.greedy(big.n, big.eu, big.ev, big.w, 13))
        assert np.array_equal(to_u32(m2), oracle.greedy(big.n, big.eu, big.ev, big.w, 14))
    finally:
        lm.lm_graph_destroy(hs)
        lm.lm_graph_destroy(hb)


def test_refusals(actx):
    lm, torch, ctx = actx
    g = synth.er(100, 300, seed=8)
    h = _dev(torch, lm, ctx, g)
    try:
        for kwargs in ({"mate": np.empty(g.n, np.uint32)},
                       {"mate": torch.empty(g.n, dtype=torch.int32, device="cuda"), "stats": True}):
            with pytest.raises(lm.LmError) as ei:
                lm.lm_match(ctx, h, 1, **kwargs)
            assert ei.value.code == lm.LM_EINVAL
    finally:
        lm.lm_graph_destroy(h)
    for bad in (lm.LM_F_ASYNC | lm.LM_F_PROFILE, lm.LM_F_ASYNC | lm.LM_F_EDGE_CENTRIC):
        with pytest.raises(lm.LmError) as ei:
            lm.lm_create(0, None, flags=bad)
        assert ei.value.code == lm.LM_EINVAL
    lm.lm_sync(ctx)
