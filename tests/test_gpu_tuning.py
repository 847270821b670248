"""Launch parameters (lm_set_tuning / lm_autotune) change speed, never results:
under every setting the CUDA path's mate[] and per-round counts must equal the
oracle's, through the C ABI, on both launch paths."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import Lm, to_u32

pytestmark = pytest.mark.gpu

SETTINGS = [
    (1, 256, 0, 4, 1024),            # every row of two or more entries becomes chunk tasks
    (4, 256, 1, 1, 64),              # tiny tasks, one CTA per SM
    (64, 1024, 3, 2, 0),             # batches of 32 rows, however many entries
    (1024, 1024, 0, 4, 512),         # the defaults
    (2048, 4096, 0, 4, 1024),
    (2048, 4096, 0, 4, 64),          # nearly every row of 64+ entries its own batch
    (1 << 20, 1 << 20, 16, 0, 1 << 20),  # everything in row batches, largest chunk
]


def _stars(sizes, seed):
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
    return synth.Graph(base, eu, ev, synth.weights(eu.shape[0], seed), f"stars{seed}")


def _graphs():
    return [(synth.rmat(scale=12, edge_factor=8, seed=5), 3),
            (synth.grid(64, 64, 0.05, seed=6), 4),
            (synth.er(3000, 12000, seed=7, unit=True), 5),
            (_stars([3, 300, 257, 1025, 5000], 8), 6),
            # rows around batch boundaries of 64 and 1024 entries, 40 of each length
            (_stars([k for k in (63, 64, 65, 1023, 1024, 1025, 1) for _ in range(40)], 9), 7)]


def _check(L, g, seed):
    mate, st = L.match(g, seed)
    want = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
    assert np.array_equal(mate, want), g.name
    _, r, rm, rn = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed)
    assert st["rounds"] == r
    k = min(r, 64)
    assert st["round_m"][:k] == [int(x) for x in rm[:k]]
    assert st["round_n"][:k] == [int(x) for x in rn[:k]]


@pytest.mark.parametrize("profile", [False, True], ids=["graph", "stream"])
@pytest.mark.parametrize("setting", SETTINGS, ids=lambda s: f"r{s[0]}_c{s[1]}_s{s[2]}_v{s[3]}_b{s[4]}")
def test_parity_under_every_setting(profile, setting):
    import paper_1302_4587_gb300 as lm
    L = Lm(profile=profile)
    try:
        lm.lm_set_tuning(L.ctx, *setting)
        got = lm.lm_get_tuning(L.ctx)
        assert (got["rmax"], got["chunk"], got["sweep_ctas_per_sm"], got["vertex_ctas_per_sm"], got["batch"]) == setting
        for g, seed in _graphs():
            _check(L, g, seed)
    finally:
        L.close()


def test_out_of_range_settings_are_rejected():
    import paper_1302_4587_gb300 as lm
    L = Lm()
    try:
        for bad in [(0, 4096, 0, 4), (64, 1000, 0, 4), (64, 128, 0, 4), (64, 1 << 21, 0, 4),
                    (64, 4096, 17, 4), (64, 4096, 0, 5), ((1 << 20) + 1, 4096, 0, 4),
                    (64, 4096, 0, 4, 32), (64, 4096, 0, 4, 1000), (64, 4096, 0, 4, 1 << 21),
                    (64, 4096, 0, 4, 512, 4), (64, 4096, 0, 4, 512, 40)]:
            with pytest.raises(lm.LmError) as ei:
                lm.lm_set_tuning(L.ctx, *bad)
            assert ei.value.code == lm.LM_EINVAL
        assert lm.lm_get_tuning(L.ctx)["rmax"] == 1024  # unchanged
    finally:
        L.close()


def test_autotune_keeps_a_candidate_and_results_stay_exact():
    import torch
    import paper_1302_4587_gb300 as lm
    L = Lm()
    try:
        gs = synth.batch(24, seed=9, n_lo=64, n_hi=4096)
        seeds = [100 + i for i in range(len(gs))]
        hs = [L.graph(g) for g in gs]
        mates = [torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")[:g.n] for g in gs]
        best = lm.lm_autotune(L.ctx, hs, seeds, mates)
        assert (best["rmax"], best["chunk"], best["batch"]) in [(256, 1024, 256), (512, 1024, 256), (1024, 1024, 512),
                                                                (2048, 4096, 1024)]
        assert best["sweep_ctas_per_sm"] in (0, 3) and best["ms"] > 0
        now = lm.lm_get_tuning(L.ctx)
        assert (now["rmax"], now["chunk"], now["sweep_ctas_per_sm"]) == (best["rmax"], best["chunk"],
                                                                       best["sweep_ctas_per_sm"])
        for g, s, m in zip(gs, seeds, mates):
            assert np.array_equal(to_u32(m), oracle.greedy(g.n, g.eu, g.ev, g.w, s)), g.name
        # one graph: the plain path is what gets timed
        best1 = lm.lm_autotune(L.ctx, hs[:1], seeds[:1], mates[:1])
        assert best1["ms"] > 0
        for h in hs:
            lm.lm_graph_destroy(h)
    finally:
        L.close()
