"""Contraction of a matching on the GPU (lm_contract) against the oracle's
contraction: coarse map, vertex weights, edge list (order, orientation) and
weights identical, after the GPU's own matching, for generator weights and
for arbitrary float weights and parallel edges (both sides sum in input
order); several levels of match-and-contract; the edge cases and refusals of
the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import NIL, Lm, to_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lmc():
    c = Lm()
    yield c
    c.close()


def _dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a).view(dt)).cuda()


def _contract(L, n, eu, ev, w, mate, vw=None):
    torch, lm = L.torch, L.lm
    args = [_dev(torch, eu, np.int32), _dev(torch, ev, np.int32), _dev(torch, w, np.float32),
            _dev(torch, mate.astype(np.uint32), np.int32)]
    dvw = _dev(torch, vw.astype(np.uint32), np.int32) if vw is not None else None
    cmap, cvw, ceu, cev, cw = lm.lm_contract(L.ctx, n, *args, vw=dvw)
    return (to_u32(cmap), to_u32(cvw), to_u32(ceu), to_u32(cev), cw.cpu().numpy())


def _same(got, want, exact_w=True):
    names = ["cmap", "cvw", "ceu", "cev", "cw"]
    for i in range(4):
        assert np.array_equal(got[i], want[i]), names[i]
    if exact_w:
        assert np.array_equal(got[4].view(np.uint32), want[4].view(np.uint32)), "cw"
    else:
        gap = np.abs(got[4].astype(np.float64) - want[4].astype(np.float64))
        assert (gap <= np.spacing(np.abs(want[4])).astype(np.float64)).all(), "cw beyond one rounding"


@pytest.mark.parametrize("which", ["er", "er_unit", "grid", "rmat", "hubs"])
def test_parity_after_the_gpu_matching(lmc, which):
    g = {"er": lambda: synth.er(10_000, 50_000, seed=1),
         "er_unit": lambda: synth.er(10_000, 50_000, seed=1, unit=True),
         "grid": lambda: synth.grid(256, 256, 0.05, seed=2),
         "rmat": lambda: synth.rmat(scale=16, edge_factor=16, seed=3),
         "hubs": lambda: synth.rmat(scale=12, edge_factor=64, a=0.7, b=0.1, c=0.1, seed=4)}[which]()
    mate, _ = lmc.match(g, 77)
    assert np.array_equal(mate, oracle.greedy(g.n, g.eu, g.ev, g.w, 77))
    vw = (np.arange(g.n) % 7 + 1).astype(np.uint32)
    for weights in (None, vw):
        got = _contract(lmc, g.n, g.eu, g.ev, g.w, mate, weights)
        _same(got, oracle.contract(g.n, g.eu, g.ev, g.w, mate, weights))


def test_arbitrary_float_weights(lmc):
    # weights over sixty binary orders of magnitude, both signs: the sums are taken in
    # input order on both sides, so they agree bit for bit even where double rounds
    g0 = synth.er(20_000, 120_000, seed=5)
    rng = np.random.default_rng(5)
    w = (rng.standard_normal(g0.m) * np.exp2(rng.integers(-30, 30, g0.m))).astype(np.float32)
    g = synth.Graph(g0.n, g0.eu, g0.ev, w, "er_wide_weights")
    mate, _ = lmc.match(g, 3)
    _same(_contract(lmc, g.n, g.eu, g.ev, g.w, mate), oracle.contract(g.n, g.eu, g.ev, g.w, mate))


def test_parallel_edges_merge_in_input_order(lmc):
    # many parallel copies of a few pairs with weights whose double sum depends on the order
    rng = np.random.default_rng(8)
    n = 40
    eu = rng.integers(0, n, 5000).astype(np.uint32)
    ev = ((eu + 1 + rng.integers(0, 5, 5000)) % n).astype(np.uint32)
    w = (rng.standard_normal(5000) * np.exp2(rng.integers(-40, 40, 5000))).astype(np.float32)
    mate = np.full(n, NIL, np.uint32)
    for a in range(0, n, 4):
        mate[a], mate[a + 1] = a + 1, a
    _same(_contract(lmc, n, eu, ev, w, mate), oracle.contract(n, eu, ev, w, mate))


def test_multilevel(lmc):
    g = synth.rmat(scale=15, edge_factor=16, seed=6)
    n, eu, ev, w, vw = g.n, g.eu, g.ev, g.w, np.ones(g.n, np.uint32)
    for level in range(5):
        lev = synth.Graph(n, eu, ev, w, f"level{level}")
        mate, _ = lmc.match(lev, 200 + level)
        assert np.array_equal(mate, oracle.greedy(n, eu, ev, w, 200 + level)), level
        got = _contract(lmc, n, eu, ev, w, mate, vw)
        want = oracle.contract(n, eu, ev, w, mate, vw)
        _same(got, want)
        n, vw, eu, ev, w = got[1].shape[0], got[1], got[2], got[3], got[4]
        assert int(vw.sum()) == g.n


def test_edge_cases(lmc):
    # no edges; empty matching (identity); a perfect matching of a small graph
    e0 = np.zeros(0, np.uint32)
    got = _contract(lmc, 5, e0, e0, np.zeros(0, np.float32), np.full(5, NIL, np.uint32))
    assert got[0].tolist() == [0, 1, 2, 3, 4] and got[1].tolist() == [1] * 5 and got[2].shape[0] == 0
    g = synth.er(3000, 12_000, seed=7)
    ident = _contract(lmc, g.n, g.eu, g.ev, g.w, np.full(g.n, NIL, np.uint32))
    assert np.array_equal(ident[2], g.eu) and np.array_equal(ident[3], g.ev) and np.array_equal(ident[4], g.w)
    eu, ev = np.array([0, 1, 2, 3, 0, 1], np.uint32), np.array([1, 2, 3, 0, 2, 3], np.uint32)
    w = np.array([1, 2, 3, 4, 5, 6], np.float32)
    mate = np.array([1, 0, 3, 2], np.uint32)
    _same(_contract(lmc, 4, eu, ev, w, mate), oracle.contract(4, eu, ev, w, mate))


def _contract_offset(L, n, eu, ev, w, mate):
    # the same arrays one element into a device buffer: 4-byte but not 16-byte aligned
    torch, lm = L.torch, L.lm
    def shifted(a, dt):
        b = np.concatenate([np.zeros(1, a.dtype), a])
        return _dev(torch, b, dt)[1:]
    args = [shifted(eu, np.int32), shifted(ev, np.int32), shifted(w, np.float32),
            _dev(torch, mate.astype(np.uint32), np.int32)]
    assert args[0].data_ptr() % 16 != 0
    cmap, cvw, ceu, cev, cw = lm.lm_contract(L.ctx, n, *args)
    return (to_u32(cmap), to_u32(cvw), to_u32(ceu), to_u32(cev), cw.cpu().numpy())


@pytest.mark.parametrize("m", [1, 2, 3, 5, 31, 33, 127, 129, 4095, 4097, 3 * 4096 + 7])
def test_ragged_sizes_and_unaligned_arrays(lmc, m):
    # edge counts around the 4-edge groups, 32-edge words and 4096-item tiles, with
    # parallel edges in both orientations, aligned and one element off
    rng = np.random.default_rng(m)
    n = max(4, m // 3)
    eu = rng.integers(0, n, m).astype(np.uint32)
    ev = ((eu + 1 + rng.integers(0, n - 1, m)) % n).astype(np.uint32)
    k = m // 4
    eu[m - k:], ev[m - k:] = ev[:k], eu[:k]
    w = synth.weights(m, m + 1)
    mate = oracle.greedy(n, eu, ev, w, 5)
    want = oracle.contract(n, eu, ev, w, mate)
    _same(_contract(lmc, n, eu, ev, w, mate), want)
    _same(_contract_offset(lmc, n, eu, ev, w, mate), want)


def test_one_pair_holds_every_edge(lmc):
    # two matched pairs, 10,000 parallel edges between them: one group, summed in input order
    m = 10_000
    rng = np.random.default_rng(9)
    eu = rng.integers(0, 2, m).astype(np.uint32)
    ev = (2 + rng.integers(0, 2, m)).astype(np.uint32)
    sw = rng.random(m) < 0.5
    eu[sw], ev[sw] = ev[sw], eu[sw]
    w = (rng.random(m) * 10 ** rng.uniform(-3, 3, m)).astype(np.float32)
    mate = np.array([1, 0, 3, 2], np.uint32)
    want = oracle.contract(4, eu, ev, w, mate)
    assert want[2].shape[0] == 1
    _same(_contract(lmc, 4, eu, ev, w, mate), want)


def test_groups_around_the_register_walk_limit(lmc):
    # groups of 63, 64, 65 and 66 parallel edges (both orientations, interleaved with
    # other edges): runs of up to 64 equal hashes are settled in registers, longer ones
    # by the pair sort; both must match the oracle
    rng = np.random.default_rng(11)
    n = 2000
    g = synth.er(n, 6000, seed=12)
    eu, ev = [g.eu], [g.ev]
    for j, mult in enumerate((63, 64, 65, 66)):
        a, b = 4 * j, 4 * j + 2          # vertices 4j..4j+3: pairs (4j, 4j+1) and (4j+2, 4j+3) once matched
        x = np.full(mult, a, np.uint32)
        y = np.full(mult, b, np.uint32)
        flip = rng.random(mult) < 0.5
        x[flip], y[flip] = b, a
        eu.append(x)
        ev.append(y)
    eu, ev = np.concatenate(eu), np.concatenate(ev)
    perm = rng.permutation(eu.shape[0])
    eu, ev = eu[perm].astype(np.uint32), ev[perm].astype(np.uint32)
    keep = eu != ev
    eu, ev = eu[keep], ev[keep]
    w = synth.weights(eu.shape[0], 13)
    mate = oracle.greedy(n, eu, ev, w, 3)
    _same(_contract(lmc, n, eu, ev, w, mate), oracle.contract(n, eu, ev, w, mate))
    # the same edges with every vertex in a pair (4j with 4j+1, 4j+2 with 4j+3)
    mate2 = np.arange(n, dtype=np.uint32) ^ 1
    _same(_contract(lmc, n, eu, ev, w, mate2), oracle.contract(n, eu, ev, w, mate2))


def test_refusals(lmc):
    lm, torch = lmc.lm, lmc.torch
    eu = _dev(torch, np.array([0, 1], np.uint32), np.int32)
    ev = _dev(torch, np.array([1, 2], np.uint32), np.int32)
    w = _dev(torch, np.array([1, 2], np.float32), np.float32)
    bad_mates = [np.array([1, 2, NIL], np.uint32), np.array([7, NIL, NIL], np.uint32), np.array([0, NIL, NIL], np.uint32)]
    for bm in bad_mates:
        with pytest.raises(lm.LmError) as ei:
            lm.lm_contract(lmc.ctx, 3, eu, ev, w, _dev(torch, bm, np.int32))
        assert ei.value.code == lm.LM_EINVAL
    with pytest.raises(lm.LmError) as ei:  # endpoint out of range
        lm.lm_contract(lmc.ctx, 2, eu, ev, w, _dev(torch, np.full(2, NIL, np.uint32), np.int32))
    assert ei.value.code == lm.LM_EINVAL
    with pytest.raises(lm.LmError) as ei:  # host memory
        lm.lm_contract(lmc.ctx, 3, eu.cpu(), ev.cpu(), w.cpu(), torch.full((3,), -1, dtype=torch.int32))
    assert ei.value.code == lm.LM_EINVAL


def test_rmat21_full_parity(lmc):
    g = synth.rmat(scale=21, edge_factor=16, seed=3)
    h = lmc.graph(g)
    try:
        mate, _ = lmc.match(g, 103, handle=h)
    finally:
        lmc.lm.lm_graph_destroy(h)
    _same(_contract(lmc, g.n, g.eu, g.ev, g.w, mate), oracle.contract(g.n, g.eu, g.ev, g.w, mate))


def _tuned_bits(L, bits):
    keep = L.lm.lm_get_tuning(L.ctx)
    L.lm.lm_set_tuning(L.ctx, keep["rmax"], keep["chunk"], keep["sweep_ctas_per_sm"], keep["vertex_ctas_per_sm"],
                       keep["batch"], contract_bits=bits)
    assert L.lm.lm_get_tuning(L.ctx)["contract_bits"] == bits
    return keep


@pytest.mark.parametrize("bits", [8, 16, 24, 32])
def test_every_sort_width(lmc, bits):
    # the hash sorted by its low 8, 16, 24 or 32 bits: buckets of thousands of edges
    # (at 8 bits on a million edges, most of them running past a block's chunk) down to
    # runs of one hash; the same contraction every time
    keep = _tuned_bits(lmc, bits)
    try:
        g = synth.rmat(scale=16, edge_factor=16, seed=3)
        mate, _ = lmc.match(g, 19)
        _same(_contract(lmc, g.n, g.eu, g.ev, g.w, mate), oracle.contract(g.n, g.eu, g.ev, g.w, mate))
        h = synth.rmat(scale=12, edge_factor=64, a=0.7, b=0.1, c=0.1, seed=4)  # hub pairs with many parallel edges
        mate = oracle.greedy(h.n, h.eu, h.ev, h.w, 5)
        _same(_contract(lmc, h.n, h.eu, h.ev, h.w, mate), oracle.contract(h.n, h.eu, h.ev, h.w, mate))
        # two levels, the second on a multigraph of summed weights
        cm, cvw, ceu, cev, cw = oracle.contract(h.n, h.eu, h.ev, h.w, mate)
        n2 = int(cvw.shape[0])
        mate2 = oracle.greedy(n2, ceu, cev, cw, 6)
        _same(_contract(lmc, n2, ceu, cev, cw, mate2, cvw), oracle.contract(n2, ceu, cev, cw, mate2, cvw))
    finally:
        lmc.lm.lm_set_tuning(lmc.ctx, keep["rmax"], keep["chunk"], keep["sweep_ctas_per_sm"],
                             keep["vertex_ctas_per_sm"], keep["batch"], contract_bits=keep["contract_bits"])


def test_buckets_longer_than_a_window(lmc):
    # 8 sort bits on 2M crossing edges leave about 8000 edges to every bucket, more than
    # a block's window: every bucket goes to the pair sort
    keep = _tuned_bits(lmc, 8)
    try:
        g = synth.rmat(scale=17, edge_factor=16, seed=7)
        mate = oracle.greedy(g.n, g.eu, g.ev, g.w, 2)
        _same(_contract(lmc, g.n, g.eu, g.ev, g.w, mate), oracle.contract(g.n, g.eu, g.ev, g.w, mate))
    finally:
        lmc.lm.lm_set_tuning(lmc.ctx, keep["rmax"], keep["chunk"], keep["sweep_ctas_per_sm"],
                             keep["vertex_ctas_per_sm"], keep["batch"], contract_bits=keep["contract_bits"])
