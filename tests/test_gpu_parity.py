"""Parity of the CUDA path (through the C ABI) with the oracle.

The result of local max under a strict order is unique, so the GPU's mate[]
must equal the oracle's bit for bit; the per-round live edge and vertex
counts must equal those of the sequential algorithm of Sec. 2."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import NIL, Lm, to_u32
from helpers import is_matching, is_maximal, load_hand_cases

pytestmark = pytest.mark.gpu

TILE = 1024   # entries per round-0 tile (TILE0)
CHUNK = 1024  # entries per chunk task of a long row (default tuning)
RMAX = 1024   # longest row handled as part of a row batch (default tuning)
BATCH = 512   # a row batch ends where its entries cross a multiple of this (default tuning)


@pytest.fixture(scope="module")
def lmctx():
    # profiled context: kernels launched one by one on the stream, per-kernel events
    c = Lm(profile=True)
    yield c
    c.close()


@pytest.fixture(scope="module")
def lmgraph():
    # default context: the whole job as one CUDA graph with a device-driven round loop
    # (the launch configuration the benchmark times)
    c = Lm(profile=False)
    yield c
    c.close()


def _check(lmctx, g, seed, rounds=True, device_out=True):
    mate, st = lmctx.match(g, seed, device_out=device_out)
    want = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
    bad = np.nonzero(mate != want)[0]
    assert bad.size == 0, f"{g.name} seed {seed}: {bad.size} vertices differ, first {bad[:5]}"
    if rounds and g.m:
        _, r, rm, rn = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seed)
        assert st["rounds"] == r, (st["rounds"], r)
        k = min(r, 64)
        assert st["round_m"][:k] == [int(x) for x in rm[:k]]
        assert st["round_n"][:k] == [int(x) for x in rn[:k]]
    assert st["matched"] == int((want != NIL).sum()) // 2
    return mate, st


@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases(lmctx, case):
    g = synth.Graph(case["n"], case["eu"], case["ev"], case["w"], case["name"])
    for seed in (0, 101):
        mate, st = _check(lmctx, g, seed)
        assert mate.tolist() == case["mate"].tolist()
        assert st["rounds"] == case["rounds"]


@pytest.mark.parametrize("seed", range(24))
def test_random_small_graphs(lmctx, seed):
    n = 2 + (seed * 37) % 300
    m = (seed * 997) % 3000
    kind = ("uniform", "unit", "few", "signed")[seed % 4]
    g = synth.pairs(n, m, seed, kind)
    _check(lmctx, g, seed * 13 + 1)


def test_host_and_device_outputs_agree(lmctx):
    g = synth.er(3000, 20000, 9)
    a, _ = lmctx.match(g, 5, device_out=True)
    b, _ = lmctx.match(g, 5, device_out=False)
    assert (a == b).all()
    h = lmctx.graph(g, device=False)
    try:
        c, _ = lmctx.match(g, 5, handle=h)
    finally:
        lmctx.lm.lm_graph_destroy(h)
    assert (a == c).all()


@pytest.mark.parametrize("m", [1, 31, 33, 255, 257, 4099])
def test_host_upload_in_chunks(lmctx, m):
    # graphs from host arrays go up in eight chunks of a multiple of 32 edges,
    # each chunk's degrees counted as it lands: sizes around that rounding
    g = synth.pairs(max(4, m // 3), m, m, "uniform")
    h = lmctx.graph(g, device=False)
    try:
        mate, _ = lmctx.match(g, 8, handle=h)
    finally:
        lmctx.lm.lm_graph_destroy(h)
    assert np.array_equal(mate, oracle.greedy(g.n, g.eu, g.ev, g.w, 8))


def test_seed_changes_unit_weight_result(lmctx):
    g = synth.er(2000, 8000, 3, unit=True)
    a, _ = _check(lmctx, g, 1)
    b, _ = _check(lmctx, g, 2)
    assert (a != b).any()


@pytest.mark.parametrize("unit", [False, True])
def test_er_config(lmctx, unit):
    g = synth.er(10_000, 50_000, 1, unit=unit)
    mate, st = _check(lmctx, g, 101)
    assert is_matching(g.n, g.eu, g.ev, mate) and is_maximal(g.eu, g.ev, mate)


@pytest.mark.parametrize("unit", [False, True])
def test_grid_config(lmctx, unit):
    g = synth.grid(1024, 1024, 0.05, seed=2, unit=unit)
    assert g.m == 2_199_859
    _check(lmctx, g, 102)


@pytest.mark.parametrize("fam,n,alpha", [("rgg", 1 << 15, 0), ("random", 1 << 13, 4),
                                         ("random", 1 << 13, 16), ("random", 1 << 12, 64)])
@pytest.mark.parametrize("ctx", ["lmctx", "lmgraph"])
def test_paper_sweep_families(request, ctx, fam, n, alpha):
    # the families of the Sec. 3 sweep: random geometric graphs (radius
    # 0.55 sqrt(ln n / n)) and random graphs with alpha n edges, through the
    # profiled launches and through the CUDA graph the benchmark times
    g = synth.rgg(n, 20) if fam == "rgg" else synth.er(n, alpha * n, seed=30)
    assert g.m > 0
    mate, st = _check(request.getfixturevalue(ctx), g, 104)
    assert is_matching(g.n, g.eu, g.ev, mate) and is_maximal(g.eu, g.ev, mate)


def test_rows_spanning_many_tiles(lmctx):
    # a star whose centre row covers ~50 tiles, plus a second hub and a path,
    # so rows start and end at every position relative to tile boundaries
    leaves = 50 * TILE + 17
    n = leaves + 3000
    eu = np.concatenate([np.zeros(leaves, np.uint32), np.full(2000, 1, np.uint32),
                         np.arange(leaves + 1, n - 1, dtype=np.uint32)])
    ev = np.concatenate([np.arange(1, leaves + 1, dtype=np.uint32),
                         np.arange(leaves + 1, leaves + 2001, dtype=np.uint32),
                         np.arange(leaves + 2, n, dtype=np.uint32)])
    for kind in ("uniform", "unit"):
        w = synth.weights(eu.shape[0], 77, unit=(kind == "unit"))
        g = synth.Graph(n, eu, ev, w, f"hubs_{kind}")
        _check(lmctx, g, 3)


@pytest.mark.parametrize("m", [1, TILE // 2 - 1, TILE // 2, TILE // 2 + 1, TILE, 3 * TILE + 5, 7 * TILE // 2])
def test_ragged_tile_tails(lmctx, m):
    g = synth.pairs(max(4, m // 3), m, m, "uniform")
    _check(lmctx, g, 7)


def test_edge_cases(lmctx):
    empty = synth.Graph(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32), "no_edges")
    mate, st = lmctx.match(empty, 1)
    assert (mate == NIL).all() and st["rounds"] == 0
    one = synth.Graph(2, np.array([0], np.uint32), np.array([1], np.uint32), np.array([0.0], np.float32), "one")
    mate, st = lmctx.match(one, 1)
    assert mate.tolist() == [1, 0] and st["rounds"] == 1
    # parallel edges, zero and signed weights, isolated vertices
    eu = np.array([0, 1, 0, 2, 2, 5], np.uint32)
    ev = np.array([1, 0, 1, 3, 3, 6], np.uint32)
    w = np.array([0.0, -0.0, 0.0, np.inf, -np.inf, -1.0], np.float32)
    _check(lmctx, synth.Graph(9, eu, ev, w, "parallel"), 4)


def test_monotone_path_many_rounds(lmctx):
    n = 3001
    eu = np.arange(n - 1, dtype=np.uint32)
    ev = eu + 1
    w = (np.arange(n - 1) + 1).astype(np.float32)
    mate, st = _check(lmctx, synth.Graph(n, eu, ev, w, "mono"), 1)
    assert st["rounds"] == math.ceil((n - 1) / 2)


def test_invalid_inputs_are_rejected(lmctx):
    import paper_1302_4587_gb300 as lm
    bad = [
        (3, [0, 1], [1, 1], [1.0, 2.0]),          # self loop
        (3, [0, 1], [1, 3], [1.0, 2.0]),          # endpoint >= n
        (3, [0, 1], [1, 2], [1.0, float("nan")]),  # NaN weight
    ]
    for n, eu, ev, w in bad:
        with pytest.raises(lm.LmError) as ei:
            lm.lm_graph_create(lmctx.ctx, n, np.array(eu, np.uint32), np.array(ev, np.uint32),
                               np.array(w, np.float32))
        assert ei.value.code == lm.LM_EINVAL
    # the context stays usable
    _check(lmctx, synth.er(100, 300, 2), 1)


def test_batch_equals_alone(lmctx):
    import paper_1302_4587_gb300 as lm
    torch = lmctx.torch
    graphs = synth.batch(count=48, seed=4, n_hi=4096)
    graphs.append(synth.Graph(7, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32), "e"))
    handles = [lmctx.graph(g) for g in graphs]
    try:
        seeds = [1000 + i for i in range(len(graphs))]
        mates = [torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")[: g.n] if i % 3 else
                 np.empty(g.n, np.uint32) for i, g in enumerate(graphs)]
        out, stats = lm.lm_batch_match(lmctx.ctx, handles, seeds, mates, stats=True)
        for i, g in enumerate(graphs):
            want = oracle.greedy(g.n, g.eu, g.ev, g.w, seeds[i])
            got = to_u32(out[i])
            assert (got == want).all(), g.name
            if g.m:
                _, r, _, _ = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seeds[i])
                assert stats[i]["rounds"] == r, g.name
            assert stats[i]["matched"] == int((want != NIL).sum()) // 2
            alone, _ = lmctx.match(g, seeds[i], handle=handles[i])
            assert (alone == got).all()
    finally:
        for h in handles:
            lm.lm_graph_destroy(h)


def test_served_results_equal_alone(lmctx):
    """Continuous batching: requests submitted while others are in flight are
    admitted between rounds; each result equals the graph matched alone."""
    import time
    import paper_1302_4587_gb300 as lm
    torch = lmctx.torch
    srv = Lm(budget=256 << 20)
    try:
        reqs = synth.request_sizes(40, seed=5, m_hi=2e5)
        graphs = [synth.request_graph(k, n, m, s, f"r{i}") for i, (k, n, m, s) in enumerate(reqs)]
        handles = [srv.graph(g) for g in graphs]
        mates, tickets = [], []
        for i, g in enumerate(graphs):
            mt = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")[: g.n] if i % 2 else np.empty(g.n, np.uint32)
            mates.append(mt)
            tickets.append(lm.lm_submit(srv.ctx, handles[i], 50 + i, mt))
            if i % 7 == 0:
                time.sleep(0.002)  # let some rounds run before the next arrivals
        for i, t in enumerate(tickets):
            assert lm.lm_wait(srv.ctx, t, 60_000)
            done, st = lm.lm_poll(srv.ctx, t)
            assert done
            g = graphs[i]
            want = oracle.greedy(g.n, g.eu, g.ev, g.w, 50 + i)
            got = to_u32(mates[i])
            assert (got == want).all(), g.name
            if g.m:
                _, r, _, _ = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, 50 + i)
                assert st["rounds"] == r
            assert st["matched"] == int((want != NIL).sum()) // 2
        with pytest.raises(lm.LmError):
            lm.lm_poll(srv.ctx, tickets[0])  # released
        for h in handles:
            lm.lm_graph_destroy(h)
    finally:
        srv.close()


def _stars(sizes, seed):
    # disjoint stars with the given leaf counts plus a path through their centres
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


def test_row_length_boundaries(lmctx):
    # rows right at the short-row limit, the chunk size and the tile size
    sizes = [RMAX - 2, RMAX - 1, RMAX, RMAX + 1, CHUNK - 1, CHUNK, CHUNK + 1, 2 * CHUNK + 1,
             TILE - 1, TILE, TILE + 1, 3 * TILE, BATCH - 1, BATCH, BATCH + 1, 2047, 2049, 4095, 4097, 8193]
    for seed in (1, 2):
        _check(lmctx, _stars(sizes, seed), seed)


def test_rows_starting_on_tile_boundaries(lmctx):
    # a first row of exactly one tile, so the next rows start on tile boundaries
    g = _stars([TILE - 1, TILE, 2 * TILE - 1, 1, 1, TILE], 5)
    _check(lmctx, g, 9)


@pytest.mark.parametrize("which", ["er", "grid", "hubs", "small"])
def test_graph_launch_path(lmgraph, which):
    """The CUDA-graph path (device-driven loop) against the oracle."""
    if which == "er":
        g, seed = synth.er(10_000, 50_000, seed=1), 101
    elif which == "grid":
        g, seed = synth.grid(256, 256, 0.05, seed=2), 102
    elif which == "hubs":
        g, seed = _stars([3 * TILE + 7, RMAX + 1, CHUNK + 3, 5], 6), 6
    else:
        g, seed = synth.pairs(40, 300, 11, "few"), 11
    _check(lmgraph, g, seed)


@pytest.mark.slow
def test_rmat_scale23_full_parity(lmgraph):
    """The headline workload at full size, in the benchmark's launch
    configuration (one CUDA graph per match), checked against the oracle
    element by element."""
    g = synth.rmat(scale=23, edge_factor=16, seed=3)
    mate, st = lmgraph.match(g, 103)
    want = oracle.greedy(g.n, g.eu, g.ev, g.w, 103)
    bad = np.nonzero(mate != want)[0]
    assert bad.size == 0, f"{bad.size} vertices differ"
    assert st["matched"] == int((want != NIL).sum()) // 2
    assert st["rounds"] <= 3 * math.ceil(math.log2(g.m + 1)) + 4
