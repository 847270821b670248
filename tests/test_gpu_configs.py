"""The batched and served configurations at their stated sizes, against the oracle.

Under a strict order fixed for the run, local max selects exactly the greedy
matching (Sec. 1 and Sec. 3), so every graph's mate[] must equal the oracle's
bit for bit and its round count the sequential local max's (Sec. 2), however
the graphs share launches.  The oracle runs on a thread pool: its C code
releases the interpreter lock, and each graph is independent."""
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import synth
from gpu_util import NIL, Lm, to_u32

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _oracle_all(graphs, seeds):
    """(greedy mate, sequential local-max rounds) of every graph."""
    def one(i):
        g = graphs[i]
        want = oracle.greedy(g.n, g.eu, g.ev, g.w, seeds[i])
        rounds = oracle.seq_local_max(g.n, g.eu, g.ev, g.w, seeds[i])[1] if g.m else 0
        return want, rounds
    with ThreadPoolExecutor(min(32, os.cpu_count() or 1)) as ex:
        return list(ex.map(one, range(len(graphs))))


def test_batched_config_full_size_equals_oracle():
    """4096 graphs, n log-uniform in [64, 65536], degree U[4, 16], ER / grid /
    R-MAT mixed (gen seed 4, match seeds 1000 + i), in one lm_batch_match with
    the autotuned launch parameters the benchmark uses."""
    import paper_1302_4587_gb300 as lm
    L = Lm()
    torch = L.torch
    graphs = synth.batch(4096, seed=4)
    assert sum(g.m for g in graphs) == 186_438_269 and max(g.n for g in graphs) > 60_000
    seeds = [1000 + i for i in range(len(graphs))]
    handles = [L.graph(g, device=False) for g in graphs]
    try:
        mates = [torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")[: g.n] for g in graphs]
        job = lm.BatchArgs(handles, seeds, mates)
        lm.lm_autotune(L.ctx, job)
        out, stats = lm.lm_batch_match(L.ctx, job, stats=True)
        got = [to_u32(m) for m in out]
        ref = _oracle_all(graphs, seeds)
        bad = [graphs[i].name for i in range(len(graphs)) if not np.array_equal(got[i], ref[i][0])]
        assert not bad, f"{len(bad)} graphs differ from the oracle, first {bad[:5]}"
        wrong_rounds = [i for i in range(len(graphs)) if stats[i]["rounds"] != ref[i][1]]
        assert not wrong_rounds, f"round counts differ for graphs {wrong_rounds[:5]}"
        for i, g in enumerate(graphs):
            assert stats[i]["matched"] == int((ref[i][0] != NIL).sum()) // 2, g.name
    finally:
        for h in handles:
            lm.lm_graph_destroy(h)
        L.close()


def test_served_config_full_size_equals_oracle():
    """The served mix at its stated sizes: edge counts log-uniform in [1e3, 4e6],
    n = m / U[2, 8], ER / grid / R-MAT (gen seed 5), 40 GB admission budget.
    Requests arrive as a Poisson stream near the server's capacity, so most
    are admitted while others are in flight; each pool graph is requested twice
    with different seeds, and every result must equal the oracle's."""
    import paper_1302_4587_gb300 as lm
    L = Lm(budget=40 << 30)
    torch = L.torch
    pool = synth.request_pool(48, seed=5)
    assert max(g.m for g in pool) > 3_000_000
    handles = [L.graph(g, device=False) for g in pool]
    nreq = 2 * len(pool)
    order = [i % len(pool) for i in range(nreq)]
    seeds = [3000 + i for i in range(nreq)]
    arr = synth.arrivals(nreq, 4000.0, seed=6)
    try:
        mates, tickets = [], []
        t0 = time.perf_counter()
        for i in range(nreq):
            while time.perf_counter() - t0 < arr[i]:
                time.sleep(0.00005)
            g = pool[order[i]]
            mt = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")[: g.n] if i % 2 else \
                np.empty(g.n, np.uint32)
            mates.append(mt)
            tickets.append(lm.lm_submit(L.ctx, handles[order[i]], seeds[i], mt))
        stats = []
        for t in tickets:
            assert lm.lm_wait(L.ctx, t, 120_000)
            done, st = lm.lm_poll(L.ctx, t)
            assert done
            stats.append(st)
        ref = _oracle_all([pool[k] for k in order], seeds)
        for i in range(nreq):
            g = pool[order[i]]
            got = to_u32(mates[i])
            assert np.array_equal(got, ref[i][0]), f"request {i} ({g.name}) differs from the oracle"
            assert stats[i]["rounds"] == ref[i][1], g.name
            assert stats[i]["matched"] == int((ref[i][0] != NIL).sum()) // 2
    finally:
        for h in handles:
            lm.lm_graph_destroy(h)
        L.close()
