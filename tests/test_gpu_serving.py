"""The served form's contract through the C ABI: admission limits, unknown
tickets, empty graphs, the same graph in flight many times with different
seeds, and shutdown with requests in flight."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import NIL, Lm, to_u32

pytestmark = pytest.mark.gpu


def test_request_larger_than_the_budget_is_refused():
    import paper_1302_4587_gb300 as lm
    srv = Lm(budget=1 << 20)  # room for about 33 thousand entries
    try:
        g = synth.er(20_000, 40_000, seed=3)
        h = srv.graph(g)
        mate = np.empty(g.n, np.uint32)
        with pytest.raises(lm.LmError) as ei:
            lm.lm_submit(srv.ctx, h, 1, mate)
        assert ei.value.code == lm.LM_ENOMEM
        small = synth.er(200, 600, seed=4)
        hs = srv.graph(small)
        ms = np.empty(small.n, np.uint32)
        t = lm.lm_submit(srv.ctx, hs, 2, ms)  # a request that fits is still served
        assert lm.lm_wait(srv.ctx, t, 60_000)
        assert lm.lm_poll(srv.ctx, t)[0]
        assert np.array_equal(ms, oracle.greedy(small.n, small.eu, small.ev, small.w, 2))
        lm.lm_graph_destroy(h)
        lm.lm_graph_destroy(hs)
    finally:
        srv.close()


def test_unknown_tickets():
    import paper_1302_4587_gb300 as lm
    srv = Lm()
    try:
        for fn in (lambda: lm.lm_poll(srv.ctx, 123456), lambda: lm.lm_wait(srv.ctx, 123456, 10)):
            with pytest.raises(lm.LmError) as ei:
                fn()
            assert ei.value.code == lm.LM_ENOTFOUND
    finally:
        srv.close()


def test_empty_graphs_are_served():
    import paper_1302_4587_gb300 as lm
    srv = Lm()
    try:
        cases = [synth.Graph(7, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32), "edgeless"),
                 synth.Graph(0, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32), "empty")]
        for g in cases:
            h = srv.graph(g, device=False)
            mate = np.full(max(g.n, 1), 5, np.uint32)[: g.n]
            t = lm.lm_submit(srv.ctx, h, 1, mate)
            assert lm.lm_wait(srv.ctx, t, 60_000)
            done, st = lm.lm_poll(srv.ctx, t)
            assert done and st["rounds"] == 0 and st["matched"] == 0
            assert (mate == NIL).all()
            lm.lm_graph_destroy(h)
    finally:
        srv.close()


def test_one_graph_many_seeds_in_flight():
    import paper_1302_4587_gb300 as lm
    srv = Lm()
    try:
        g = synth.grid(128, 128, 0.05, seed=12, unit=True)  # unit weights: the seed decides
        h = srv.graph(g)
        mates = [srv.torch.empty(g.n, dtype=srv.torch.int32, device="cuda") for _ in range(16)]
        tickets = [lm.lm_submit(srv.ctx, h, 900 + i, m) for i, m in enumerate(mates)]
        for i, t in enumerate(tickets):
            assert lm.lm_wait(srv.ctx, t, 60_000)
            assert lm.lm_poll(srv.ctx, t)[0]
            assert np.array_equal(to_u32(mates[i]), oracle.greedy(g.n, g.eu, g.ev, g.w, 900 + i))
        lm.lm_graph_destroy(h)
    finally:
        srv.close()


def test_destroy_with_requests_in_flight_returns():
    import paper_1302_4587_gb300 as lm
    srv = Lm()
    g = synth.grid(256, 256, 0.05, seed=13)
    h = srv.graph(g)
    mates = [srv.torch.empty(g.n, dtype=srv.torch.int32, device="cuda") for _ in range(8)]
    for i, m in enumerate(mates):
        lm.lm_submit(srv.ctx, h, i, m)
    t0 = time.perf_counter()
    srv.close()  # stops the scheduler; must not hang on the requests in flight
    assert time.perf_counter() - t0 < 30
    # (the graph belonged to the destroyed context: its handle is abandoned, not destroyed)
