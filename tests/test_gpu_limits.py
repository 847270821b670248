"""The error contract of the C ABI, provoked without faulting a GPU.

LM_ETIMEOUT: a round cap or time limit (lm_set_limits) that a long run
exceeds.  The device-driven loop checks both after every second round and
returns an error status; the profiled path checks them on the host.  A path
with monotone weights needs ceil((n - 1) / 2) rounds under the fixed order
(Sec. 2 bounds the rounds only in expectation), so it runs past any small cap.

LM_ENOMEM: allocation failures injected on the host (LM_FAULT=alloc[:N], read
by lm_create); nothing is allocated short on the device.

After either error the context must still match a graph bit-exactly."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import NIL, Lm

pytestmark = pytest.mark.gpu


def _mono_path(n):
    eu = np.arange(n - 1, dtype=np.uint32)
    return synth.Graph(n, eu, eu + 1, (np.arange(n - 1) + 1).astype(np.float32), f"mono{n}")


def _exact(L, g, seed, handle=None):
    mate, st = L.match(g, seed, handle=handle)
    want = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
    assert np.array_equal(mate, want), g.name
    assert st["matched"] == int((want != NIL).sum()) // 2
    return st


@pytest.mark.parametrize("profile", [False, True], ids=["graph", "profiled"])
def test_round_cap_times_out_and_the_context_stays_usable(profile):
    import paper_1302_4587_gb300 as lm
    L = Lm(profile=profile)
    try:
        path = _mono_path(3001)   # 1500 rounds
        h = L.graph(path)
        lm.lm_set_limits(L.ctx, 10, 0)
        with pytest.raises(lm.LmError) as ei:
            L.match(path, 1, handle=h)
        assert ei.value.code == lm.LM_ETIMEOUT
        # a graph that needs fewer rounds than the cap is not affected
        st = _exact(L, synth.er(10_000, 50_000, 1), 101)
        assert st["rounds"] <= 10
        # without the cap the long path runs to its end
        lm.lm_set_limits(L.ctx, 0, 0)
        st = _exact(L, path, 1, handle=h)
        assert st["rounds"] == math.ceil((path.n - 1) / 2)
        lm.lm_graph_destroy(h)
    finally:
        L.close()


@pytest.mark.parametrize("profile", [False, True], ids=["graph", "profiled"])
def test_time_limit_times_out_and_the_context_stays_usable(profile):
    import paper_1302_4587_gb300 as lm
    L = Lm(profile=profile)
    try:
        path = _mono_path(20_001)  # 10,000 rounds: far more than 1 ms on any GPU
        h = L.graph(path)
        lm.lm_set_limits(L.ctx, 0, 1)
        with pytest.raises(lm.LmError) as ei:
            L.match(path, 1, handle=h)
        assert ei.value.code == lm.LM_ETIMEOUT
        lm.lm_graph_destroy(h)
        lm.lm_set_limits(L.ctx, 0, 0)
        _exact(L, synth.er(10_000, 50_000, 1, unit=True), 101)
    finally:
        L.close()


def test_round_cap_applies_to_batches():
    import paper_1302_4587_gb300 as lm
    L = Lm()
    try:
        graphs = [_mono_path(3001), synth.er(2000, 8000, 5)]
        hs = [L.graph(g) for g in graphs]
        mates = [L.torch.empty(g.n, dtype=L.torch.int32, device="cuda") for g in graphs]
        lm.lm_set_limits(L.ctx, 10, 0)
        with pytest.raises(lm.LmError) as ei:
            lm.lm_batch_match(L.ctx, hs, [1, 2], mates)
        assert ei.value.code == lm.LM_ETIMEOUT
        lm.lm_set_limits(L.ctx, 0, 0)
        out = lm.lm_batch_match(L.ctx, hs, [1, 2], mates)
        for g, s, mt in zip(graphs, [1, 2], out):
            assert np.array_equal(mt.cpu().numpy().view(np.uint32), oracle.greedy(g.n, g.eu, g.ev, g.w, s))
        for h in hs:
            lm.lm_graph_destroy(h)
    finally:
        L.close()


def test_injected_allocation_failures_return_enomem(monkeypatch):
    import paper_1302_4587_gb300 as lm
    g = synth.er(3000, 9000, 2)
    # the next allocation of the context fails: graph creation reports LM_ENOMEM
    # and the context is not poisoned
    monkeypatch.setenv("LM_FAULT", "alloc:1")
    A = Lm()
    monkeypatch.delenv("LM_FAULT")
    try:
        with pytest.raises(lm.LmError) as ei:
            A.graph(g)
        assert ei.value.code == lm.LM_ENOMEM
        h = A.graph(g)
        _exact(A, g, 3, handle=h)
        # a match whose workspace allocation fails, then the same match again
        monkeypatch.setenv("LM_FAULT", "alloc:1")
        B = Lm()
        monkeypatch.delenv("LM_FAULT")
        try:
            with pytest.raises(lm.LmError) as ei:
                B.match(g, 4, handle=h)
            assert ei.value.code == lm.LM_ENOMEM
            _exact(B, g, 4, handle=h)
        finally:
            B.close()
        # every allocation failing: graph creation, matching and contraction all refuse
        monkeypatch.setenv("LM_FAULT", "alloc")
        C = Lm()
        monkeypatch.delenv("LM_FAULT")
        try:
            for call in (lambda: C.graph(g), lambda: C.match(g, 5, handle=h)):
                with pytest.raises(lm.LmError) as ei:
                    call()
                assert ei.value.code == lm.LM_ENOMEM
            torch = C.torch
            eu = torch.from_numpy(g.eu.view(np.int32)).cuda()
            ev = torch.from_numpy(g.ev.view(np.int32)).cuda()
            w = torch.from_numpy(g.w).cuda()
            mate = torch.from_numpy(oracle.greedy(g.n, g.eu, g.ev, g.w, 3).view(np.int32)).cuda()
            with pytest.raises(lm.LmError) as ei:
                lm.lm_contract(C.ctx, g.n, eu, ev, w, mate)
            assert ei.value.code == lm.LM_ENOMEM
        finally:
            C.close()
        lm.lm_graph_destroy(h)
    finally:
        A.close()
