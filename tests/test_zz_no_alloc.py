"""lm_match_small_noalloc through the C ABI (file named to be collected last).

The entry point serves callers that must not allocate device memory while
they run (a fixed device footprint, or all free memory handed to another
allocator): it matches one small device-resident graph with a static device
array as its only scratch.  Its result must equal the oracle's greedy matching
under the same order and lm_match's on the same graph and seed, on
consecutive calls (nothing may leak from one call into the next), up to the
scratch's limits, with unit weights (every comparison decided by the
permutation) and with parallel edges.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import Lm, to_u32

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    eu = torch.from_numpy(g.eu.view(np.int32)).cuda()
    ev = torch.from_numpy(g.ev.view(np.int32)).cuda()
    w = torch.from_numpy(g.w).cuda()
    return eu, ev, w


def _parallel_edges(seed):
    # an ER graph plus repeats of some of its edges (both orientations) with new weights
    g = synth.er(5000, 20_000, seed)
    k = 4000
    eu = np.concatenate([g.eu, g.eu[:k], g.ev[k:2 * k]])
    ev = np.concatenate([g.ev, g.ev[:k], g.eu[k:2 * k]])
    w = np.concatenate([g.w, synth.weights(2 * k, seed + 100)])
    return synth.Graph(g.n, eu, ev, w.astype(np.float32), f"parallel{seed}")


def _mono_path(n):
    eu = np.arange(n - 1, dtype=np.uint32)
    return synth.Graph(n, eu, eu + 1, (np.arange(n - 1) + 1).astype(np.float32), f"mono{n}")


def _cases():
    import paper_1302_4587_gb300 as lm
    at_limits = synth.er(lm.LM_NOALLOC_MAX_N, lm.LM_NOALLOC_MAX_M, seed=34)
    assert at_limits.n == lm.LM_NOALLOC_MAX_N and at_limits.m == lm.LM_NOALLOC_MAX_M
    er = synth.er(20_000, 120_000, seed=31)
    return [(er, 5), (er, 5),                                          # the same call twice
            (at_limits, 7), (at_limits, 7),                            # every scratch slot in use
            (synth.er(3_000, 9_000, seed=32), 9),
            (synth.er(8_000, 40_000, seed=35, unit=True), 11),         # unit weights
            (synth.grid(64, 64, 0.05, seed=33, unit=True), 1),
            (_parallel_edges(36), 13),
            (_mono_path(2001), 3),                                     # 1000 rounds
            (synth.Graph(6, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32), "empty"), 1)]


def test_noalloc_equals_the_oracle_and_lm_match_on_consecutive_calls():
    import torch
    import paper_1302_4587_gb300 as lm
    L = Lm()
    try:
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        for g, seed in _cases():
            assert g.n <= lm.LM_NOALLOC_MAX_N and g.m <= lm.LM_NOALLOC_MAX_M
            want = oracle.greedy(g.n, g.eu, g.ev, g.w, seed)
            eu, ev, w = _dev(g)
            mate = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            lm.lm_match_small_noalloc(g.n, eu, ev, w, seed, mate, status)
            torch.cuda.synchronize()
            assert int(status.item()) == 0, g.name
            got = to_u32(mate)
            bad = np.nonzero(got != want)[0]
            assert bad.size == 0, f"{g.name}: {bad.size} vertices differ from the oracle"
            plain, _ = L.match(g, seed)
            np.testing.assert_array_equal(got, plain)
    finally:
        L.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_1302_4587_gb300 as lm
    one = torch.zeros(1, dtype=torch.int32, device="cuda")
    w = torch.zeros(1, dtype=torch.float32, device="cuda")
    mate = torch.zeros(lm.LM_NOALLOC_MAX_N + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(lm.LmError) as ei:
        lm.lm_match_small_noalloc(lm.LM_NOALLOC_MAX_N + 1, one, one, w, 1, mate, one)
    assert ei.value.code == lm.LM_EINVAL
    big = torch.zeros(lm.LM_NOALLOC_MAX_M + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(lm.LmError) as ei:
        lm.lm_match_small_noalloc(10, big, big, big.float(), 1, mate, one)
    assert ei.value.code == lm.LM_EINVAL


def test_noalloc_rejects_memory_that_is_not_on_the_current_device():
    # the C entry point itself refuses host pointers (the binding refuses them earlier)
    import torch
    import paper_1302_4587_gb300 as lm
    lib = lm.load()
    g = synth.er(100, 300, seed=37)
    eu, ev, w = _dev(g)
    mate = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    host = np.zeros(max(g.n, g.m), np.uint32)
    hp = host.ctypes.data
    args = [eu.data_ptr(), ev.data_ptr(), w.data_ptr(), mate.data_ptr(), status.data_ptr()]
    for k in range(5):
        a = list(args)
        a[k] = hp
        rc = lib.lm_match_small_noalloc(g.n, g.m, a[0], a[1], a[2], 1, a[3], a[4], None)
        assert rc == lm.LM_EINVAL, k
    assert lib.lm_match_small_noalloc(g.n, g.m, *args[:3], 1, *args[3:], None) == lm.LM_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    np.testing.assert_array_equal(to_u32(mate), oracle.greedy(g.n, g.eu, g.ev, g.w, 1))
    with pytest.raises(ValueError):
        lm.lm_match_small_noalloc(g.n, eu.cpu(), ev, w, 1, mate, status)


def test_noalloc_flags_invalid_edges():
    import torch
    import paper_1302_4587_gb300 as lm
    eu = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda")
    ev = torch.tensor([1, 1, 3], dtype=torch.int32, device="cuda")  # a self loop
    w = torch.tensor([1.0, 2.0, 3.0], dtype=torch.float32, device="cuda")
    mate = torch.zeros(4, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    lm.lm_match_small_noalloc(4, eu, ev, w, 1, mate, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    assert (to_u32(mate) == lm.LM_NIL).all()
    # the next call on valid input is unaffected
    ev2 = torch.tensor([1, 2, 3], dtype=torch.int32, device="cuda")
    lm.lm_match_small_noalloc(4, eu, ev2, w, 1, mate, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert to_u32(mate).tolist() == [1, 0, 3, 2]  # the heaviest edge (2, 3), then (0, 1)
    want = oracle.greedy(4, np.array([0, 1, 2], np.uint32), np.array([1, 2, 3], np.uint32),
                         np.array([1.0, 2.0, 3.0], np.float32), 1)
    np.testing.assert_array_equal(to_u32(mate), want)
