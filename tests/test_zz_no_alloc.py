"""lm_match_small_noalloc through the C ABI (file named to be collected last).

The entry point matches one small device-resident graph with no allocation,
its only scratch a static device array; its result must equal lm_match's on
the same graph and seed, on consecutive calls (nothing may leak from one call
into the next).
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from gpu_util import Lm, to_u32

pytestmark = pytest.mark.gpu


def _dev(g):
    import torch
    eu = torch.from_numpy(g.eu.view(np.int32)).cuda()
    ev = torch.from_numpy(g.ev.view(np.int32)).cuda()
    w = torch.from_numpy(g.w).cuda()
    return eu, ev, w


def test_noalloc_equals_lm_match_on_consecutive_calls():
    import torch
    import paper_1302_4587_gb300 as lm
    L = Lm()
    try:
        cases = [(synth.er(20_000, 120_000, seed=31), 5), (synth.er(20_000, 120_000, seed=31), 5),
                 (synth.er(3_000, 9_000, seed=32), 9), (synth.grid(64, 64, 0.05, seed=33), 1)]
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        for g, seed in cases:
            assert g.n <= lm.LM_NOALLOC_MAX_N and g.m <= lm.LM_NOALLOC_MAX_M
            want, _ = L.match(g, seed)
            eu, ev, w = _dev(g)
            mate = torch.full((g.n,), 12345, dtype=torch.int32, device="cuda")
            lm.lm_match_small_noalloc(g.n, eu, ev, w, seed, mate, status)
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            np.testing.assert_array_equal(to_u32(mate), want)
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
