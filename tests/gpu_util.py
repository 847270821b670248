"""Helpers for the GPU tests: run the CUDA path through the C ABI."""
from __future__ import annotations

import numpy as np

NIL = 0xFFFFFFFF


def to_u32(t) -> np.ndarray:
    import torch
    if isinstance(t, torch.Tensor):
        return t.detach().cpu().numpy().view(np.uint32).copy()
    return np.asarray(t).astype(np.uint32)


class Lm:
    """One lm context on cuda:0 for a test session."""

    def __init__(self, profile: bool = False, budget: int = 0, edge_centric: bool = False, renew: bool = False):
        import torch
        import paper_1302_4587_gb300 as lm
        self.lm = lm
        self.torch = torch
        torch.cuda.init()
        flags = ((lm.LM_F_PROFILE if profile else 0) | (lm.LM_F_EDGE_CENTRIC if edge_centric else 0)
                 | (lm.LM_F_RENEW if renew else 0))
        self.ctx = lm.lm_create(0, None, hbm_budget_bytes=budget, flags=flags)

    def close(self):
        if self.ctx is not None:
            self.lm.lm_destroy(self.ctx)
            self.ctx = None

    def graph(self, g, device: bool = True):
        torch = self.torch
        if device:
            eu = torch.from_numpy(g.eu.view(np.int32)).cuda()
            ev = torch.from_numpy(g.ev.view(np.int32)).cuda()
            w = torch.from_numpy(g.w).cuda()
            return self.lm.lm_graph_create(self.ctx, g.n, eu, ev, w)
        return self.lm.lm_graph_create(self.ctx, g.n, g.eu, g.ev, g.w)

    def match(self, g, seed: int, device_out: bool = True, handle=None):
        torch = self.torch
        h = handle if handle is not None else self.graph(g)
        try:
            if device_out:
                mate = torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")[: g.n]
            else:
                mate = np.empty(g.n, dtype=np.uint32)
            mate, st = self.lm.lm_match(self.ctx, h, seed, mate, stats=True)
            return to_u32(mate), st
        finally:
            if handle is None:
                self.lm.lm_graph_destroy(h)
