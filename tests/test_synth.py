"""The random geometric graph generator against brute force (CPU)."""
from __future__ import annotations

import math

import numpy as np

import synth


def test_rgg_equals_all_pairs_closer_than_the_radius():
    for n, seed in ((300, 6), (1000, 7), (2048, 8)):
        g = synth.rgg(n, seed)
        r = 0.55 * math.sqrt(math.log(n) / n)
        d = synth.draws(synth.derive(seed, 13), 2 * n).astype(np.uint64)
        pts = (d >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        x, y = pts[0::2], pts[1::2]
        dx = x[:, None] - x[None, :]
        dy = y[:, None] - y[None, :]
        close = (dx * dx + dy * dy) < r * r
        iu, ju = np.nonzero(np.triu(close, 1))
        want = set(zip(iu.tolist(), ju.tolist()))
        got = set(zip(g.eu.tolist(), g.ev.tolist()))
        assert len(got) == g.m  # no duplicates
        assert got == want
        assert (g.eu < g.ev).all()
