"""Seeded synthetic graph generators shared by the tests, the oracle runs and
the benchmark.

This module only draws graphs (edge lists ``eu, ev`` of uint32 and weights
``w`` of float32); it holds none of the matching method's arithmetic.  The
heavy lifting is plain C (``gen.c``), compiled on first use into
``synth/_build/``.

Workload families (shapes of the paper's inputs, Sec. 3; the paper's own data
sets are not available, so these stand in for them):

* ``er``    -- random graph G(n, m) with weights uniform in [0, 1)
* ``grid``  -- 2D 4-neighbour grid plus a fraction of random long-range edges
* ``rmat``  -- R-MAT (a, b, c, d) = (.57, .19, .19, .05), random relabel,
  loops dropped, duplicates removed
* ``batch`` -- many small uneven graphs of the three kinds
* ``request_sizes`` -- a Poisson request stream for the serving loop
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def build() -> str:
    """Compile gen.c into synth/_build/libsynth.so (rebuilt when the source is newer)."""
    src = os.path.join(_HERE, "gen.c")
    out = os.path.join(_BUILD, "libsynth.so")
    os.makedirs(_BUILD, exist_ok=True)
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall",
                               "-o", tmp, src, "-lpthread", "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            f32p = ctypes.POINTER(ctypes.c_float)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.sx_at.restype = ctypes.c_uint64
            lib.sx_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.sx_derive.restype = ctypes.c_uint64
            lib.sx_derive.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gen_er.restype = ctypes.c_int64
            lib.gen_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.gen_rgg.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, u32p, u32p, ctypes.c_uint64]
            lib.gen_rgg.restype = ctypes.c_int64
            lib.gen_grid.restype = ctypes.c_int64
            lib.gen_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_uint64, u32p, u32p, ctypes.c_uint64]
            lib.gen_rmat.restype = ctypes.c_int64
            lib.gen_rmat.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, u32p, u32p, ctypes.c_uint64,
                                     ctypes.c_int]
            lib.gen_rmat_small.restype = ctypes.c_int64
            lib.gen_rmat_small.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                           ctypes.c_uint64, u32p, u32p]
            lib.gen_weights.restype = None
            lib.gen_weights.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, f32p]
            lib.gen_draws.restype = None
            lib.gen_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p]
            _LIB = lib
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class Graph:
    """An undirected edge list: edge i joins eu[i] and ev[i] with weight w[i]."""
    n: int
    eu: np.ndarray  # uint32[m]
    ev: np.ndarray  # uint32[m]
    w: np.ndarray   # float32[m]
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])


def draws(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of SplitMix64 seeded with `seed` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    if count:
        _lib().gen_draws(seed & (2**64 - 1), count, _p(out, ctypes.c_uint64))
    return out


def derive(seed: int, tag: int) -> int:
    return int(_lib().sx_derive(seed & (2**64 - 1), tag))


def weights(m: int, seed: int, unit: bool = False) -> np.ndarray:
    w = np.empty(m, dtype=np.float32)
    if m:
        _lib().gen_weights(m, seed & (2**64 - 1), 1 if unit else 0, _p(w, ctypes.c_float))
    return w


def er(n: int = 10_000, m: int = 50_000, seed: int = 1, unit: bool = False) -> Graph:
    """G(n, m): m distinct non-loop pairs, uniform; weights U[0,1) or all ones."""
    eu = np.empty(max(m, 1), dtype=np.uint32)
    ev = np.empty(max(m, 1), dtype=np.uint32)
    got = _lib().gen_er(n, m, derive(seed, 10), _p(eu, ctypes.c_uint32), _p(ev, ctypes.c_uint32))
    if got < 0:
        raise ValueError("gen_er failed")
    return Graph(n, eu[:got].copy(), ev[:got].copy(), weights(got, derive(seed, 3), unit),
                 f"er_n{n}_m{m}_s{seed}{'_unit' if unit else ''}")


def rgg(n: int, seed: int = 6) -> Graph:
    """Random geometric graph of Sec. 3: n points uniform in the unit square, an
    edge between points closer than 0.55 sqrt(ln n / n); weights U[0,1) (the
    paper states no weights for this family)."""
    r = 0.55 * math.sqrt(math.log(n) / n) if n > 1 else 0.0
    cap = int(n * math.pi * r * r * n * 0.75) + 4 * n + 1024
    eu = np.empty(max(cap, 1), dtype=np.uint32)
    ev = np.empty(max(cap, 1), dtype=np.uint32)
    got = _lib().gen_rgg(n, r, derive(seed, 13), _p(eu, ctypes.c_uint32), _p(ev, ctypes.c_uint32), cap)
    if got < 0:
        raise ValueError("gen_rgg failed")
    return Graph(n, eu[:got].copy(), ev[:got].copy(), weights(got, derive(seed, 3)), f"rgg_n{n}_s{seed}")


def grid(rows: int = 1024, cols: int = 1024, frac_long: float = 0.05, seed: int = 2,
         unit: bool = False, n_vertices: int | None = None, max_edges: int | None = None,
         n_long: int | None = None) -> Graph:
    """rows x cols 4-neighbour grid plus floor(frac_long * grid_edges) random long edges."""
    n = rows * cols if n_vertices is None else n_vertices
    grid_edges = rows * (cols - 1) + (rows - 1) * cols
    if n_long is None:
        n_long = int(math.floor(frac_long * grid_edges))
    if max_edges is None:
        max_edges = grid_edges
    cap = min(grid_edges, max_edges) + n_long + 1
    eu = np.empty(cap, dtype=np.uint32)
    ev = np.empty(cap, dtype=np.uint32)
    got = _lib().gen_grid(rows, cols, n, n_long, max_edges, derive(seed, 11),
                          _p(eu, ctypes.c_uint32), _p(ev, ctypes.c_uint32), cap)
    if got < 0:
        raise ValueError("gen_grid failed")
    return Graph(n, eu[:got].copy(), ev[:got].copy(), weights(got, derive(seed, 3), unit),
                 f"grid_{rows}x{cols}_s{seed}{'_unit' if unit else ''}")


def rmat(scale: int = 23, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 3, unit: bool = False, threads: int | None = None) -> Graph:
    """R-MAT with 2^scale vertices and edge_factor * 2^scale generated edges,
    relabelled by a seeded random permutation, loops dropped, duplicates removed."""
    n_gen = edge_factor << scale
    eu = np.empty(n_gen, dtype=np.uint32)
    ev = np.empty(n_gen, dtype=np.uint32)
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    got = _lib().gen_rmat(scale, n_gen, a, b, c, derive(seed, 12), _p(eu, ctypes.c_uint32),
                          _p(ev, ctypes.c_uint32), n_gen, threads)
    if got < 0:
        raise ValueError("gen_rmat failed")
    eu = eu[:got].copy()
    ev = ev[:got].copy()
    return Graph(1 << scale, eu, ev, weights(got, derive(seed, 3), unit),
                 f"rmat_s{scale}_ef{edge_factor}_s{seed}{'_unit' if unit else ''}")


def _uniform(x: np.uint64) -> float:
    return float(int(x) >> 11) * (1.0 / 9007199254740992.0)


def batch(count: int = 4096, seed: int = 4, n_lo: int = 64, n_hi: int = 65536,
          d_lo: float = 4.0, d_hi: float = 16.0) -> list[Graph]:
    """Mixed batch: n = floor(exp(U[ln n_lo, ln n_hi])), average degree d ~ U[d_lo, d_hi],
    target m = floor(n d / 2), generator chosen uniformly from {ER, grid, R-MAT}."""
    par = draws(derive(seed, 20), 4 * count)
    shapes = []
    for i in range(count):
        x0, x1, x2, x3 = (par[4 * i + k] for k in range(4))
        n = int(math.floor(math.exp(math.log(n_lo) + _uniform(x0) * (math.log(n_hi) - math.log(n_lo)))))
        n = max(2, min(n, n_hi))
        d = d_lo + _uniform(x1) * (d_hi - d_lo)
        m = int(math.floor(n * d / 2))
        m = min(m, n * (n - 1) // 2)
        shapes.append((int(_uniform(x2) * 3), n, m, int(x3), f"b{i}"))
    return _generate(shapes)


def _generate(shapes, threads: int | None = None) -> list[Graph]:
    """Graphs of the given (kind, n, m, graph seed, name) shapes.  Each graph
    depends on its own shape only, so they are drawn on a thread pool (the C
    generators release the interpreter lock) with the same result as one by one."""
    from concurrent.futures import ThreadPoolExecutor
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    if threads <= 1 or len(shapes) < 2:
        return [_graph_of_kind(*s) for s in shapes]
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda s: _graph_of_kind(*s), shapes))


def _graph_of_kind(kind: int, n: int, m: int, gseed: int, name: str) -> Graph:
    if kind == 0:
        g = er(n, m, gseed)
    elif kind == 1:
        side = int(math.ceil(math.sqrt(n)))
        rows = int(math.ceil(n / side))
        grid_edges_max = rows * (side - 1) + (rows - 1) * side
        g = grid(rows, side, seed=gseed, n_vertices=n, max_edges=m, n_long=max(0, m - min(m, grid_edges_max)))
    else:
        eu = np.empty(max(m, 1), dtype=np.uint32)
        ev = np.empty(max(m, 1), dtype=np.uint32)
        got = _lib().gen_rmat_small(n, m, 0.57, 0.19, 0.19, derive(gseed, 12), 64 * max(m, 1),
                                    _p(eu, ctypes.c_uint32), _p(ev, ctypes.c_uint32))
        if got < 0:
            raise ValueError("gen_rmat_small failed")
        g = Graph(n, eu[:got].copy(), ev[:got].copy(), weights(got, derive(gseed, 3)))
    g.name = f"{name}_{('er', 'grid', 'rmat')[kind]}_n{n}_m{g.m}"
    return g


def request_sizes(count: int, seed: int = 5, m_lo: float = 1e3, m_hi: float = 4e6):
    """Request shapes for the serving stream: m = floor(exp(U[ln m_lo, ln m_hi])),
    n = max(2, floor(m / U[2, 8])), generator uniform over {ER, grid, R-MAT}.
    Returns a list of (kind, n, m, graph_seed)."""
    par = draws(derive(seed, 30), 4 * count)
    out = []
    for i in range(count):
        x0, x1, x2, x3 = (par[4 * i + k] for k in range(4))
        m = int(math.floor(math.exp(math.log(m_lo) + _uniform(x0) * (math.log(m_hi) - math.log(m_lo)))))
        n = max(2, int(math.floor(m / (2.0 + 6.0 * _uniform(x1)))))
        m = min(m, n * (n - 1) // 2)
        out.append((int(_uniform(x2) * 3), n, m, int(x3)))
    return out


def request_graph(kind: int, n: int, m: int, gseed: int, name: str = "req") -> Graph:
    return _graph_of_kind(kind, n, m, gseed, name)


def request_pool(count: int, seed: int = 5, m_lo: float = 1e3, m_hi: float = 4e6) -> list[Graph]:
    """The graphs of request_sizes(count, seed, m_lo, m_hi), named r0, r1, ..."""
    return _generate([(*sz, f"r{i}") for i, sz in enumerate(request_sizes(count, seed, m_lo, m_hi))])


def arrivals(count: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Poisson arrival times (seconds from 0) with the given rate."""
    u = draws(derive(seed, 31), count)
    gaps = np.array([-math.log(1.0 - _uniform(x)) / rate_per_s for x in u], dtype=np.float64)
    return np.cumsum(gaps)


def pairs(n: int, m: int, seed: int, weight_kind: str = "uniform") -> Graph:
    """m random non-loop pairs on n vertices, parallel edges allowed (test inputs).

    weight_kind: 'uniform' (U[0,1)), 'unit' (all 1.0), 'few' (values in {0,.25,.5,.75}),
    'signed' (U[-1,1) plus the specials -0.0, 0.0, -inf, inf mixed in)."""
    if n < 2:
        return Graph(n, np.zeros(0, np.uint32), np.zeros(0, np.uint32), np.zeros(0, np.float32))
    x = draws(derive(seed, 40), 2 * m + 64)
    eu, ev = [], []
    i = 0
    while len(eu) < m:
        a = int((int(x[i]) & 0xFFFFFFFF) * n >> 32)
        b = int((int(x[i]) >> 32) * n >> 32)
        i += 1
        if i >= x.shape[0]:
            x = np.concatenate([x, draws(derive(seed, 41 + i), 2 * m + 64)])
        if a != b:
            eu.append(a)
            ev.append(b)
    w = weights(m, derive(seed, 3), unit=(weight_kind == "unit"))
    if weight_kind == "few":
        w = (np.floor(w * 4.0) / 4.0).astype(np.float32)
    elif weight_kind == "signed":
        w = (w * 2.0 - 1.0).astype(np.float32)
        sp = np.array([-0.0, 0.0, -np.inf, np.inf, 1e-45, -1e-45], dtype=np.float32)
        for k in range(min(m, 6)):
            w[(k * 7919) % m] = sp[k]
    return Graph(n, np.array(eu, dtype=np.uint32), np.array(ev, dtype=np.uint32),
                 w.astype(np.float32), f"pairs_n{n}_m{m}_s{seed}_{weight_kind}")
