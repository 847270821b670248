"""Checks on matchings that need neither the oracle nor the CUDA path."""
from __future__ import annotations

import os

import numpy as np

NIL = 0xFFFFFFFF
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def is_matching(n, eu, ev, mate) -> bool:
    """mate is symmetric, and every matched pair is an edge of the graph."""
    mate = np.asarray(mate, dtype=np.int64)
    matched = np.nonzero(mate != NIL)[0]
    if matched.size and (mate[matched] >= n).any():
        return False
    if matched.size and (mate[mate[matched]] != matched).any():
        return False
    if matched.size and (mate[matched] == matched).any():
        return False
    edges = set(zip(np.minimum(eu, ev).tolist(), np.maximum(eu, ev).tolist()))
    for v in matched.tolist():
        u = int(mate[v])
        if (min(u, v), max(u, v)) not in edges:
            return False
    return True


def is_maximal(eu, ev, mate) -> bool:
    """No edge has both endpoints unmatched (Sec. 1: maximality)."""
    mate = np.asarray(mate)
    free_u = mate[np.asarray(eu, dtype=np.int64)] == NIL
    free_v = mate[np.asarray(ev, dtype=np.int64)] == NIL
    return not bool((free_u & free_v).any())


def dominated(eu, ev, keys, mate) -> bool:
    """The local-max characterisation: an edge is in M exactly when no heavier
    adjacent edge is in M.  For a matching M this says: every edge outside M
    has an endpoint whose matched edge is heavier than it.  Checked edge by
    edge, without sorting."""
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    keys = np.asarray(keys, dtype=np.uint64)
    mate = np.asarray(mate, dtype=np.int64)
    n = mate.shape[0]
    # key of the matched edge at each vertex (0 = none).  With parallel edges
    # the matched edge of v is the edge (v, mate[v]) that is in M; identify it
    # as the heaviest edge between v and mate[v] whose both ends chose it.
    mk = np.zeros(n, dtype=np.uint64)
    in_m = np.zeros(eu.shape[0], dtype=bool)
    best = {}
    for i in range(eu.shape[0]):
        a, b = int(eu[i]), int(ev[i])
        if mate[a] == b and mate[b] == a:
            p = (min(a, b), max(a, b))
            if p not in best or keys[i] > keys[best[p]]:
                best[p] = i
    for p, i in best.items():
        in_m[i] = True
        mk[p[0]] = keys[i]
        mk[p[1]] = keys[i]
    for i in range(eu.shape[0]):
        if in_m[i]:
            continue
        if not (mk[eu[i]] > keys[i] or mk[ev[i]] > keys[i]):
            return False
    return True


def load_hand_cases():
    cases = []
    cur = None
    with open(os.path.join(GOLDEN, "hand_cases.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"name": tok[1], "n": int(tok[2]), "eu": [], "ev": [], "w": []}
                cases.append(cur)
            elif tok[0] == "e":
                cur["eu"].append(int(tok[1]))
                cur["ev"].append(int(tok[2]))
                cur["w"].append(float(tok[3]))
            elif tok[0] == "mate":
                cur["mate"] = [NIL if int(x) < 0 else int(x) for x in tok[1:]]
            elif tok[0] == "rounds":
                cur["rounds"] = int(tok[1])
    for c in cases:
        c["eu"] = np.array(c["eu"], dtype=np.uint32)
        c["ev"] = np.array(c["ev"], dtype=np.uint32)
        c["w"] = np.array(c["w"], dtype=np.float32)
        c["mate"] = np.array(c["mate"], dtype=np.uint32)
    return cases


def load_hash_vectors():
    sm, fm = [], []
    with open(os.path.join(GOLDEN, "hash_vectors.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "splitmix64_seq":
                sm.append((int(tok[1], 0), [int(x, 16) for x in tok[2:]]))
            elif tok[0] == "fmix32":
                fm.append((int(tok[1], 16), int(tok[2], 16)))
    return sm, fm
