"""Brute-force extremum graph for tiny grids, written independently of the oracle.

Differences from the oracle on purpose, so that one cannot share a mistake with
the other:
  * the order is a rank obtained by sorting (value, index) pairs, not a
    pairwise comparison;
  * adjacency is Algorithm 1 (Sec. 3.2) applied to EVERY pair of grid
    vertices, not a table of offsets;
  * link edges are every adjacent pair inside the neighbour set (the link of a
    flag complex, Sec. 3.3), and components are counted by breadth-first
    search (the paper's first formulation, Sec. 3.3), not union-find;
  * gradient paths are walked naively from every vertex (Algorithm 2's loop).
"""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np


def coords(extents):
    """All vertex coordinates, in linear-index order (axis 0 fastest)."""
    rngs = [range(e) for e in reversed(extents)]
    return [tuple(reversed(c)) for c in itertools.product(*rngs)]


def alg1_adjacent(p, q):
    diffs = {a - b for a, b in zip(p, q)}
    if p == q:
        return False
    return diffs <= {0, 1} or diffs <= {0, -1}


def sos_rank(values, minimum=False):
    """rank[v]: position of v in the total order (value, then index)."""
    n = len(values)
    idx = np.arange(n)
    order = np.lexsort((idx, values))  # ascending value, ties by ascending index
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    if minimum:
        rank = (n - 1) - rank
    return rank


def brute_graph(field, extents, minimum=False, dtype=np.float32):
    # values stay in their own element type: numpy's sort compares them exactly
    vals = np.asarray(field, dtype=dtype).reshape(-1)
    n = vals.size
    X = coords(extents)
    assert len(X) == n
    rank = sos_rank(vals, minimum)
    nbrs = [[w for w in range(n) if alg1_adjacent(X[v], X[w])] for v in range(n)]

    asc = np.empty(n, np.int64)
    beta = np.empty(n, np.int64)
    reps = {}
    for v in range(n):
        up = [w for w in nbrs[v] if rank[w] > rank[v]]
        asc[v] = max(up, key=lambda w: rank[w]) if up else v
        seen, comps = set(), []
        for s in up:
            if s in seen:
                continue
            comp, dq = [], deque([s])
            seen.add(s)
            while dq:
                a = dq.popleft()
                comp.append(a)
                for b in up:
                    if b not in seen and alg1_adjacent(X[a], X[b]):
                        seen.add(b)
                        dq.append(b)
            comps.append(comp)
        beta[v] = len(comps)
        reps[v] = [max(c, key=lambda w: rank[w]) for c in comps]

    label = np.empty(n, np.int64)
    for v in range(n):
        u = v
        while asc[u] != u:
            u = asc[u]
        label[v] = u

    maxima = [v for v in range(n) if beta[v] == 0]
    saddles = [v for v in range(n) if beta[v] >= 2]
    arcs = {(s, int(label[r])) for s in saddles for r in reps[s]}
    # arc geometry: per saddle and per representative in ascending id order,
    # the saddle and the naive walk from the representative
    paths = []
    for s in saddles:
        for r in sorted(int(x) for x in reps[s]):
            walk = [s, r]
            while asc[walk[-1]] != walk[-1]:
                walk.append(int(asc[walk[-1]]))
            paths.append(walk)
    return dict(asc=asc, label=label, beta=beta, maxima=maxima, saddles=saddles,
                arcs=arcs, reps=reps, paths=paths)
