"""Exact references for tiny graphs, written from definitions, independent of the oracle.

* ``sigma_ic``: the expected number of activated vertices under the IC model, computed by
  enumerating the cascade process itself (Sec. 2: in every round each newly activated vertex
  tries each incident edge once, succeeding with probability p), with exact fractions.
  It never forms a live-edge world.
* ``world_components``: per live-edge world, connected components from
  ``scipy.sparse.csgraph.connected_components`` (a library routine).
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from itertools import combinations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components


def sigma_ic(n: int, edges, S, p: Fraction) -> Fraction:
    adj = [set() for _ in range(n)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    q = 1 - p

    @lru_cache(maxsize=None)
    def expect(active: frozenset, frontier: frozenset) -> Fraction:
        if not frontier:
            return Fraction(len(active))
        tries = {}
        for u in frontier:
            for w in adj[u]:
                if w not in active:
                    tries[w] = tries.get(w, 0) + 1
        targets = sorted(tries)
        total = Fraction(0)
        for mask in range(1 << len(targets)):
            pr = Fraction(1)
            new = []
            for i, w in enumerate(targets):
                fail = q ** tries[w]
                if mask >> i & 1:
                    pr *= 1 - fail
                    new.append(w)
                else:
                    pr *= fail
            if pr == 0:
                continue
            total += pr * expect(active | frozenset(new), frozenset(new))
        return total

    s = frozenset(S)
    return expect(s, s)


def world_components(n: int, edges, live_mask: int) -> np.ndarray:
    """Component id per vertex (scipy) in the world whose live edges are the bits of live_mask."""
    sel = [i for i in range(len(edges)) if live_mask >> i & 1]
    if sel:
        a = np.array([edges[i][0] for i in sel])
        b = np.array([edges[i][1] for i in sel])
    else:
        a = b = np.zeros(0, dtype=np.int64)
    A = coo_matrix((np.ones(len(a)), (a, b)), shape=(n, n))
    _, comp = connected_components(A, directed=False)
    return comp


def world_spread(n: int, edges, live_mask: int, S) -> int:
    comp = world_components(n, edges, live_mask)
    hit = {comp[s] for s in S}
    return int(sum(1 for v in range(n) if comp[v] in hit))


def sigma_worlds(n: int, edges, S, p: Fraction) -> Fraction:
    """Weighted sum over all live-edge worlds (library components); equals sigma_ic."""
    m = len(edges)
    tot = Fraction(0)
    for mask in range(1 << m):
        k = bin(mask).count("1")
        tot += p ** k * (1 - p) ** (m - k) * world_spread(n, edges, mask, S)
    return tot


def best_k_subset(n: int, value, k: int):
    """Exhaustive optimum of a set function over all k-subsets."""
    best = None
    for S in combinations(range(n), k):
        val = value(S)
        if best is None or val > best[0]:
            best = (val, S)
    return best
