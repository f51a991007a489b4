"""Brute-force checkers written independently of the oracle (pure Python / numpy).

They recompute quantities from the definitions in the paper by exhaustive
enumeration on tiny inputs: connection strengths by scanning every edge, cuts
and block weights by summation, optimal partitions by enumerating all k^n
labelings.  Used by the CPU tests to pin the oracle to something other than
itself.
"""
from __future__ import annotations

import itertools

import numpy as np

M64 = (1 << 64) - 1


def mix64(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def tie(seed: int, rnd: int, v: int, L: int) -> int:
    h = mix64(seed ^ ((rnd + 1) << 32) ^ v)
    return mix64(h ^ L) >> 32


def colour(seed: int, rnd: int, v: int, S: int) -> int:
    return (mix64(seed ^ ((rnd + 1) << 32) ^ v) >> 32) % S


def edges(g):
    """Undirected edge list (u < v, w) from a CSR dict of numpy arrays."""
    x, a, w = g["xadj"], g["adjncy"], g["adjwgt"]
    out = []
    for v in range(len(x) - 1):
        for i in range(x[v], x[v + 1]):
            if v < a[i]:
                out.append((v, int(a[i]), int(w[i])))
    return out


def omega(g, lab, v, L):
    """Connection strength of v to the set of nodes labelled L (any node but v)."""
    s = 0
    for (a, b, w) in edges(g):
        if a == v and lab[b] == L:
            s += w
        elif b == v and lab[a] == L:
            s += w
    return s


def cut(g, part):
    return sum(w for (a, b, w) in edges(g) if part[a] != part[b])


def block_weights(g, part, k):
    bw = [0] * k
    for v, c in enumerate(g["vwgt"]):
        bw[part[v]] += int(c)
    return bw


def label_weights(g, lab, nlabels):
    W = [0] * nlabels
    for v, c in enumerate(g["vwgt"]):
        W[lab[v]] += int(c)
    return W


def improving_moves(g, lab, nlabels, B, overload_rule):
    """All single moves (v, L) that the move rule would still allow: L is the label
    of some neighbour, L != own, W(L) + c(v) <= B, and either the gain is positive
    or (refinement) v's own label is overloaded."""
    n = len(g["xadj"]) - 1
    W = label_weights(g, lab, nlabels)
    out = []
    nb = [set() for _ in range(n)]
    for (a, b, w) in edges(g):
        nb[a].add(b)
        nb[b].add(a)
    for v in range(n):
        own = lab[v]
        labs = {lab[u] for u in nb[v]}
        w_own = omega(g, lab, v, own)
        for L in labs:
            if L == own or W[L] + int(g["vwgt"][v]) > B:
                continue
            if omega(g, lab, v, L) > w_own or (overload_rule and W[own] > B):
                out.append((v, L))
    return out


def optimal_cut(g, k, B):
    """Minimum cut over all k^n partitions with every block weight <= B
    (None if no such partition exists)."""
    n = len(g["xadj"]) - 1
    E = edges(g)
    c = [int(x) for x in g["vwgt"]]
    best = None
    for part in itertools.product(range(k), repeat=n):
        bw = [0] * k
        for v in range(n):
            bw[part[v]] += c[v]
        if max(bw) > B:
            continue
        ct = sum(w for (a, b, w) in E if part[a] != part[b])
        if best is None or ct < best:
            best = ct
    return best


def dense_adjacency(g):
    n = len(g["xadj"]) - 1
    A = np.zeros((n, n), dtype=np.int64)
    for (a, b, w) in edges(g):
        A[a, b] += w
        A[b, a] += w
    return A


def sync_plain_lp_step(g, lab, seed, rnd):
    """One synchronous (S = 1) unconstrained label-propagation step computed by
    brute force: every node looks at every label present among its neighbours,
    takes the strongest (ties: smaller tie hash, then smaller label) and moves
    iff that strictly beats its own label; all moves happen at once."""
    n = len(g["xadj"]) - 1
    nb = [set() for _ in range(n)]
    for (a, b, w) in edges(g):
        nb[a].add(b)
        nb[b].add(a)
    new = list(lab)
    for v in range(n):
        own = lab[v]
        cands = sorted({lab[u] for u in nb[v]} - {own})
        if not cands:
            continue
        scored = [(-omega(g, lab, v, L), tie(seed, rnd, v, L), L) for L in cands]
        s, _, L = min(scored)
        if -s > omega(g, lab, v, own):
            new[v] = L
    return new
