"""Sharded SCLaP on simulated ranks: the distributed-memory design (Sec. IV.A-C)
run as torch.distributed ranks on CPU (gloo), one process per rank.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: it shows that the
sharded design computes exactly what the single-rank oracle computes, and it is
run by ``tests/test_sharded.py`` with 2, 3 and 4 ranks.  The product is
single-GPU (several GPUs run independent replicas); this module is the
host-side protocol a multi-GPU product would follow, with each rank's local
arithmetic written here in numpy.

Layout (Sec. IV.A): rank r owns the contiguous node range [lo_r, hi_r) (1-D
partition, n/P nodes each), the rows of its nodes, and halo copies of the
labels of the non-owned neighbours of its nodes.  A cluster label is a node
id and lives with the owner of that node; the k block weights of refinement
are replicated (kept equal by an allreduce of the round's deltas, Sec. IV.B).

One sub-round (the method's reading R1-R5, as the oracle):
  1. every rank proposes for its nodes of the sub-round's colour against the
     state at sub-round start (clustering: the weights of the candidate
     labels are fetched from their owners first);
  2. refinement: departures from overloaded blocks are ordered by the
     block's owner (block b lives on rank b mod P), which returns keep flags;
  3. each proposal goes to the owner of its target, which admits them in
     (gain desc, id asc) order against the capacity and returns admit flags;
  4. admitted moves are applied; weight deltas go to the label owners
     (clustering) or are summed over all ranks (refinement);
  5. the new labels of moved boundary nodes go to the ranks that hold them as
     halo.
Because the admission order is a total order, every rank ends each sub-round
with the single-rank result.  Contraction (Sec. IV.C): used labels are marked
at their owners, an exclusive scan of the per-rank counts numbers them (the
coarse ids), every rank maps its nodes and halo, and each coarse edge (cu, cv,
w) goes to the owner of cu, which merges parallel edges.  Projection asks the
owner of each coarse node for its block.
"""
from __future__ import annotations

import numpy as np
import torch.distributed as dist

_M = np.uint64(0xFFFFFFFFFFFFFFFF)


def mix64(z):
    """SplitMix64 output function on uint64 numpy values (wrapping products)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def node_hash(seed, rnd, v):
    return mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(rnd + 1) << np.uint64(32))
                 ^ np.asarray(v, dtype=np.uint64))


def ranges(n, P):
    """Node range [lo, hi) of every rank: n/P nodes each, the last takes the rest."""
    per = n // P
    return [(r * per, (r + 1) * per if r < P - 1 else n) for r in range(P)]


def owner_of(x, bounds):
    """Rank owning each node id in x (bounds: the ranks' range starts)."""
    return np.searchsorted(bounds, np.asarray(x, dtype=np.int64), side="right") - 1


def exchange(outgoing):
    """All-to-all of python objects: outgoing[d] goes to rank d; returns the
    list of objects received, indexed by sender."""
    P = dist.get_world_size()
    rank = dist.get_rank()
    gathered = [None] * P
    dist.all_gather_object(gathered, outgoing)
    return [gathered[s][rank] for s in range(P)]


def allsum(x):
    y = [None] * dist.get_world_size()
    dist.all_gather_object(y, x)
    return sum(y)


class Shard:
    """One rank's part of a graph (global ids) with halo labels."""

    def __init__(self, g, P, rank):
        self.n = len(g["vwgt"])
        self.P, self.rank = P, rank
        self.rng = ranges(self.n, P)
        self.bounds = np.array([lo for lo, _ in self.rng], np.int64)
        self.lo, self.hi = self.rng[rank]
        lo, hi = self.lo, self.hi
        x = np.asarray(g["xadj"], np.int64)
        self.xadj = x[lo:hi + 1] - x[lo]
        self.adj = np.asarray(g["adjncy"][x[lo]:x[hi]], np.int64)
        self.w = np.asarray(g["adjwgt"][x[lo]:x[hi]], np.int64)
        self.c = np.asarray(g["vwgt"][lo:hi], np.int64)
        self.deg = np.diff(self.xadj)
        nb = self.adj[(self.adj < lo) | (self.adj >= hi)]
        self.halo = np.unique(nb)                       # sorted non-owned neighbours
        self.halo_owner = owner_of(self.halo, self.bounds)
        # which ranks hold each owned node as halo (sent to them when it moves)
        want = exchange([self.halo[self.halo_owner == d] for d in range(P)])
        self.watchers = {}
        for src, ids in enumerate(want):
            for v in ids:
                self.watchers.setdefault(int(v), []).append(src)

    def label_of(self, lab, halo_lab, u):
        """Labels of global ids u (owned or halo)."""
        u = np.asarray(u, np.int64)
        own = (u >= self.lo) & (u < self.hi)
        out = np.empty(u.size, np.int64)
        out[own] = lab[u[own] - self.lo]
        out[~own] = halo_lab[np.searchsorted(self.halo, u[~own])]
        return out


def _propose(sh, lab, halo_lab, Wq, B, seed, rnd, S, j, refine, lb_of):
    """Proposals (v, T, own, gain, c) of the rank's nodes of colour j.  Wq(L)
    returns the weight of label L at sub-round start."""
    props = []
    v_all = np.arange(sh.lo, sh.hi, dtype=np.int64)
    h = node_hash(seed, rnd, v_all)
    col = ((h >> np.uint64(32)) % np.uint64(S)).astype(np.int64)
    for i in np.nonzero((col == j) & (sh.deg > 0))[0]:
        v = sh.lo + i
        e0, e1 = sh.xadj[i], sh.xadj[i + 1]
        L = sh.label_of(lab, halo_lab, sh.adj[e0:e1])
        acc = {}
        for l, w in zip(L.tolist(), sh.w[e0:e1].tolist()):
            acc[l] = acc.get(l, 0) + w
        own = int(lab[i])
        w_own = acc.get(own, 0)
        cv = int(sh.c[i])
        overloaded = refine and Wq(own) > B
        best, key = None, None
        for l, w in acc.items():
            if l == own or Wq(l) + cv > B:
                continue
            t = int(mix64(h[i] ^ np.uint64(l - lb_of(v))) >> np.uint64(32))
            k = (-w, t, l)
            if key is None or k < key:
                best, key = l, k
        if best is not None:
            gain = acc[best] - w_own
            if gain > 0 or overloaded:
                props.append((int(v), best, own, gain, cv))
    return props


def _admit(props, cap):
    """Admission at one target: (gain desc, id asc) order, inclusive prefix of
    c <= cap (weight-0 moves always)."""
    out, s = {}, 0
    for v, T, own, gain, c in sorted(props, key=lambda p: (-p[3], p[0])):
        s += c
        out[v] = c == 0 or s <= cap
    return out


def lp_run(sh, lab, nW, B, refine, seed, rounds, S):
    """SCLaP rounds on the shard; lab: the owned nodes' labels (updated in place).
    Returns the rounds done.  Clustering: labels are node ids, the weight of
    label L lives at owner(L).  Refinement: nW block weights, replicated."""
    P, rank = sh.P, sh.rank
    # initial halo labels
    req = exchange([sh.halo[sh.halo_owner == d] for d in range(P)])
    rep = exchange([lab[np.asarray(ids, np.int64) - sh.lo] for ids in req])
    halo_lab = np.empty(sh.halo.size, np.int64)
    for d in range(P):
        halo_lab[sh.halo_owner == d] = rep[d]
    # label weights
    if refine:
        W = allsum(np.bincount(lab, weights=sh.c, minlength=nW).astype(np.int64))
    else:
        Wloc = sh.c.copy()               # label L = node L, owned by owner(L)
    owner_T = (lambda T: T % P) if refine else (lambda T: int(owner_of([T], sh.bounds)[0]))
    done = 0
    for rnd in range(rounds):
        moves = 0
        for j in range(S):
            if refine:
                Wq = lambda L: int(W[L])
            else:
                # fetch W of every label this rank's colour-j nodes may look at
                need = set(lab.tolist()) | set(halo_lab.tolist())
                need = np.array(sorted(need), np.int64)
                own_of = owner_of(need, sh.bounds)
                asked = exchange([need[own_of == d] for d in range(P)])
                got = exchange([Wloc[np.asarray(a, np.int64) - sh.lo] for a in asked])
                wmap = {}
                for d in range(P):
                    wmap.update(zip(need[own_of == d].tolist(), np.asarray(got[d]).tolist()))
                Wq = lambda L, m=wmap: int(m[L])
            props = _propose(sh, lab, halo_lab, Wq, B, seed, rnd, S, j, refine,
                             lambda v: 0)
            keep = {p[0]: True for p in props}
            if refine:  # R3: departures from overloaded blocks, ordered by the block owner
                out = [[] for _ in range(P)]
                for p in props:
                    if W[p[2]] > B:
                        out[p[2] % P].append(p)
                got = exchange(out)
                mine = [p for part in got for p in part]
                reply = [{} for _ in range(P)]
                by_b = {}
                for p in mine:
                    by_b.setdefault(p[2], []).append(p)
                for b, ps in by_b.items():
                    excess, dep = int(W[b]) - B, 0
                    for p in sorted(ps, key=lambda p: (-p[3], p[0])):
                        ok = dep < excess
                        if ok:
                            dep += p[4]
                        reply[int(owner_of([p[0]], sh.bounds)[0])][p[0]] = ok
                for part in exchange(reply):
                    keep.update(part)
            # R4: admission by the owner of each target
            out = [[] for _ in range(P)]
            for p in props:
                if keep[p[0]]:
                    out[owner_T(p[1])].append(p)
            got = exchange(out)
            by_t = {}
            for part in got:
                for p in part:
                    by_t.setdefault(p[1], []).append(p)
            reply = [{} for _ in range(P)]
            for T, ps in by_t.items():
                cap = B - (int(W[T]) if refine else int(Wloc[T - sh.lo]))
                for v, ok in _admit(ps, cap).items():
                    reply[int(owner_of([v], sh.bounds)[0])][v] = ok
            admitted = {}
            for part in exchange(reply):
                admitted.update(part)
            # R5: apply; weight deltas; halo updates
            delta = np.zeros(nW, np.int64) if refine else None
            wout = [[] for _ in range(P)]
            hout = [[] for _ in range(P)]
            for v, T, own, gain, c in props:
                if not admitted.get(v, False):
                    continue
                lab[v - sh.lo] = T
                moves += 1
                if refine:
                    delta[T] += c
                    delta[own] -= c
                else:
                    wout[owner_T(T)].append((T, c))
                    wout[owner_T(own)].append((own, -c))
                for d in sh.watchers.get(v, []):
                    hout[d].append((v, T))
            if refine:
                W = W + allsum(delta)
            else:
                for part in exchange(wout):
                    for L, dc in part:
                        Wloc[L - sh.lo] += dc
            for part in exchange(hout):
                for v, T in part:
                    halo_lab[np.searchsorted(sh.halo, v)] = T
        done = rnd + 1
        if allsum(moves) == 0:
            break
    return done


def pack_isolated(sh, lab, U):
    """R6: nodes without neighbours, in id order, into groups of weight <= U
    (U' = U - cmax + 1, group floor(P(v)/U'), labelled by its smallest id);
    the prefix P(v) runs over the ranks by an exclusive scan."""
    iso = np.nonzero(sh.deg == 0)[0]
    cmax = max(x for x in _allgather(int(sh.c[iso].max()) if iso.size else 0))
    tot = _allgather(int(sh.c[iso].sum()))
    if sum(_allgather(int(iso.size))) == 0:
        return
    Up = U - cmax + 1
    P0 = sum(tot[:sh.rank])
    pre = P0 + np.concatenate([[0], np.cumsum(sh.c[iso])[:-1]]).astype(np.int64)
    grp = pre // Up
    first = {}
    for g_, i in zip(grp.tolist(), iso.tolist()):
        first.setdefault(g_, sh.lo + i)
    rep = {}
    for part in _allgather(first):
        for g_, v in part.items():
            rep[g_] = min(rep.get(g_, v), v)
    for g_, i in zip(grp.tolist(), iso.tolist()):
        lab[i] = rep[g_]


def _allgather(x):
    y = [None] * dist.get_world_size()
    dist.all_gather_object(y, x)
    return y


def cluster(g, U, rounds, S, seed):
    """Sharded size-constrained clustering (R1-R6); returns (this rank's labels,
    node range, rounds done)."""
    P, rank = dist.get_world_size(), dist.get_rank()
    sh = Shard(g, P, rank)
    lab = np.arange(sh.lo, sh.hi, dtype=np.int64)
    rd = lp_run(sh, lab, sh.n, U, False, seed, rounds, S) if rounds > 0 else 0
    pack_isolated(sh, lab, U)
    return lab, (sh.lo, sh.hi), rd


def refine(g, k, B, rounds, S, seed, part):
    """Sharded refinement with bound B on k blocks; part: the full start
    partition (each rank uses its range).  Returns (this rank's blocks, range,
    rounds done)."""
    P, rank = dist.get_world_size(), dist.get_rank()
    sh = Shard(g, P, rank)
    lab = np.asarray(part, np.int64)[sh.lo:sh.hi].copy()
    rd = lp_run(sh, lab, k, B, True, seed, rounds, S)
    return lab, (sh.lo, sh.hi), rd


def contract(g, labels_full):
    """Sharded contraction (Sec. IV.C) of the clustering labels_full.  Returns
    this rank's part: (coarse node range, its rows as (cxadj, cadj, cw), its
    coarse weights, f2c of its fine nodes)."""
    P, rank = dist.get_world_size(), dist.get_rank()
    sh = Shard(g, P, rank)
    lab = np.asarray(labels_full, np.int64)[sh.lo:sh.hi]
    # used labels are marked at their owners; an exclusive scan numbers them
    lo_of = owner_of(lab, sh.bounds)
    marked = exchange([np.unique(lab[lo_of == d]) for d in range(P)])
    used = np.unique(np.concatenate([np.asarray(m, np.int64) for m in marked]))
    counts = _allgather(int(used.size))
    base = sum(counts[:rank])
    q = dict(zip(used.tolist(), range(base, base + used.size)))
    # ask the label owners for the coarse ids of this rank's labels and halo labels
    halo_lab = np.asarray(labels_full, np.int64)[sh.halo] if sh.halo.size else np.zeros(0, np.int64)
    want = np.unique(np.concatenate([lab, halo_lab]))
    wo = owner_of(want, sh.bounds)
    asked = exchange([want[wo == d] for d in range(P)])
    answers = exchange([[q[int(L)] for L in a] for a in asked])
    qmap = {}
    for d in range(P):
        qmap.update(zip(want[wo == d].tolist(), answers[d]))
    f2c = np.array([qmap[int(L)] for L in lab], np.int64)
    fh = np.array([qmap[int(L)] for L in halo_lab], np.int64)
    # coarse ids are owned by the owner of their label: contiguous ranges
    cbounds = np.array(np.cumsum([0] + counts[:-1]), np.int64)
    # coarse weights and edges go to the owner of the coarse node
    wout = [[] for _ in range(P)]
    eout = [[] for _ in range(P)]
    for i in range(sh.hi - sh.lo):
        cu = int(f2c[i])
        d = int(owner_of([cu], cbounds)[0])
        wout[d].append((cu, int(sh.c[i])))
        for e in range(sh.xadj[i], sh.xadj[i + 1]):
            u = int(sh.adj[e])
            cv = int(f2c[u - sh.lo]) if sh.lo <= u < sh.hi else int(fh[np.searchsorted(sh.halo, u)])
            if cv != cu:
                eout[d].append((cu, cv, int(sh.w[e])))
    clo = base
    chi = base + used.size
    cvw = np.zeros(used.size, np.int64)
    for part in exchange(wout):
        for cu, c in part:
            cvw[cu - clo] += c
    merged = {}
    for part in exchange(eout):
        for cu, cv, w in part:
            merged[(cu, cv)] = merged.get((cu, cv), 0) + w
    keys = sorted(merged)
    cxadj = np.zeros(used.size + 1, np.int64)
    for cu, _ in keys:
        cxadj[cu - clo + 1] += 1
    cxadj = np.cumsum(cxadj)
    cadj = np.array([cv for _, cv in keys], np.int64)
    cw = np.array([merged[kk] for kk in keys], np.int64)
    return (clo, chi), (cxadj, cadj, cw), cvw, f2c


def project(f2c_local, coarse_part_full):
    """Uncoarsening: the block of each owned fine node from its coarse node
    (the full coarse partition stands for the owners' replies)."""
    return np.asarray(coarse_part_full, np.int64)[np.asarray(f2c_local, np.int64)]
