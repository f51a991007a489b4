"""Seeded synthetic graph generators (inputs only; none of the method's arithmetic).

Both the CUDA path and the CPU oracle consume the arrays these functions return:
a graph is generated once, on one device, and the same bytes are handed to both.
All randomness is counter based -- a SplitMix64 output function applied to
(seed, stream, index) -- and written with plain torch integer ops, so one
function serves CPU and GPU without a stateful generator.

A graph is a dict of torch tensors in CSR form (both directions of every
undirected edge stored, no self-loops, no duplicate entries):
  xadj   int64 [n+1]   row offsets
  adjncy int32 [nnz]   neighbour ids
  adjwgt int32 [nnz]   edge weights  (> 0)
  vwgt   int32 [n]     node weights  (>= 0)
The workloads stand in for the paper's social and web graphs (Table I), which
are not available here: Chung-Lu power-law graphs and R-MAT graphs.
"""
from __future__ import annotations

import math

import torch

_M64 = (1 << 64) - 1


def _s64(x: int) -> int:
    """uint64 constant -> the int64 with the same bits."""
    x &= _M64
    return x - (1 << 64) if x >= (1 << 63) else x


_C1 = _s64(0xBF58476D1CE4E5B9)
_C2 = _s64(0x94D049BB133111EB)
_GOLD = _s64(0x9E3779B97F4A7C15)


def _lsr(z: torch.Tensor, s: int) -> torch.Tensor:
    return (z >> s) & ((1 << (64 - s)) - 1)


def hash64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 tensors holding uint64 bits."""
    z = (z ^ _lsr(z, 30)) * _C1
    z = (z ^ _lsr(z, 27)) * _C2
    return z ^ _lsr(z, 31)


def _stream_key(seed: int, stream: int) -> int:
    z = (seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return _s64(z ^ (z >> 31))


def rand_bits(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """64 random bits per index (int64 tensor)."""
    return hash64((idx * _GOLD) ^ _stream_key(seed, stream))


def rand_uniform(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return _lsr(rand_bits(seed, stream, idx), 11).to(torch.float64) * (2.0 ** -53)


def rand_below(seed: int, stream: int, idx: torch.Tensor, bound: int) -> torch.Tensor:
    """Integers in [0, bound) (63-bit draw reduced mod bound)."""
    return _lsr(rand_bits(seed, stream, idx), 1) % bound


def permutation(n: int, seed: int, stream: int, device) -> torch.Tensor:
    """A seeded permutation of 0..n-1 (sort by hash, ties impossible to matter)."""
    idx = torch.arange(n, dtype=torch.int64, device=device)
    key = _lsr(rand_bits(seed, stream, idx), 1)
    return torch.argsort(key, stable=True)


def csr_from_edges(n: int, u: torch.Tensor, v: torch.Tensor, w: torch.Tensor | None = None,
                   vwgt: torch.Tensor | None = None) -> dict:
    """Undirected edge list -> symmetric CSR.  Self-loops are dropped and duplicate
    pairs are merged (their weights summed)."""
    device = u.device
    u = u.to(torch.int64)
    v = v.to(torch.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    if w is None:
        w = torch.ones_like(u)
    else:
        w = w.to(torch.int64)[keep]
    a = torch.minimum(u, v)
    b = torch.maximum(u, v)
    key = a * n + b
    ukey, inv = torch.unique(key, return_inverse=True)
    uw = torch.zeros(ukey.numel(), dtype=torch.int64, device=device)
    uw.index_add_(0, inv, w)
    a = ukey // n
    b = ukey % n
    src = torch.cat([a, b])
    dst = torch.cat([b, a])
    ww = torch.cat([uw, uw])
    order = torch.argsort(src * n + dst)
    src, dst, ww = src[order], dst[order], ww[order]
    deg = torch.bincount(src, minlength=n)
    xadj = torch.zeros(n + 1, dtype=torch.int64, device=device)
    xadj[1:] = torch.cumsum(deg, 0)
    if vwgt is None:
        vwgt = torch.ones(n, dtype=torch.int32, device=device)
    if ww.numel() and int(ww.max()) > 2**31 - 1:
        raise ValueError("edge weight does not fit int32")
    return {"xadj": xadj, "adjncy": dst.to(torch.int32).contiguous(),
            "adjwgt": ww.to(torch.int32).contiguous(), "vwgt": vwgt.to(torch.int32).contiguous()}


def csr_from_unique_keys(n: int, key: torch.Tensor, vwgt: torch.Tensor | None = None) -> dict:
    """Symmetric unit-weight CSR from sorted, distinct keys a * n + b with a < b
    (undirected edges).  The same arrays csr_from_edges returns, built without
    sorting all 2m entries: row v holds its smaller neighbours (from the edges
    (b, v), ordered by a stable sort on b) followed by its larger ones (the
    edges (v, b), already in order)."""
    device = key.device
    a = key // n
    b = key % n
    deg_fwd = torch.bincount(a, minlength=n)
    deg_rev = torch.bincount(b, minlength=n)
    xadj = torch.zeros(n + 1, dtype=torch.int64, device=device)
    xadj[1:] = torch.cumsum(deg_fwd + deg_rev, 0)
    nnz = int(xadj[-1])
    adjncy = torch.empty(nnz, dtype=torch.int32, device=device)
    # larger neighbours: edge i (a_i, b_i) is entry i - fwd_start[a_i] of a_i's upper part
    fwd_start = torch.cumsum(deg_fwd, 0) - deg_fwd
    i = torch.arange(key.numel(), dtype=torch.int64, device=device)
    pos = xadj[:-1][a] + deg_rev[a] + (i - fwd_start[a])
    adjncy[pos] = b.to(torch.int32)
    del pos
    # smaller neighbours: the edges in (b, a) order
    order = torch.sort(b, stable=True).indices
    bs, as_ = b[order], a[order]
    del order, a, b
    rev_start = torch.cumsum(deg_rev, 0) - deg_rev
    pos = xadj[:-1][bs] + (i - rev_start[bs])
    adjncy[pos] = as_.to(torch.int32)
    del pos, bs, as_, i
    if vwgt is None:
        vwgt = torch.ones(n, dtype=torch.int32, device=device)
    return {"xadj": xadj, "adjncy": adjncy,
            "adjwgt": torch.ones(nnz, dtype=torch.int32, device=device),
            "vwgt": vwgt.to(torch.int32).contiguous()}


def _chung_lu_pairs(n, gamma, mean_deg, seed, stream0, m_target, device, w=None, dmax=None):
    """Sample endpoint pairs with P(endpoint = i) proportional to the expected
    degree w_i ~ (i + i0)^(-1/(gamma-1)); i0 is chosen so that the largest expected
    degree is about dmax (default sqrt(n * mean_deg))."""
    beta = 1.0 / (gamma - 1.0)
    if dmax is None:
        dmax = math.sqrt(n * mean_deg)
    idx = torch.arange(n, dtype=torch.float64, device=device)
    # choose i0 with (i0)^-beta / mean((i+i0)^-beta) ~= dmax / mean_deg
    lo, hi = 0.0, float(n)
    for _ in range(60):
        i0 = 0.5 * (lo + hi)
        ww = (idx + i0) ** (-beta)
        ratio = float(ww[0] / ww.mean())
        if ratio > dmax / mean_deg:
            lo = i0
        else:
            hi = i0
    ww = (idx + max(i0, 1e-9)) ** (-beta) if w is None else w
    iw = torch.clamp((ww / ww.max() * (1 << 40)).to(torch.int64), min=1)
    cum = torch.cumsum(iw, 0)
    total = int(cum[-1])
    got = None
    drawn = 0
    stream = stream0
    while True:
        need = m_target - (0 if got is None else got.numel())
        if need <= 0:
            break
        batch = need
        s = torch.arange(drawn, drawn + batch, dtype=torch.int64, device=device)
        ra = rand_below(seed, stream, s, total)
        rb = rand_below(seed, stream + 1, s, total)
        a = torch.searchsorted(cum, ra, right=True)
        b = torch.searchsorted(cum, rb, right=True)
        drawn += batch
        keep = a != b
        a, b = a[keep], b[keep]
        key = torch.minimum(a, b) * n + torch.maximum(a, b)
        got = torch.unique(key if got is None else torch.cat([got, key]))
    return got


def chung_lu(n: int = 16384, gamma: float = 2.1, mean_deg: float = 16.0, seed: int = 1,
             device="cpu") -> dict:
    """Chung-Lu power-law graph with about n*mean_deg/2 distinct undirected edges,
    node ids permuted by a seeded permutation, unit weights."""
    m_target = int(n * mean_deg / 2)
    key = _chung_lu_pairs(n, gamma, mean_deg, seed, 10, m_target, device)
    a, b = key // n, key % n
    perm = permutation(n, seed, 20, device)
    return csr_from_edges(n, perm[a], perm[b])


def rmat(scale: int = 22, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1, device="cpu", chunk: int = 1 << 24) -> dict:
    """R-MAT graph (Graph500 style): 2^scale nodes, edge_factor * 2^scale samples,
    quadrant probabilities a, b, c, d = 1-a-b-c, random vertex relabelling,
    symmetrised, duplicates merged into unit-weight edges, self-loops dropped."""
    n = 1 << scale
    m = edge_factor * n
    perm = permutation(n, seed, 1, device)
    keys = []
    for start in range(0, m, chunk):
        cnt = min(chunk, m - start)
        s = torch.arange(start, start + cnt, dtype=torch.int64, device=device)
        src = torch.zeros(cnt, dtype=torch.int64, device=device)
        dst = torch.zeros(cnt, dtype=torch.int64, device=device)
        for lvl in range(scale):
            u = rand_uniform(seed, 100 + lvl, s)
            bit_dst = ((u >= a) & (u < a + b)) | (u >= a + b + c)
            bit_src = u >= a + b
            src |= bit_src.to(torch.int64) << lvl
            dst |= bit_dst.to(torch.int64) << lvl
        src, dst = perm[src], perm[dst]
        keep = src != dst
        src, dst = src[keep], dst[keep]
        keys.append(torch.unique(torch.minimum(src, dst) * n + torch.maximum(src, dst)))
        del s, src, dst
    key = torch.unique(torch.cat(keys))
    del keys
    u, v = key // n, key % n
    del key
    g = csr_from_edges(n, u, v)
    return g


def web_graph(n: int = 1 << 26, gamma: float = 2.0, mean_deg: float = 32.0,
              dmax: float = float(1 << 20), long_frac: float = 0.05, seed: int = 1,
              device="cpu") -> dict:
    """Web-like graph: n * mean_deg / 2 Chung-Lu edges (exponent gamma, largest
    expected degree about dmax) plus long_frac as many again between uniform
    random endpoints; ids permuted, unit weights, duplicates merged."""
    m = int(n * mean_deg / 2)
    m_long = int(m * long_frac)
    key = _chung_lu_pairs(n, gamma, mean_deg, seed, 30, m, device, dmax=dmax)
    s = torch.arange(m_long, dtype=torch.int64, device=device)
    la = rand_below(seed, 40, s, n)
    lb = rand_below(seed, 41, s, n)
    del s
    keep = la != lb
    la, lb = la[keep], lb[keep]
    key = torch.unique(torch.cat([key, torch.minimum(la, lb) * n + torch.maximum(la, lb)]))
    del la, lb, keep
    perm = permutation(n, seed, 42, device)
    a, b = perm[key // n], perm[key % n]
    del key, perm
    key = torch.sort(torch.minimum(a, b) * n + torch.maximum(a, b)).values
    del a, b
    return csr_from_unique_keys(n, key)


def rgg(scale: int, seed: int = 1, device="cpu", radius_factor: float = 0.55) -> dict:
    """Random geometric graph rggX (the paper's mesh-type family, Sec. V.A):
    n = 2^scale points uniform in the unit square, an edge between two points
    whose Euclidean distance is below radius_factor * sqrt(ln n / n); unit
    weights.  Node ids follow the points' grid-cell order (row-major cells of
    side >= the radius), so neighbours have nearby ids as in mesh orderings.
    Pairs are found cell by cell: each point against its own cell (higher ids)
    and four of its eight neighbouring cells, which covers every pair once."""
    n = 1 << scale
    r = radius_factor * math.sqrt(math.log(n) / n)
    idx = torch.arange(n, dtype=torch.int64, device=device)
    x = rand_uniform(seed, 700, idx)
    y = rand_uniform(seed, 701, idx)
    G = max(1, int(1.0 / r))                   # G x G cells of side 1/G >= r
    cx = torch.clamp((x * G).to(torch.int64), max=G - 1)
    cy = torch.clamp((y * G).to(torch.int64), max=G - 1)
    order = torch.argsort(cy * G + cx, stable=True)
    x, y, cx, cy = x[order], y[order], cx[order], cy[order]
    cell = cy * G + cx
    counts = torch.bincount(cell, minlength=G * G)
    start = torch.cumsum(counts, 0) - counts
    us, vs = [], []
    r2 = r * r
    for dx, dy in ((0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)):
        nx, ny = cx + dx, cy + dy
        ok = (nx >= 0) & (nx < G) & (ny < G)
        p = idx[ok]
        nc = (ny * G + nx)[ok]
        cnt = counts[nc]
        tot = int(cnt.sum())
        if tot == 0:
            continue
        rep_p = torch.repeat_interleave(p, cnt)
        base = torch.repeat_interleave(start[nc] - (torch.cumsum(cnt, 0) - cnt), cnt)
        q = base + torch.arange(tot, dtype=torch.int64, device=device)
        d2 = (x[rep_p] - x[q]) ** 2 + (y[rep_p] - y[q]) ** 2
        keep = d2 < r2
        if dx == 0 and dy == 0:
            keep &= q > rep_p
        us.append(rep_p[keep])
        vs.append(q[keep])
        del rep_p, base, q, d2, keep
    u = torch.cat(us) if us else idx[:0]
    v = torch.cat(vs) if vs else idx[:0]
    return csr_from_edges(n, u, v)


def population(count: int = 32, nmin: int = 2000, nmax: int = 200000, seed: int = 1,
               device="cpu") -> list:
    """Coarse-graph population: `count` Chung-Lu graphs (gamma 2.1, mean degree
    8) with n log-uniform in [nmin, nmax], node weights uniform in 1..500 and
    edge weights lognormal(mu = 3, sigma = 1.5) rounded and clamped to 1..1000
    (Box-Muller from two counter-based uniforms keyed by the edge)."""
    import math
    graphs = []
    for t in range(count):
        u = float(rand_uniform(seed, 500 + t, torch.zeros(1, dtype=torch.int64))[0])
        n = int(round(math.exp(math.log(nmin) + u * (math.log(nmax) - math.log(nmin)))))
        base = chung_lu(n, 2.1, 8.0, seed=seed * 1000 + t, device=device)
        src = torch.repeat_interleave(torch.arange(n, device=device),
                                      base["xadj"][1:] - base["xadj"][:-1])
        dst = base["adjncy"].to(torch.int64)
        up = src < dst
        a, b = src[up], dst[up]
        key = a * n + b
        u1 = rand_uniform(seed * 1000 + t, 600, key).clamp_min(1e-12)
        u2 = rand_uniform(seed * 1000 + t, 601, key)
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
        w = torch.exp(3.0 + 1.5 * z).round().clamp(1, 1000).to(torch.int64)
        c = 1 + rand_below(seed * 1000 + t, 602, torch.arange(n, device=device), 500)
        graphs.append(csr_from_edges(n, a, b, w, c.to(torch.int32)))
    return graphs


def ring_of_cliques(k: int, s: int, bridges: int = 1, seed: int = 1, device="cpu") -> dict:
    """k cliques of s nodes (unit weights) in a ring: clique c is joined to
    clique (c + 1) mod k by `bridges` edges between uniformly drawn members;
    node ids permuted.  Returns the graph and the clique of every node (int64
    [k*s]).  The partition into the cliques cuts total weight k * bridges
    (repeated bridges merge and sum their weights); any partition that splits
    a clique cuts at least s - 1."""
    n = k * s
    i, j = torch.triu_indices(s, s, 1, device=device)
    base = torch.arange(k, dtype=torch.int64, device=device).repeat_interleave(i.numel()) * s
    u = base + i.repeat(k)
    v = base + j.repeat(k)
    b = torch.arange(k * bridges, dtype=torch.int64, device=device)
    c = b // bridges
    bu = c * s + rand_below(seed, 1, b, s)
    bv = ((c + 1) % k) * s + rand_below(seed, 2, b, s)
    perm = permutation(n, seed, 3, device)  # old id -> new id
    g = csr_from_edges(n, perm[torch.cat([u, bu])], perm[torch.cat([v, bv])])
    clique = torch.empty(n, dtype=torch.int64, device=device)
    clique[perm] = torch.arange(n, dtype=torch.int64, device=device) // s
    return g, clique


def path_graph(n: int, weights=None) -> dict:
    u = torch.arange(n - 1)
    v = u + 1
    w = None if weights is None else torch.tensor(weights, dtype=torch.int64)
    return csr_from_edges(n, u, v, w)


def random_graph(n: int, m: int, seed: int, max_w: int = 1, max_c: int = 1, device="cpu",
                 min_c: int = 1) -> dict:
    """Small Erdos-Renyi-like multigraph collapsed to a simple graph; weights uniform
    in 1..max_w (edges) and min_c..max_c (nodes)."""
    s = torch.arange(m, dtype=torch.int64, device=device)
    u = rand_below(seed, 1, s, n)
    v = rand_below(seed, 2, s, n)
    w = rand_below(seed, 3, s, max_w) + 1
    c = rand_below(seed, 4, torch.arange(n, dtype=torch.int64, device=device),
                   max_c - min_c + 1) + min_c
    return csr_from_edges(n, u, v, w, c.to(torch.int32))


def to_numpy(g: dict) -> dict:
    return {k: v.detach().cpu().numpy() for k, v in g.items()}


def to_device(g: dict, device) -> dict:
    return {k: v.to(device).contiguous() for k, v in g.items()}


def num_edges(g: dict) -> int:
    """Undirected edges m (= nnz / 2)."""
    return int(g["adjncy"].numel()) // 2
