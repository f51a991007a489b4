"""The rggX generator (random geometric graphs, the paper's mesh-type inputs):
exact agreement with a brute-force all-pairs construction on small inputs,
symmetric canonical CSR, and the edge count of the paper's rgg26 entry."""
import math

import numpy as np
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I


def test_rgg_equals_brute_force_pairs():
    for scale, seed in ((8, 1), (10, 3), (11, 7)):
        n = 1 << scale
        g = I.to_numpy(I.rgg(scale, seed=seed))
        assert oracle.validate(g) == oracle.OK
        # the same points, every pair compared
        idx = torch.arange(n, dtype=torch.int64)
        x = I.rand_uniform(seed, 700, idx).numpy()
        y = I.rand_uniform(seed, 701, idx).numpy()
        r = 0.55 * math.sqrt(math.log(n) / n)
        d2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
        want = (d2 < r * r) & ~np.eye(n, dtype=bool)
        # relabel: the generator numbers points in grid-cell order
        G = max(1, int(1.0 / r))
        cx = np.minimum((x * G).astype(np.int64), G - 1)
        cy = np.minimum((y * G).astype(np.int64), G - 1)
        order = np.argsort(cy * G + cx, kind="stable")
        want = want[np.ix_(order, order)]
        got = np.zeros((n, n), dtype=bool)
        rows = np.repeat(np.arange(n), np.diff(g["xadj"]))
        got[rows, g["adjncy"]] = True
        assert np.array_equal(got, want)
        assert (g["adjwgt"] == 1).all() and (g["vwgt"] == 1).all()


def test_rgg_edge_count_matches_the_papers_rgg26_density():
    # Table I lists rgg26 with about 67.1M nodes and 575M edges: m ~ n * pi r^2 n / 2
    # with r = 0.55 sqrt(ln n / n), i.e. about 8.57 n for n = 2^26.  At a smaller
    # scale the same formula holds up to the boundary loss (points near the edge
    # of the square have fewer neighbours), a few percent here.
    n26 = 1 << 26
    per_node_26 = math.pi * 0.55 ** 2 * math.log(n26) / 2
    assert abs(per_node_26 * n26 / 575e6 - 1) < 0.01
    scale = 16
    n = 1 << scale
    g = I.rgg(scale, seed=2)
    m = I.num_edges(g)
    expect = math.pi * 0.55 ** 2 * math.log(n) / 2 * n
    assert 0.93 < m / expect < 1.0


def test_csr_from_unique_keys_equals_csr_from_edges():
    for n, m, seed in ((50, 200, 1), (1000, 6000, 2), (7, 0, 3)):
        s = torch.arange(m, dtype=torch.int64)
        u = I.rand_below(seed, 1, s, n)
        v = I.rand_below(seed, 2, s, n)
        keep = u != v
        key = torch.unique(torch.minimum(u[keep], v[keep]) * n + torch.maximum(u[keep], v[keep]))
        want = I.csr_from_edges(n, key // n, key % n)
        got = I.csr_from_unique_keys(n, key)
        for k in ("xadj", "adjncy", "adjwgt", "vwgt"):
            assert torch.equal(got[k], want[k]), k


def test_web_graph_adds_the_long_range_edges():
    n = 1 << 12
    g = I.web_graph(n, 2.0, 16.0, dmax=800.0, long_frac=0.05, seed=2)
    m = I.num_edges(g)
    assert oracle.validate(I.to_numpy(g)) == oracle.OK
    # n * mean / 2 Chung-Lu edges plus 5% more, minus the few long-range pairs
    # that repeat a Chung-Lu edge
    assert 1.04 < m / (n * 16 / 2) <= 1.05
