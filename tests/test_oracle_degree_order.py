"""Pins of degree-ordered clustering sub-rounds (the closest synchronous
analogue of the paper's increasing-degree traversal): group sizes, the
degree order, the hash order inside a degree, S = 1 equal to hash colours,
and the clustering invariants."""
import numpy as np
import pytest

import oracle
from paper_1404_4797_gb300 import inputs as I
from tests import brute

GRAPHS = {
    "chunglu": lambda: I.to_numpy(I.chung_lu(2048, 2.1, 8.0, seed=3)),
    "weighted": lambda: I.to_numpy(I.random_graph(3000, 12000, seed=5, max_w=20, max_c=9)),
}


@pytest.mark.parametrize("S", [1, 3, 4, 8])
def test_groups_are_balanced_and_in_degree_order(S):
    g = GRAPHS["chunglu"]()
    n = g["vwgt"].size
    deg = np.diff(g["xadj"])
    for rnd in (0, 1, 5):
        col = oracle.degree_colours(g, 11, rnd, S)
        sizes = np.bincount(col, minlength=S)
        assert sizes.max() - sizes.min() <= 1 and sizes.sum() == n
        # every node of sub-round j has degree <= every node of sub-round j + 1
        for j in range(S - 1):
            assert deg[col == j].max() <= deg[col == j + 1].min()


def test_hash_order_inside_a_degree_and_per_round_change():
    g = GRAPHS["chunglu"]()
    deg = np.diff(g["xadj"])
    S = 4
    c0 = oracle.degree_colours(g, 11, 0, S)
    c1 = oracle.degree_colours(g, 11, 1, S)
    assert not np.array_equal(c0, c1)  # the split inside boundary degrees moves per round
    # inside one degree value, a node with a smaller hash never acts later
    d = int(np.bincount(deg).argmax())
    nodes = np.nonzero(deg == d)[0]
    h = np.array([brute.mix64(11 ^ (1 << 32) ^ int(v)) >> 32 for v in nodes])  # h(v, 0) >> 32
    order = nodes[np.argsort(h, kind="stable")]
    assert np.all(np.diff(c0[order]) >= 0)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_one_subround_equals_hash_colours(name):
    g = GRAPHS[name]()
    cV = int(g["vwgt"].sum())
    U = max(int(g["vwgt"].max()), cV // 40)
    a, ra = oracle.cluster(g, U, 5, 1, 7)
    b, rb = oracle.cluster(g, U, 5, 1, 7, degree_ordered=True)
    assert np.array_equal(a, b) and ra == rb


@pytest.mark.parametrize("name", list(GRAPHS))
def test_degree_ordered_clustering_invariants(name):
    g = GRAPHS[name]()
    cV = int(g["vwgt"].sum())
    U = max(int(g["vwgt"].max()), cV // 40)
    lab, rd = oracle.cluster(g, U, 30, 4, 7, degree_ordered=True)
    w = np.bincount(lab, weights=g["vwgt"], minlength=lab.size)
    assert w.max() <= U
    if rd < 30:  # converged: no admissible improving move is left
        assert brute.improving_moves(g, lab, lab.size, U, False) == []
