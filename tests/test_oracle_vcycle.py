"""Pins of the oracle's iterated V-cycle: constrained coarsening keeps every
cluster inside one block, so with no refinement anywhere the cycle returns
its input partition; balance and determinism otherwise."""
import numpy as np
import pytest

import oracle
from paper_1404_4797_gb300 import inputs as I

GRAPHS = {
    "chunglu": lambda: I.to_numpy(I.chung_lu(4096, 2.1, 8.0, seed=3)),
    "weighted": lambda: I.to_numpy(I.random_graph(5000, 20000, seed=5, max_w=20, max_c=9)),
    "sparse": lambda: I.to_numpy(I.random_graph(4000, 1500, seed=9)),  # isolated nodes
}


def params(k, **kw):
    p = oracle.default_params(k, 0.03, 7)
    p.update(n_stop=200)
    p.update(kw)
    return p


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("k", [2, 8])
def test_without_refinement_the_cycle_returns_its_input(name, k):
    g = GRAPHS[name]()
    n = g["vwgt"].size
    part = ((np.arange(n, dtype=np.int64) * 2654435761) % k).astype(np.int32)
    out, st = oracle.vcycle(g, params(k, refine_rounds=0, init_rounds=0), part)
    assert np.array_equal(out, part)
    assert st["levels"] >= 2 and st["init_best"] == -1
    assert st["cut"] == oracle.cut(g, part)
    # the coarsest graph carries the same cut and block weights
    assert st["init_cut"] == st["cut"]
    assert st["init_maxbw"] == int(oracle.block_weights(g, part, k).max())


@pytest.mark.parametrize("name", list(GRAPHS))
def test_cycle_after_multilevel_stays_feasible_and_is_deterministic(name):
    g = GRAPHS[name]()
    k = 8
    p0, s0 = oracle.multilevel(g, params(k))
    p1, s1 = oracle.vcycle(g, params(k, seed=8), p0)
    p2, s2 = oracle.vcycle(g, params(k, seed=8), p0)
    assert np.array_equal(p1, p2) and s1 == s2
    assert s1["maxbw"] <= s1["lmax"] or s0["maxbw"] > s0["lmax"]
    assert s1["cut"] == oracle.cut(g, p1)
    assert 0 <= p1.min() and p1.max() < k


def test_cycle_rejects_out_of_range_blocks():
    g = GRAPHS["weighted"]()
    part = np.zeros(g["vwgt"].size, np.int32)
    part[3] = 5
    with pytest.raises(oracle.OracleError):
        oracle.vcycle(g, params(4), part)


def _level_seed(seed, l):
    return oracle.mix64(seed ^ ((0x9E3779B97F4A7C15 * (l + 1)) & (2**64 - 1)))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_every_level_of_the_cycle_carries_the_seed_partition(name):
    """Rebuilds the cycle's hierarchy from the constrained clustering and the
    contraction, one level at a time, and checks at every level what holds by
    construction (Sec. IV.E): each coarse node's members share one block, so
    the inherited partition has the input's block weights and cut.  The level
    sizes must be those the oracle's V-cycle reports."""
    g = GRAPHS[name]()
    k = 4
    n = g["vwgt"].size
    part = ((np.arange(n, dtype=np.int64) * 2654435761) % k).astype(np.int32)
    prm = params(k, refine_rounds=0, init_rounds=0)
    _, st = oracle.vcycle(g, prm, part)
    cV = int(g["vwgt"].sum())
    U = max(int(g["vwgt"].max()), cV // (10 * k))
    want_cut = oracle.cut(g, part)
    want_bw = oracle.block_weights(g, part, k)
    cur, cp, sizes = g, part, [n]
    for lvl in range(st["levels"] - 1):
        lab, _ = oracle.cluster(cur, U, prm["cluster_rounds"], prm["subrounds"],
                                _level_seed(prm["seed"], lvl), constraint_part=cp)
        assert np.array_equal(cp[lab], cp), "a cluster crosses a block"
        coarse, f2c = oracle.contract(cur, lab)
        ccp = np.full(coarse["vwgt"].size, -1, np.int32)
        ccp[f2c] = cp
        assert np.array_equal(ccp[f2c], cp) and (ccp >= 0).all()
        assert oracle.cut(coarse, ccp) == want_cut
        assert np.array_equal(oracle.block_weights(coarse, ccp, k), want_bw)
        cur, cp = coarse, ccp
        sizes.append(coarse["vwgt"].size)
    assert sizes == st["n"]
