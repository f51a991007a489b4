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
