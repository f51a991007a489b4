"""Threshold invariance: the degree-bin and segment thresholds route rows and
contested segments between kernel paths that compute the same selection and
arbitration, so labels, partitions, coarse graphs and cuts must be identical
(and equal to the oracle's) under every setting; the autotuner must find them
identical too."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SETTINGS = [(32, 256, 4096, 6144), (32, 256, 2048, 6144), (4, 16, 512, 64), (8, 64, 1024, 2048),
            (16, 200, 512, 300)]


def _graph():
    # R-MAT rows of every class plus two stars whose hubs take the CTA-table
    # and cluster paths, weighted
    base = I.rmat(14, 16, seed=6)
    n0 = base["vwgt"].numel()
    src = torch.repeat_interleave(torch.arange(n0), base["xadj"][1:] - base["xadj"][:-1])
    dst = base["adjncy"].to(torch.int64)
    up = src < dst
    u, v = src[up], dst[up]
    hubs = [(0, 3000), (1, 9000)]
    us, vs = [u], [v]
    for h, cnt in hubs:
        leaves = (torch.arange(cnt) * 7919 + 13 + h) % n0
        us.append(torch.full((cnt,), h, dtype=torch.int64))
        vs.append(leaves)
    u, v = torch.cat(us), torch.cat(vs)
    w = I.rand_below(3, 9, u * n0 + v, 5) + 1
    c = I.rand_below(3, 10, torch.arange(n0), 4) + 1
    return I.csr_from_edges(n0, u, v, w, c.to(torch.int32))


def test_results_identical_under_every_threshold_setting():
    import paper_1404_4797_gb300 as S
    g = _graph()
    gn = I.to_numpy(g)
    gd = I.to_device(g, "cuda")
    n = gn["vwgt"].size
    k = 16
    U = max(int(gn["vwgt"].max()), int(gn["vwgt"].sum()) // 160)
    p0 = I.rand_below(5, 7, torch.arange(n), k).to(torch.int32)
    prm = S.default_params(k, 0.03, seed=2, n_stop=500)
    want_lab, _ = oracle.cluster(gn, U, 4, 4, 9)
    want_part = oracle.refine(gn, k, 0.03, 6, 4, 9, p0.numpy())[0]
    want_ml, want_st = oracle.multilevel(gn, dict(prm))
    old = S.get_tuning()
    try:
        for st_ in SETTINGS:
            S.set_tuning(*st_)
            lab, _ = S.sclap_cluster(gd, U, 4, 4, 9)
            assert np.array_equal(lab.cpu().numpy(), want_lab), st_
            part = S.sclap_refine(gd, k, 0.03, 6, 4, 9, p0.cuda())[0]
            assert np.array_equal(part.cpu().numpy(), want_part), st_
            cg, f2c = S.contract_graph(gd, lab)
            ocg, of2c = oracle.contract(gn, want_lab)
            assert np.array_equal(f2c.cpu().numpy(), of2c)
            for key in ("xadj", "adjncy", "adjwgt", "vwgt"):
                assert np.array_equal(cg[key].cpu().numpy(), ocg[key]), (st_, key)
            ml, st = S.partition_multilevel(gd, prm)
            assert st == want_st and np.array_equal(ml.cpu().numpy(), want_ml), st_
    finally:
        S.set_tuning(**old)


def test_tuning_rejects_unsupported_values():
    import paper_1404_4797_gb300 as S
    old = S.get_tuning()
    for bad in ((12, 256, 2048, 6144), (32, 300, 2048, 6144), (32, 16, 2048, 6144),
                (32, 256, 700, 6144), (32, 256, 2048, 7000), (32, 256, 2048, 10)):
        with pytest.raises(S.SclapError):
            S.set_tuning(*bad)
    assert S.get_tuning() == old


def test_autotuner_finds_candidates_identical_and_applies_the_fastest(tmp_path):
    import paper_1404_4797_gb300 as S
    from paper_1404_4797_gb300 import autotune
    g = I.to_device(_graph(), "cuda")
    old = S.get_tuning()
    try:
        res = autotune.autotune(g, 16, cache=str(tmp_path / "t.json"), reps=1)
        assert res["identical"]
        assert S.get_tuning() == res["best"]
        again = autotune.load_or_tune(g, 16, cache=str(tmp_path / "t.json"))
        assert again["cached"] and again["best"] == res["best"]
    finally:
        S.set_tuning(**old)


def test_autotuner_on_the_multilevel_call(tmp_path):
    """Tuning on the whole multilevel partition: every candidate returns the
    same partition, and the cache entry is keyed apart from the sweep one."""
    import paper_1404_4797_gb300 as S
    from paper_1404_4797_gb300 import autotune
    g = I.to_device(_graph(), "cuda")
    params = S.default_params(8, 0.03, 3)
    old = S.get_tuning()
    try:
        cache = str(tmp_path / "t.json")
        res = autotune.autotune(g, 8, cache=cache, reps=1, ml_params=params,
                                candidates=autotune.CANDIDATES[:3])
        assert res["identical"] and res["workload"] == "multilevel"
        assert S.get_tuning() == res["best"]
        sweeps = autotune.load_or_tune(g, 8, cache=cache)
        assert not sweeps["cached"]  # a different entry
        again = autotune.load_or_tune(g, 8, cache=cache, ml_params=params)
        assert again["cached"] and again["best"] == res["best"]
    finally:
        S.set_tuning(**old)
