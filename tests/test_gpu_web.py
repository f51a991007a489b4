"""Config 3, the web-like graph: Chung-Lu (exponent 2.0, mean degree 32, hubs up
to ~2^20 neighbours) plus 5% uniform long-range edges.  A small instance is
checked bit for bit against the oracle.  The full instance (n = 2^26, ~1.1
billion edges, 2.2 billion directed entries, so row offsets and entry indices
beyond 2^31) is checked by properties that hold at any size: block ids in
range, the reported cut equal to an independent cut kernel's, the balance
bound, and level sizes that shrink."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_web_like_small_matches_oracle():
    import paper_1404_4797_gb300 as S
    g = I.web_graph(1 << 13, 2.0, 32.0, dmax=float(1 << 10), long_frac=0.05, seed=3)
    gn = I.to_numpy(g)
    prm = S.default_params(64, 0.03, seed=2, n_stop=1000)
    got, st = S.partition_multilevel(I.to_device(g, "cuda"), prm)
    want, ws = oracle.multilevel(gn, dict(prm))
    assert st == ws and np.array_equal(got.cpu().numpy(), want)


def test_web_like_full_size_properties():
    import paper_1404_4797_gb300 as S
    torch.cuda.empty_cache()
    g = I.web_graph(1 << 26, 2.0, 32.0, dmax=float(1 << 20), long_frac=0.05, seed=1,
                    device="cuda")
    torch.cuda.empty_cache()
    n, nnz = g["vwgt"].numel(), g["adjncy"].numel()
    assert nnz > 2**31  # entry offsets beyond 32 bits
    k = 64
    prm = S.default_params(k, 0.03, seed=1)
    old = S.set_validation(True)
    try:
        part, st = S.partition_multilevel(g, prm)
    finally:
        S.set_validation(old)
    p = part
    assert int(p.min()) >= 0 and int(p.max()) < k
    cut, bw = S.sclap_cut(g, p, k)
    assert cut == st["cut"] and int(bw.max()) == st["maxbw"] and int(bw.sum()) == n
    if st["init_maxbw"] <= st["lmax"]:
        assert st["maxbw"] <= st["lmax"]
    assert 0 < cut < nnz // 2
    ns = st["n"]
    assert all(ns[i + 1] < ns[i] for i in range(len(ns) - 1)) and st["nnz"][0] == nnz
