"""Failure detection without a GPU fault: the arbitration kernel's grid
barrier is the library's only in-kernel wait.  Its bound is exercised by a
launch in which one CTA never arrives; the waiting CTA must give up, raise the
error flag and return, the host must read SCLAP_ETIMEOUT, and the context must
stay usable for the next call."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_is_reported():
    import paper_1404_4797_gb300 as S
    # about a millisecond of waiting at GB300 clocks, then the flag
    assert S.wait_selftest(2_000_000) == S.ETIMEOUT
    assert S.wait_selftest(0) == S.ETIMEOUT
    # the next real call still runs and matches the oracle
    g = I.random_graph(3000, 15000, seed=8, max_w=5, max_c=3)
    gd = I.to_device(g, "cuda")
    k = 8
    p0 = I.rand_below(3, 1, torch.arange(3000), k).to(torch.int32)
    got, cut, bw, rd = S.sclap_refine(gd, k, 0.03, 4, 4, 5, p0.cuda())
    want = oracle.refine(I.to_numpy(g), k, 0.03, 4, 4, 5, p0.numpy())[0]
    assert np.array_equal(got.cpu().numpy(), want)


def test_wait_selftest_rejects_negative_limit():
    import paper_1404_4797_gb300 as S
    assert S.wait_selftest(-1) == S.EINVAL
