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


@pytest.mark.parametrize("after", [0, 2, 8])
def test_injected_allocation_failure_is_reported_and_the_next_call_runs(after):
    """A scratch allocation made to fail (a host-side hook, no device fault):
    the call returns ENOMEM with its partition untouched, and the next call
    matches the oracle."""
    import paper_1404_4797_gb300 as S
    g = I.random_graph(3000, 15000, seed=9, max_w=5, max_c=3)
    gd = I.to_device(g, "cuda")
    k = 8
    p0 = I.rand_below(4, 1, torch.arange(3000), k).to(torch.int32)
    part = p0.cuda()
    S.inject_alloc_failure(after)
    try:
        with pytest.raises(S.SclapError) as e:
            S.sclap_refine(gd, k, 0.03, 4, 4, 5, part)
        assert e.value.code == S.ENOMEM
    finally:
        S.inject_alloc_failure(-1)
    assert torch.equal(part.cpu(), p0)
    got = S.sclap_refine(gd, k, 0.03, 4, 4, 5, part)[0]
    want = oracle.refine(I.to_numpy(g), k, 0.03, 4, 4, 5, p0.numpy())[0]
    assert np.array_equal(got.cpu().numpy(), want)


def test_injected_allocation_failure_inside_the_multilevel_call():
    import paper_1404_4797_gb300 as S
    g = I.chung_lu(4096, 2.1, 8.0, seed=3)
    gd = I.to_device(g, "cuda")
    prm = S.default_params(4, 0.03, 1, n_stop=300)
    S.inject_alloc_failure(25)
    try:
        with pytest.raises(S.SclapError) as e:
            S.partition_multilevel(gd, prm)
        assert e.value.code == S.ENOMEM
    finally:
        S.inject_alloc_failure(-1)
    got, st = S.partition_multilevel(gd, prm)
    want, wst = oracle.multilevel(I.to_numpy(g), dict(prm))
    assert st == wst and np.array_equal(got.cpu().numpy(), want)
