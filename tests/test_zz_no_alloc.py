"""The allocation-free cut entry point (sclap_cut_noalloc).

Some callers cannot let a library allocate device memory: loops with a latency
budget (cudaMalloc and cudaFree can synchronise the whole device) and programs
whose device memory is handed out by their own pool.  sclap_cut_noalloc serves
them from a fixed device array shared by every call.  This file is collected
last on purpose.  Calls run back to back, including a smaller k after a larger
one, so a sum left in the shared array by one call would show up in the next;
results are compared with sclap_cut and with the CPU oracle's cut and block
weights."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _part(n, k, seed):
    return I.rand_below(seed, 1, torch.arange(n), k).to(torch.int32)


def test_cut_noalloc_matches_cut_and_oracle_on_calls_in_a_row():
    import paper_1404_4797_gb300 as S
    g1h = I.random_graph(5000, 30000, seed=3, max_w=9, max_c=5)
    g2h = I.rmat(14, 16, seed=5)
    g1, g2 = I.to_device(g1h, "cuda"), I.to_device(g2h, "cuda")
    # k above 2048 takes the global-atomic path of the block-weight kernel;
    # 65536 is the largest k the fixed array holds; then k shrinks again
    cases = [(g1, g1h, 16, 11), (g2, g2h, 300, 12), (g2, g2h, 5000, 14),
             (g2, g2h, 65536, 15), (g1, g1h, 16, 13), (g1, g1h, 3, 16)]
    for g, gh, k, seed in cases:
        n = g["vwgt"].numel()
        ph = _part(n, k, seed)
        part = ph.cuda()
        want_cut, want_bw = S.sclap_cut(g, part, k)
        got_cut, got_bw = S.sclap_cut_noalloc(g, part, k)
        assert got_cut == want_cut
        assert np.array_equal(got_bw.numpy(), want_bw.numpy())
        gn = I.to_numpy(gh)
        assert got_cut == oracle.cut(gn, ph.numpy())
        assert np.array_equal(got_bw.numpy(), oracle.block_weights(gn, ph.numpy(), k))


def test_cut_noalloc_rejects_k_beyond_its_array():
    import paper_1404_4797_gb300 as S
    g = I.to_device(I.random_graph(100, 300, seed=1), "cuda")
    part = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SclapError) as e:
        S.sclap_cut_noalloc(g, part, 65537)
    assert e.value.code == S.EINVAL


@pytest.mark.parametrize("bad", [16, -1, 70000])
def test_cut_noalloc_and_cut_reject_block_ids_out_of_range(bad):
    import paper_1404_4797_gb300 as S
    g = I.to_device(I.random_graph(500, 2000, seed=2), "cuda")
    part = _part(500, 16, 4)
    part[7] = bad
    part = part.cuda()
    for fn in (S.sclap_cut_noalloc, S.sclap_cut):
        with pytest.raises(S.SclapError) as e:
            fn(g, part, 16)
        assert e.value.code == S.EINVAL
    # the next valid call is unaffected by the rejected one
    ok = _part(500, 16, 5).cuda()
    assert S.sclap_cut_noalloc(g, ok, 16)[0] == S.sclap_cut(g, ok, 16)[0]
