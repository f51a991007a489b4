"""The allocation-free cut entry point (sclap_cut_noalloc) against sclap_cut.

Some callers cannot let a library allocate device memory (for example while
another framework is capturing a CUDA graph, or when a custom allocator owns
all memory); sclap_cut_noalloc serves them from a fixed device array.  This file
is collected last on purpose.  It checks two calls in a row, so a result left in
the shared array by the first call cannot leak into the second."""
import numpy as np
import pytest
import torch

from paper_1404_4797_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_cut_noalloc_matches_cut_on_two_calls_in_a_row():
    import paper_1404_4797_gb300 as S
    g1 = I.to_device(I.random_graph(5000, 30000, seed=3, max_w=9, max_c=5), "cuda")
    g2 = I.to_device(I.rmat(14, 16, seed=5), "cuda")
    cases = [(g1, 16, 11), (g2, 300, 12), (g1, 16, 13)]
    for g, k, seed in cases:
        n = g["vwgt"].numel()
        part = I.rand_below(seed, 1, torch.arange(n, device="cuda"), k).to(torch.int32)
        want_cut, want_bw = S.sclap_cut(g, part, k)
        got_cut, got_bw = S.sclap_cut_noalloc(g, part, k)
        assert got_cut == want_cut
        assert np.array_equal(got_bw.numpy(), want_bw.numpy())


def test_cut_noalloc_rejects_k_beyond_its_array():
    import paper_1404_4797_gb300 as S
    g = I.to_device(I.random_graph(100, 300, seed=1), "cuda")
    part = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SclapError) as e:
        S.sclap_cut_noalloc(g, part, 65537)
    assert e.value.code == S.EINVAL
