"""The Python binding's argument checks, which run before any CUDA call (no
GPU needed): CPU tensors, wrong dtypes and wrong parameter sizes are
rejected with TypeError; the status table matches the header."""
import pytest
import torch

import paper_1404_4797_gb300 as S
from paper_1404_4797_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def _lib():
    S.lib()
    yield


def graph():
    return I.random_graph(50, 100, seed=1)


def test_cpu_tensors_are_rejected():
    g = graph()
    p = torch.zeros(50, dtype=torch.int32)
    with pytest.raises(TypeError):
        S.sclap_refine(g, 2, 0.03, 1, 1, 1, p)
    with pytest.raises(TypeError):
        S.sclap_refine_learned(g, 2, 0.03, 1, 1, 1, p)
    with pytest.raises(TypeError):
        S.sclap_mlp_score(torch.zeros(4, 6), torch.zeros(1313, dtype=torch.int16))


def test_graph_dtypes_are_checked():
    g = dict(graph())
    g["adjncy"] = g["adjncy"].to(torch.int64)
    with pytest.raises(TypeError):
        S._graph(g)
    g = dict(graph())
    g["xadj"] = g["xadj"].to(torch.int32)
    with pytest.raises(TypeError):
        S._graph(g)


def test_status_strings():
    want = {0: "ok", 1: "invalid argument", 2: "graph failed validation",
            3: "weights exceed the 32-bit range", 4: "out of device memory", 5: "CUDA error",
            6: "device wait timed out", 7: "not implemented", 99: "unknown error"}
    for code, text in want.items():
        assert S.lib().sclap_strerror(code).decode() == text


def test_default_params_are_the_fast_preset():
    p = S.default_params(16, 0.03, 1)
    assert p["k"] == 16 and p["eps"] == 0.03
    assert p["cluster_rounds"] == 3 and p["refine_rounds"] == 6
    assert p["subrounds"] == 4 and p["n_stop"] == 2000
