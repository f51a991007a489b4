"""The C ABI library loads and exports every function include/sclap.h declares
(no compute: runs without a GPU)."""
import ctypes
import os
import re

from paper_1404_4797_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sclap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sclap_cluster", "sclap_refine", "contract_graph", "project_partition",
                 "partition_multilevel", "sclap_graph_free", "sclap_strerror",
                 "sclap_refine_batched", "sclap_refine_learned", "sclap_mlp_score",
                 "sclap_mlp_loss_grad", "sclap_mlp_train", "sclap_cut_noalloc"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1404_4797_gb300 as S
    assert set(S.EXPORTS) <= set(declared_functions())
    S.lib()
    assert S.strerror(S.EGRAPH) == "graph failed validation"


def test_alloc_failure_hook_rejects_bad_counts_without_a_gpu():
    import paper_1404_4797_gb300 as S
    S.lib()
    with __import__("pytest").raises(S.SclapError) as e:
        S.inject_alloc_failure(-2)
    assert e.value.code == S.EINVAL
    S.inject_alloc_failure(-1)  # off: no device work involved
