"""Parity at the benchmark's full size and launch configuration: the R-MAT scale-22
workload (k = 16, eps = 0.03, l = 3, r = 6, S = 4) partitioned by the CUDA path
and by the CPU oracle must agree bit for bit, level sizes included."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_rmat22_multilevel_bit_exact():
    import bench
    import paper_1404_4797_gb300 as S
    cfg = bench.WORKLOAD
    g = I.rmat(cfg["scale"], cfg["edge_factor"], seed=cfg["seed"], device="cuda")
    params = bench.params_for(cfg)
    t0 = time.perf_counter()
    part, st = S.partition_multilevel(g, params)
    torch.cuda.synchronize()
    t_gpu = time.perf_counter() - t0
    gn = I.to_numpy(g)
    t0 = time.perf_counter()
    want, ws = oracle.multilevel(gn, params)
    t_cpu = time.perf_counter() - t0
    print(f"\nR-MAT 22: n={gn['vwgt'].size} m={gn['adjncy'].size // 2} levels={st['n']} "
          f"cut={st['cut']} maxbw={st['maxbw']} lmax={st['lmax']} gpu {t_gpu:.3f}s "
          f"oracle {t_cpu:.1f}s")
    assert st == ws
    assert np.array_equal(part.cpu().numpy(), want)
