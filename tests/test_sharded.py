"""The sharded design (1-D node ranges with halos, proposal exchange to the
target owners, owner arbitration, exscan contraction; Sec. IV.A-C) on 2, 3 and
4 simulated ranks (gloo, CPU processes; 3 ranks own node ranges of unequal
sizes) gives bit for bit what the single-rank
oracle gives: clustering labels, refinement partitions, coarse graphs and
projections.  Not measured on GPUs: the product runs one GPU per process."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import sharded as SH
from paper_1404_4797_gb300 import inputs as I


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _graphs():
    return {
        "weighted": I.to_numpy(I.random_graph(700, 1800, seed=3, max_w=9, max_c=4)),
        "chunglu": I.to_numpy(I.chung_lu(1024, 2.1, 8.0, seed=5)),
    }


def _worker(rank, P, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=P)
    res = {}
    for name, g in _graphs().items():
        n = len(g["vwgt"])
        cV = int(g["vwgt"].sum())
        U = max(int(g["vwgt"].max()), cV // 40)
        lab, (lo, hi), rd = SH.cluster(g, U, 5, 4, 11)
        labs = [None] * P
        dist.all_gather_object(labs, (lo, lab, rd))
        full_lab = np.concatenate([x[1] for x in sorted(labs, key=lambda t: t[0])])
        k = 6
        B = oracle.lmax(cV, k, 0.03)
        p0 = (np.arange(n, dtype=np.int64) * 2654435761 % k).astype(np.int64)
        part, _, rr = SH.refine(g, k, B, 6, 4, 13, p0)
        parts = [None] * P
        dist.all_gather_object(parts, (lo, part, rr))
        full_part = np.concatenate([x[1] for x in sorted(parts, key=lambda t: t[0])])
        (clo, chi), (cx, ca, cw), cvw, f2c = SH.contract(g, full_lab)
        cparts = [None] * P
        dist.all_gather_object(cparts, (clo, chi, cx, ca, cw, cvw, lo, f2c))
        # projection of a coarse partition back to the fine nodes
        cn = max(t[1] for t in cparts)
        cpart = (np.arange(cn) * 40503 % k).astype(np.int64)
        proj = SH.project(f2c, cpart)
        projs = [None] * P
        dist.all_gather_object(projs, (lo, proj))
        if rank == 0:
            res[name] = dict(lab=full_lab, rd=[x[2] for x in labs], part=full_part,
                             rr=[x[2] for x in parts], coarse=sorted(cparts, key=lambda t: t[0]),
                             cpart=cpart,
                             proj=np.concatenate([x[1] for x in sorted(projs, key=lambda t: t[0])]))
    if rank == 0:
        np.save(os.path.join(out_dir, "res.npy"), res, allow_pickle=True)
    dist.destroy_process_group()


@pytest.mark.parametrize("P", [2, 3, 4])
def test_sharded_ranks_match_the_single_rank_oracle(P, tmp_path):
    mp.spawn(_worker, args=(P, _free_port(), str(tmp_path)), nprocs=P, join=True)
    res = np.load(tmp_path / "res.npy", allow_pickle=True).item()
    for name, g in _graphs().items():
        r = res[name]
        n = len(g["vwgt"])
        cV = int(g["vwgt"].sum())
        U = max(int(g["vwgt"].max()), cV // 40)
        want_lab, want_rd = oracle.cluster(g, U, 5, 4, 11)
        assert np.array_equal(r["lab"], want_lab), name
        assert all(x == want_rd for x in r["rd"])
        k = 6
        B = oracle.lmax(cV, k, 0.03)
        p0 = (np.arange(n, dtype=np.int64) * 2654435761 % k).astype(np.int32)
        want_part, want_rr = oracle.refine_bound(g, k, B, 6, 4, 13, p0)
        assert np.array_equal(r["part"], want_part), name
        assert all(x == want_rr for x in r["rr"])
        cg, f2c = oracle.contract(g, want_lab)
        got_x = [0]
        got_a, got_w, got_c, got_f = [], [], [], []
        for clo, chi, cx, ca, cw, cvw, lo, f in r["coarse"]:
            got_x.extend((got_x[-1] + cx[1:]).tolist())
            got_a.extend(ca.tolist())
            got_w.extend(cw.tolist())
            got_c.extend(cvw.tolist())
            got_f.extend(f.tolist())
        assert np.array_equal(np.array(got_x), cg["xadj"]) and np.array_equal(got_a, cg["adjncy"])
        assert np.array_equal(got_w, cg["adjwgt"]) and np.array_equal(got_c, cg["vwgt"])
        assert np.array_equal(got_f, f2c)
        assert np.array_equal(r["proj"], oracle.project(f2c, r["cpart"].astype(np.int32)))
        # the runs moved nodes and the graph had isolated nodes to pack
        assert not np.array_equal(want_lab, np.arange(n))
