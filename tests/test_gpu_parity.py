"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element, on seeded inputs.  Integer work: bit-exact equality is the bar."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I

pytestmark = pytest.mark.gpu

S = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global S
    import paper_1404_4797_gb300 as mod
    mod.lib()
    S = mod
    yield


def dev(g):
    return I.to_device(g, "cuda")


def star(n_leaves, w=1):
    u = torch.zeros(n_leaves, dtype=torch.int64)
    v = torch.arange(1, n_leaves + 1, dtype=torch.int64)
    return I.csr_from_edges(n_leaves + 1, u, v, torch.full((n_leaves,), w, dtype=torch.int64))


GRAPHS = {
    "chunglu2k": lambda: I.chung_lu(2048, 2.1, 8.0, seed=3),
    "weighted": lambda: I.random_graph(3000, 12000, seed=5, max_w=20, max_c=9),
    "rmat14": lambda: I.rmat(14, 16, seed=2),
    "star5k": lambda: star(5000),                # hub beyond shared memory
    "stars": lambda: I.csr_from_edges(                # hubs of 600, 1600 and 3100 leaves
        5303, torch.cat([torch.zeros(600), torch.ones(1600), torch.full((3100,), 2)]).long(),
        torch.arange(3, 5303), (torch.arange(5300) % 7 + 1)),
    "sparse": lambda: I.random_graph(4000, 1500, seed=9),  # many isolated nodes
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("Sr", [1, 4])
def test_cluster_matches_oracle(name, Sr):
    g = GRAPHS[name]()
    gn = I.to_numpy(g)
    cV = int(gn["vwgt"].sum())
    U = max(int(gn["vwgt"].max()), cV // 40)
    want, rd_w = oracle.cluster(gn, U, 5, Sr, 11)
    got, rd_g = S.sclap_cluster(dev(g), U, 5, Sr, 11)
    assert rd_g == rd_w
    assert np.array_equal(got.cpu().numpy(), want)


def test_cluster_unit_U_and_constraint():
    g = GRAPHS["weighted"]()
    gn = I.to_numpy(g)
    got, rd = S.sclap_cluster(dev(I.random_graph(500, 2000, seed=1)), 1, 3, 4, 1)
    assert rd == 1 and np.array_equal(got.cpu().numpy(), np.arange(500))
    cp = (np.arange(gn["vwgt"].size) * 7919 % 3).astype(np.int32)
    U = int(gn["vwgt"].sum()) // 30
    want, _ = oracle.cluster(gn, U, 4, 4, 5, constraint_part=cp)
    got, _ = S.sclap_cluster(dev(g), U, 4, 4, 5, torch.from_numpy(cp).cuda())
    assert np.array_equal(got.cpu().numpy(), want)


def test_cluster_isolated_packing_with_constraint():
    g = GRAPHS["sparse"]()
    gn = I.to_numpy(g)
    gn["vwgt"] = (np.arange(gn["vwgt"].size) % 5 + 1).astype(np.int32)
    g = {k: torch.from_numpy(v) for k, v in gn.items()}
    cp = (np.arange(gn["vwgt"].size) * 40503 % 4).astype(np.int32)
    for U in (7, 60, 1000):
        want, _ = oracle.cluster(gn, U, 3, 4, 9, constraint_part=cp)
        got, _ = S.sclap_cluster(dev(g), U, 3, 4, 9, torch.from_numpy(cp).cuda())
        assert np.array_equal(got.cpu().numpy(), want), U
        want, _ = oracle.cluster(gn, U, 3, 4, 9)
        got, _ = S.sclap_cluster(dev(g), U, 3, 4, 9)
        assert np.array_equal(got.cpu().numpy(), want), U


@pytest.mark.parametrize("name", ["chunglu2k", "weighted", "rmat14", "star5k", "stars"])
@pytest.mark.parametrize("k", [2, 16, 64, 100])
def test_refine_matches_oracle(name, k):
    g = GRAPHS[name]()
    gn = I.to_numpy(g)
    n = gn["vwgt"].size
    p0 = (np.arange(n, dtype=np.int64) * 2654435761 % k).astype(np.int32)
    want, cut_w, bw_w, rd_w = oracle.refine(gn, k, 0.03, 6, 4, 21, p0)
    got, cut_g, bw_g, rd_g = S.sclap_refine(dev(g), k, 0.03, 6, 4, 21, torch.from_numpy(p0).cuda())
    assert rd_g == rd_w
    assert np.array_equal(got.cpu().numpy(), want)
    assert cut_g == cut_w and np.array_equal(bw_g.numpy(), bw_w)


def test_refine_overloaded_start_matches_oracle():
    g = GRAPHS["weighted"]()
    gn = I.to_numpy(g)
    n = gn["vwgt"].size
    p0 = np.zeros(n, np.int32)
    p0[: n // 5] = 1
    p0[n // 5: n // 4] = 2
    for k in (4, 80):
        want, cut_w, bw_w, rd_w = oracle.refine(gn, k, 0.03, 8, 4, 3, p0)
        got, cut_g, bw_g, rd_g = S.sclap_refine(dev(g), k, 0.03, 8, 4, 3,
                                                torch.from_numpy(p0).cuda())
        assert np.array_equal(got.cpu().numpy(), want), k
        assert cut_g == cut_w and rd_g == rd_w


@pytest.mark.parametrize("k,eps", [(2, 0.03), (5, 0.0), (5, 0.2)])
def test_refine_long_segments_match_oracle(k, eps):
    # tens of thousands of proposals per target block and sub-round: the
    # select runs over tiles spread across the grid
    g = I.random_graph(120000, 600000, seed=13, max_w=5, max_c=7)
    gn = I.to_numpy(g)
    n = gn["vwgt"].size
    p0 = (np.arange(n, dtype=np.int64) * 2654435761 % k).astype(np.int32)
    for Sr in (1, 4):
        want, cut_w, bw_w, rd_w = oracle.refine(gn, k, eps, 5, Sr, 8, p0)
        got, cut_g, bw_g, rd_g = S.sclap_refine(dev(g), k, eps, 5, Sr, 8,
                                                torch.from_numpy(p0).cuda())
        assert rd_g == rd_w, Sr
        assert np.array_equal(got.cpu().numpy(), want), Sr
        assert cut_g == cut_w and np.array_equal(bw_g.numpy(), bw_w)


@pytest.mark.parametrize("leaves,U", [(20000, 500), (30000, 29000), (30000, 40000),
                                      (70000, 500)])
def test_cluster_long_segments_match_oracle(leaves, U):
    # every leaf proposes the hub's label in the same sub-round: one contested
    # segment per sub-round, above the shared-memory bound, selected by the
    # whole grid
    g = star(leaves, w=3)
    gn = I.to_numpy(g)
    gn["vwgt"] = (np.arange(leaves + 1) % 4 + 1).astype(np.int32)
    g = {k: torch.from_numpy(v) for k, v in gn.items()}
    for Sr in (1, 2):
        want, rd_w = oracle.cluster(gn, U, 4, Sr, 5)
        got, rd_g = S.sclap_cluster(dev(g), U, 4, Sr, 5)
        assert rd_g == rd_w
        assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_contract_matches_oracle(name):
    g = GRAPHS[name]()
    gn = I.to_numpy(g)
    cV = int(gn["vwgt"].sum())
    lab, _ = oracle.cluster(gn, max(int(gn["vwgt"].max()), cV // 50), 3, 4, 2)
    want, f2c_w = oracle.contract(gn, lab)
    got, f2c_g = S.contract_graph(dev(g), torch.from_numpy(lab).cuda())
    assert np.array_equal(f2c_g.cpu().numpy(), f2c_w)
    for key in ("xadj", "adjncy", "adjwgt", "vwgt"):
        assert np.array_equal(got[key].cpu().numpy(), want[key]), key


def test_contract_identity_and_single_cluster():
    g = GRAPHS["weighted"]()
    gn = I.to_numpy(g)
    n = gn["vwgt"].size
    for lab in (np.arange(n, dtype=np.int32), np.full(n, 17, np.int32)):
        want, f2c_w = oracle.contract(gn, lab)
        got, f2c_g = S.contract_graph(dev(g), torch.from_numpy(lab).cuda())
        assert np.array_equal(f2c_g.cpu().numpy(), f2c_w)
        for key in ("xadj", "adjncy", "adjwgt", "vwgt"):
            assert np.array_equal(got[key].cpu().numpy(), want[key]), key


def test_project_matches_oracle():
    f2c = (np.arange(10007, dtype=np.int64) * 31 % 977).astype(np.int32)
    cp = (np.arange(977) % 7).astype(np.int32)
    got = S.project_partition(torch.from_numpy(f2c).cuda(), torch.from_numpy(cp).cuda())
    assert np.array_equal(got.cpu().numpy(), oracle.project(f2c, cp))


@pytest.mark.parametrize("name", ["chunglu2k", "weighted"])
def test_initial_partition_matches_oracle(name):
    g = GRAPHS[name]()
    gn = I.to_numpy(g)
    k = 8
    B = oracle.lmax(int(gn["vwgt"].sum()), k, 0.03)
    want, cw, mw, bw = oracle.initial_partition(gn, k, B, 8, 6, 4, 99)
    got, cg, mg, bg = S.sclap_initial_partition(dev(g), k, B, 8, 6, 4, 99)
    assert bg == bw
    assert np.array_equal(cg.numpy(), cw) and np.array_equal(mg.numpy(), mw)
    assert np.array_equal(got.cpu().numpy(), want)


def test_multilevel_config1_matches_oracle():
    # Chung-Lu n = 16,384, ~131k edges, exponent 2.1, mean degree 16; k = 4,
    # eps = 0.03, U = max(max c, c(V)/(10k)), 10 rounds per level, n_stop 2000.
    g = I.chung_lu(16384, 2.1, 16.0, seed=1)
    params = oracle.default_params(4, 0.03, seed=1, cluster_rounds=10, refine_rounds=10,
                                   n_stop=2000)
    want, ws = oracle.multilevel(I.to_numpy(g), params)
    got, gs = S.partition_multilevel(dev(g), params)
    assert gs == ws
    assert np.array_equal(got.cpu().numpy(), want)
    assert gs["maxbw"] <= gs["lmax"]


def test_multilevel_host_buffers_match_device():
    g = I.chung_lu(8192, 2.1, 12.0, seed=4)
    params = oracle.default_params(8, 0.03, seed=4, n_stop=500)
    gh = {k: v.pin_memory() for k, v in g.items()}
    out_h = torch.empty(8192, dtype=torch.int32).pin_memory()
    got_h, sh = S.partition_multilevel(gh, params, part_out=out_h)
    got_d, sd = S.partition_multilevel(dev(g), params)
    want, ws = oracle.multilevel(I.to_numpy(g), params)
    assert sh == sd == ws
    assert np.array_equal(got_h.numpy(), want) and np.array_equal(got_d.cpu().numpy(), want)


def test_multilevel_weighted_matches_oracle():
    g = I.random_graph(20000, 90000, seed=12, max_w=50, max_c=20)
    params = oracle.default_params(16, 0.05, seed=3, n_stop=1000)
    want, ws = oracle.multilevel(I.to_numpy(g), params)
    got, gs = S.partition_multilevel(dev(g), params)
    assert gs == ws
    assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("k,s,bridges", [(4, 50, 1), (16, 30, 1), (3, 100, 5)])
def test_multilevel_planted_partition_matches_oracle(k, s, bridges):
    # rings of cliques: with U = s the oracle recovers the cliques (cut k * bridges)
    g, clique = I.ring_of_cliques(k, s, bridges, seed=k)
    params = oracle.default_params(k, 0.03, seed=2, n_stop=50, U=s)
    want, ws = oracle.multilevel(I.to_numpy(g), params)
    got, gs = S.partition_multilevel(dev(g), params)
    assert gs == ws and np.array_equal(got.cpu().numpy(), want)
    assert gs["cut"] == k * bridges


def test_repeatable_runs_are_identical():
    g = dev(I.rmat(15, 16, seed=8))
    params = oracle.default_params(16, 0.03, seed=5, n_stop=2000)
    a, sa = S.partition_multilevel(g, params)
    b, sb = S.partition_multilevel(g, params)
    assert sa == sb and torch.equal(a, b)


def test_edge_cases():
    empty = {"xadj": torch.zeros(1, dtype=torch.int64), "adjncy": torch.zeros(0, dtype=torch.int32),
             "adjwgt": torch.zeros(0, dtype=torch.int32), "vwgt": torch.zeros(0, dtype=torch.int32)}
    lab, rd = S.sclap_cluster(dev(empty), 1, 3, 4, 1)
    assert lab.numel() == 0 and rd == 0
    # isolated nodes only
    iso = {"xadj": torch.zeros(11, dtype=torch.int64), "adjncy": torch.zeros(0, dtype=torch.int32),
           "adjwgt": torch.zeros(0, dtype=torch.int32), "vwgt": torch.ones(10, dtype=torch.int32)}
    lab, rd = S.sclap_cluster(dev(iso), 3, 3, 4, 1)
    # packed in id order into groups of weight <= U = 3
    assert lab.cpu().tolist() == [0, 0, 0, 3, 3, 3, 6, 6, 6, 9] and rd == 1
    cg, f2c = S.contract_graph(dev(iso), lab)
    assert cg["xadj"].numel() == 5 and cg["adjncy"].numel() == 0
    assert cg["vwgt"].cpu().tolist() == [3, 3, 3, 1]
    # k = 1 refinement never moves
    g = dev(GRAPHS["weighted"]())
    p, cut, bw, rd = S.sclap_refine(g, 1, 0.03, 4, 4, 1, torch.zeros(3000, dtype=torch.int32,
                                                                      device="cuda"))
    assert cut == 0 and rd == 1 and int(p.abs().sum()) == 0


def test_errors_are_reported():
    g = dev(GRAPHS["weighted"]())
    with pytest.raises(S.SclapError) as e:
        S.sclap_cluster(g, 1, 3, 4, 1)             # U < max c(v)
    assert e.value.code == S.EINVAL
    bad = {k: v.clone() for k, v in g.items()}
    bad["adjwgt"][0] += 1                          # asymmetric
    with pytest.raises(S.SclapError) as e:
        S.sclap_cluster(bad, 10**6, 3, 4, 1)
    assert e.value.code == S.EGRAPH
    # the cut validates the graph before it reads part[] at the neighbour ids
    zeros = torch.zeros(3000, dtype=torch.int32, device="cuda")
    oob = {k: v.clone() for k, v in g.items()}
    oob["adjncy"][0] = 3000                        # neighbour id past n
    for graph in (bad, oob):
        with pytest.raises(S.SclapError) as e:
            S.sclap_cut(graph, zeros, 4)
        assert e.value.code == S.EGRAPH
    p = torch.full((3000,), 5, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SclapError) as e:
        S.sclap_refine(g, 4, 0.03, 3, 4, 1, p)     # block id out of range
    assert e.value.code == S.EINVAL
    big = {k: v.clone() for k, v in g.items()}
    big["vwgt"][:] = 2**30                          # c(V) overflows int32
    with pytest.raises(S.SclapError) as e:
        S.sclap_cluster(big, 2**31 - 1, 3, 4, 1)
    assert e.value.code == S.EOVERFLOW
    # edge weights: the undirected total decides (coarse edge weights and
    # omega(v, L) never exceed it); the directed sum may pass INT32_MAX
    heavy = I.to_device(I.path_graph(3, [10**9, 10**9]), "cuda")   # 2e9 undirected
    lab, _ = S.sclap_cluster(heavy, 3, 2, 1, 1)
    assert lab.cpu().tolist() == oracle.cluster(I.to_numpy(I.path_graph(3, [10**9, 10**9])),
                                                3, 2, 1, 1)[0].tolist()
    over = I.to_device(I.path_graph(4, [10**9, 10**9, 10**9]), "cuda")  # 3e9 undirected
    with pytest.raises(S.SclapError) as e:
        S.sclap_cluster(over, 4, 2, 1, 1)
    assert e.value.code == S.EOVERFLOW


def test_batched_runs_match_oracle():
    gens = [I.random_graph(n, 4 * n, seed=n, max_w=30, max_c=20) for n in (700, 2500, 6000, 1200)]
    gs = [I.to_numpy(g) for g in gens]
    gd = [dev(g) for g in gens]
    rg = [3, 0, 2, 2, 1, 0, 3, 2, 1, 1, 0, 2]
    seeds = [9 + 7 * r for r in range(len(rg))]
    seeds[5] = 2**64 - 1
    for k in (4, 16):
        want, wc, wm = oracle.refine_batched(gs, k, 0.03, 6, 4, seeds, rg)
        got, gc, gm = S.sclap_refine_batched(gd, k, 0.03, 6, 4, seeds, rg)
        assert np.array_equal(gc.numpy(), wc) and np.array_equal(gm.numpy(), wm)
        for r in range(len(rg)):
            assert np.array_equal(got[r].cpu().numpy(), want[r]), (k, r)
    # a run alone (batch of one) on the GPU equals the same run in the batch
    for r in (0, 5, 11):
        alone, ca, ma = S.sclap_refine_batched([gd[rg[r]]], 16, 0.03, 6, 4, [seeds[r]], [0])
        assert np.array_equal(alone[0].cpu().numpy(), want[r]) and int(ca[0]) == int(wc[r])


def test_population_batched_runs_match_oracle():
    # the coarse-graph population generator (lognormal edge weights up to
    # 1000, node weights up to 500), 8 graphs, 32 runs: graph (s - 1) mod 8
    gens = I.population(8, 2000, 12000, seed=4)
    gs = [I.to_numpy(g) for g in gens]
    gd = [dev(g) for g in gens]
    rg = [s % 8 for s in range(32)]
    seeds = list(range(1, 33))
    want, wc, wm = oracle.refine_batched(gs, 16, 0.03, 6, 4, seeds, rg)
    got, gc, gm = S.sclap_refine_batched(gd, 16, 0.03, 6, 4, seeds, rg)
    assert np.array_equal(gc.numpy(), wc) and np.array_equal(gm.numpy(), wm)
    for r in range(len(rg)):
        assert np.array_equal(got[r].cpu().numpy(), want[r]), r


@pytest.mark.parametrize("name", ["chunglu2k", "weighted", "sparse", "rmat14"])
def test_vcycle_matches_oracle(name):
    g = GRAPHS[name]()
    gn = I.to_numpy(g)
    k = 8
    params = oracle.default_params(k, 0.03, 7)
    params.update(n_stop=200)
    p0, _ = oracle.multilevel(gn, params)
    vparams = dict(params, seed=8)
    want, ws = oracle.vcycle(gn, vparams, p0)
    got, st = S.sclap_vcycle(dev(g), vparams, torch.from_numpy(p0).cuda())
    assert st == ws
    assert np.array_equal(got.cpu().numpy(), want)
    # no refinement anywhere: the cycle returns its input
    still, st0 = S.sclap_vcycle(dev(g), dict(vparams, refine_rounds=0, init_rounds=0),
                                torch.from_numpy(p0).cuda())
    assert np.array_equal(still.cpu().numpy(), p0) and st0["init_best"] == -1



def test_rounds_identical_in_every_launch_mode():
    """The rounds of a call run one at a time, enqueued ahead with a device
    stop flag, or from one captured CUDA graph; all must end after the same
    round with the same result."""
    import paper_1404_4797_gb300 as S
    g = I.rmat(13, 16, seed=4)
    gd = I.to_device(g, "cuda")
    n = g["vwgt"].numel()
    p0 = I.rand_below(9, 7, torch.arange(n), 8).to(torch.int32).cuda()
    prm = S.default_params(8, 0.03, seed=3, n_stop=300)
    out = {}
    old = S.set_launch_mode(-1)
    try:
        for mode in (0, 1, 2, -1):
            S.set_launch_mode(mode)
            lab, rd = S.sclap_cluster(gd, 40, 8, 4, 11)
            part, cut, bw, rdr = S.sclap_refine(gd, 8, 0.03, 40, 4, 5, p0)
            mp, st = S.partition_multilevel(gd, prm)
            out[mode] = (lab.cpu().numpy(), rd, part.cpu().numpy(), cut, rdr, mp.cpu().numpy(),
                         st["cut"], st["refine_rounds_done"], st["cluster_rounds_done"])
    finally:
        S.set_launch_mode(old)
    for mode in (1, 2, -1):
        for x, y in zip(out[0], out[mode]):
            if isinstance(x, np.ndarray):
                assert np.array_equal(x, y)
            else:
                assert x == y
    # the refinement converged after 18 of its 40 rounds (the oracle's count):
    # the stop rule ended it
    gn = I.to_numpy(g)
    assert out[2][4] == oracle.refine(gn, 8, 0.03, 40, 4, 5, p0.cpu().numpy())[3] < 40


@pytest.mark.parametrize("S_", [1, 3, 4])
def test_degree_ordered_cluster_matches_oracle(S_):
    """Degree-ordered sub-rounds (Sec. III.A's increasing-degree traversal): a
    per-round sort on the GPU against the oracle's order, bit for bit."""
    for g in (I.chung_lu(4096, 2.1, 8.0, seed=3), I.random_graph(5000, 20000, seed=5, max_w=20,
                                                                  max_c=9), I.rmat(13, 16, seed=2)):
        gn = I.to_numpy(g)
        cV = int(gn["vwgt"].sum())
        U = max(int(gn["vwgt"].max()), cV // 40)
        want, wr = oracle.cluster(gn, U, 6, S_, 7, degree_ordered=True)
        got, gr = S.sclap_cluster(dev(g), U, 6, S_, 7, degree_ordered=True)
        assert gr == wr and np.array_equal(got.cpu().numpy(), want)


def test_multilevel_and_vcycle_degree_ordered_match_oracle():
    g = I.chung_lu(8192, 2.1, 12.0, seed=9)
    gn = I.to_numpy(g)
    prm = S.default_params(8, 0.03, seed=5, n_stop=400, degree_order=1)
    got, st = S.partition_multilevel(dev(g), prm)
    want, ws = oracle.multilevel(gn, dict(prm))
    assert st == ws and np.array_equal(got.cpu().numpy(), want)
    got2, st2 = S.sclap_vcycle(dev(g), dict(prm, seed=6), got)
    want2, ws2 = oracle.vcycle(gn, dict(prm, seed=6), want)
    assert st2 == ws2 and np.array_equal(got2.cpu().numpy(), want2)


def test_rgg_multilevel_matches_oracle():
    g = I.rgg(14, seed=4)
    gn = I.to_numpy(g)
    prm = S.default_params(16, 0.03, seed=2, n_stop=500)
    got, st = S.partition_multilevel(dev(g), prm)
    want, ws = oracle.multilevel(gn, dict(prm))
    assert st == ws and np.array_equal(got.cpu().numpy(), want)


def _hub_graph():
    # hubs whose rows take each long-row path of the hash modes: one CTA table
    # (3,000), the thread-block cluster (9,000) and the pieces merged in
    # global tables (40,000 and 80,000), over a weighted random graph
    n = 100_000
    base = I.random_graph(n, 300_000, seed=21, max_w=7, max_c=4)
    src = torch.repeat_interleave(torch.arange(n), base["xadj"][1:] - base["xadj"][:-1])
    dst = base["adjncy"].to(torch.int64)
    up = src < dst
    us, vs = [src[up]], [dst[up]]
    for h, cnt in ((11, 3000), (22, 9000), (33, 40000), (44, 80000)):
        leaves = (torch.arange(cnt) * 7919 + 101 + h) % n
        leaves = leaves[leaves != h]
        us.append(torch.full((leaves.numel(),), h, dtype=torch.int64))
        vs.append(leaves)
    u, v = torch.cat(us), torch.cat(vs)
    w = I.rand_below(9, 3, u * n + v, 6) + 1
    c = I.rand_below(9, 4, torch.arange(n), 3) + 1
    return I.csr_from_edges(n, u, v, w, c.to(torch.int32))


def test_long_rows_of_every_class_match_oracle():
    g = _hub_graph()
    gn = I.to_numpy(g)
    deg = np.diff(gn["xadj"])
    assert deg.max() > 65536 and ((deg > 16384) & (deg <= 65536)).any()
    cV = int(gn["vwgt"].sum())
    U = max(int(gn["vwgt"].max()), cV // 400)
    want, rd_w = oracle.cluster(gn, U, 3, 4, 7)
    got, rd_g = S.sclap_cluster(dev(g), U, 3, 4, 7)
    assert rd_g == rd_w
    assert np.array_equal(got.cpu().numpy(), want)
    k = 100  # above the dense bound: the hash refinement path
    p0 = I.rand_below(3, 8, torch.arange(gn["vwgt"].size), k).to(torch.int32)
    want_p, cut_w, bw_w, rd_w = oracle.refine(gn, k, 0.03, 4, 4, 7, p0.numpy())
    got_p, cut_g, bw_g, rd_g = S.sclap_refine(dev(g), k, 0.03, 4, 4, 7, p0.cuda())
    assert rd_g == rd_w
    assert np.array_equal(got_p.cpu().numpy(), want_p)
    assert cut_g == cut_w and np.array_equal(bw_g.numpy(), bw_w)
