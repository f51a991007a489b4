"""Pins for the CPU oracle (no GPU): published hash vectors, hand-derived worked
examples, closed forms, invariants and brute force on tiny graphs.

Each worked example states the rule of the paper (or of the deterministic
reading of it) that fixes the expected value:
  Sec. II.A  L_max, cut, quotient graph
  Sec. III.A size-constrained label propagation, overloaded-block rule
  Sec. IV.C  contraction map q / C and projection
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1404_4797_gb300 import inputs as I
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def mk(n, edge_list, vw=None):
    u = torch.tensor([e[0] for e in edge_list], dtype=torch.int64)
    v = torch.tensor([e[1] for e in edge_list], dtype=torch.int64)
    w = torch.tensor([e[2] if len(e) > 2 else 1 for e in edge_list], dtype=torch.int64)
    c = None if vw is None else torch.tensor(vw, dtype=torch.int32)
    return I.to_numpy(I.csr_from_edges(n, u, v, w, c))


# ---------------------------------------------------------------- hashing

def test_mix64_matches_published_splitmix64_sequence():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert rows
    for row in rows:
        state = int(row[0])
        for want in row[1:]:
            state = (state + 0x9E3779B97F4A7C15) & brute.M64
            assert oracle.mix64(state) == int(want, 16)
            assert brute.mix64(state) == int(want, 16)


def test_colour_and_tie_follow_their_definitions():
    for seed in (0, 1, 0xDEADBEEF12345678):
        for v in (0, 1, 17, 2**31 - 1):
            for S in (1, 2, 4, 7):
                for rnd in (0, 3):
                    assert oracle.colour(seed, rnd, v, S) == brute.colour(seed, rnd, v, S)
            for rnd in (0, 5):
                for L in (0, 3, 2**30):
                    assert oracle.tie(seed, rnd, v, L) == brute.tie(seed, rnd, v, L)


def test_generator_hash_equals_splitmix64():
    z = torch.tensor([0, 1, 2**40 + 7, -1], dtype=torch.int64)
    got = I.hash64(z).tolist()
    want = [brute.mix64(x & brute.M64) for x in [0, 1, 2**40 + 7, -1]]
    assert [g & brute.M64 for g in got] == want


# ---------------------------------------------------------------- Sec. II.A

def test_lmax_hand_values():
    # (1+eps) * ceil(c(V)/k), rounded down
    assert oracle.lmax(100, 3, 0.03) == 35          # ceil(100/3)=34, 35.02
    assert oracle.lmax(16384, 4, 0.03) == 4218      # 4096 * 1.03 = 4218.88
    assert oracle.lmax(10, 1, 0.0) == 10
    assert oracle.lmax(7, 2, 0.0) == 4               # ceil(3.5) = 4
    assert oracle.lmax(5, 3, 0.0) == 2


def test_cut_and_block_weights_hand_graph():
    g = mk(4, [(0, 1, 2), (1, 2, 3), (2, 3, 4), (0, 3, 5)], vw=[1, 2, 3, 4])
    part = np.array([0, 0, 1, 1], np.int32)
    assert oracle.cut(g, part) == 3 + 5
    assert list(oracle.block_weights(g, part, 2)) == [3, 7]


def test_validate_rejects_malformed_graphs():
    g = mk(3, [(0, 1), (1, 2)])
    assert oracle.validate(g) == oracle.OK
    bad = {k: v.copy() for k, v in g.items()}
    bad["adjwgt"][0] = 2                      # asymmetric weight
    assert oracle.validate(bad) == oracle.EGRAPH
    bad = {k: v.copy() for k, v in g.items()}
    bad["adjncy"][0] = 0                      # self loop (row 0 -> 0)
    assert oracle.validate(bad) == oracle.EGRAPH
    bad = {k: v.copy() for k, v in g.items()}
    bad["adjwgt"][:] = 0                      # omega must be > 0
    assert oracle.validate(bad) == oracle.EGRAPH
    bad = {k: v.copy() for k, v in g.items()}
    bad["vwgt"][1] = -1                       # c must be >= 0
    assert oracle.validate(bad) == oracle.EGRAPH
    bad = {k: v.copy() for k, v in g.items()}
    bad["adjncy"][1] = 7                      # id out of range
    assert oracle.validate(bad) == oracle.EGRAPH


# ---------------------------------------------------------------- Sec. III.A clustering

def test_U_equal_one_keeps_singletons():
    # Sec. II.A: with U = 1 on unit weights the only feasible clustering is
    # every node on its own.
    g = I.to_numpy(I.chung_lu(512, 2.1, 8.0, seed=3))
    lab, rd, mv = oracle.cluster(g, 1, 5, 4, 99, return_moves=True)
    assert np.array_equal(lab, np.arange(512))
    assert rd == 1 and list(mv) == [0]


def test_two_node_path_swaps_forever_with_one_subround():
    # R1 with S = 1: both nodes propose each other's label against the same
    # state, both are admitted (U = 2), so the labels swap every round.
    g = mk(2, [(0, 1)])
    lab, rd, mv = oracle.cluster(g, 2, 3, 1, 5, return_moves=True)
    assert list(lab) == [1, 0] and rd == 3 and list(mv) == [2, 2, 2]
    lab, rd, mv = oracle.cluster(g, 2, 4, 1, 5, return_moves=True)
    assert list(lab) == [0, 1] and list(mv) == [2, 2, 2, 2]


def test_star_capacity_admits_lowest_ids_first():
    # Star: centre 0, leaves 1..4, unit weights, U = 3, S = 1, one round.
    # Every leaf proposes label 0 (gain 1); cap(0) = U - W(0) = 2, so with
    # equal gains ids 1 and 2 are admitted (inclusive prefixes 1, 2 <= 2) and
    # 3, 4 are rejected.  The centre proposes the leaf label with the smallest
    # tie hash (all leaves tie on omega = 1); it is that label's only proposer.
    g = mk(5, [(0, 1), (0, 2), (0, 3), (0, 4)])
    seed = 12345
    lab, rd = oracle.cluster(g, 3, 1, 1, seed)
    best = min(range(1, 5), key=lambda L: (brute.tie(seed, 0, 0, L), L))
    assert lab[1] == 0 and lab[2] == 0 and lab[3] == 3 and lab[4] == 4
    assert lab[0] == best


def test_target_arbitration_prefers_higher_gain():
    # Node 0 is joined to 1, 2, 3 with weights 1, 5, 3 (no other edges); U = 2.
    # Leaves propose label 0 with gains 1, 5, 3; cap(0) = 1 admits only the
    # highest gain (node 2).  Node 0 proposes label 2 (omega 5), cap(2) = 1,
    # admitted.  Applied together: 0 and 2 swap labels.
    g = mk(4, [(0, 1, 1), (0, 2, 5), (0, 3, 3)])
    lab, rd = oracle.cluster(g, 2, 1, 1, 7)
    assert list(lab) == [2, 1, 0, 3]


def test_cluster_weights_never_exceed_U_after_any_round():
    g = I.to_numpy(I.random_graph(300, 1500, seed=11, max_w=9, max_c=5))
    U = 17
    for r in range(1, 7):
        lab, rd = oracle.cluster(g, U, r, 3, 2024)
        W = np.bincount(lab, weights=g["vwgt"], minlength=300)
        assert W.max() <= U
        if rd < r:
            break


def test_cluster_converged_state_has_no_admissible_improving_move():
    g = I.to_numpy(I.random_graph(60, 200, seed=5, max_w=4, max_c=3))
    U = 9
    lab, rd = oracle.cluster(g, U, 200, 4, 77)
    assert rd < 200  # converged
    assert brute.improving_moves(g, list(lab), 60, U, overload_rule=False) == []


def test_unconstrained_single_subround_is_plain_synchronous_lp():
    # U = infinity, S = 1 reduces SCLaP to synchronous label propagation
    # (Raghavan et al.), recomputed here by brute force round by round.
    g = I.to_numpy(I.random_graph(40, 90, seed=8, max_w=5))
    seed = 31
    lab = list(range(40))
    for r in range(1, 6):
        lab = brute.sync_plain_lp_step(g, lab, seed, r - 1)
        got, _ = oracle.cluster(g, 10**9, r, 1, seed)
        assert list(got) == lab


def test_isolated_nodes_are_packed_up_to_U():
    # R6: nodes without neighbours, in id order, join group floor(P(v) / U')
    # with U' = U - cmax + 1; each group is labelled by its smallest id.
    # Unit weights, U = 2: U' = 2, P = 0,1,2,3,4 -> groups {0,1} {2,3} {4}.
    iso5 = {"xadj": np.zeros(6, np.int64), "adjncy": np.zeros(0, np.int32),
            "adjwgt": np.zeros(0, np.int32), "vwgt": np.ones(5, np.int32)}
    lab, rd = oracle.cluster(iso5, 2, 3, 4, 1)
    assert list(lab) == [0, 0, 2, 2, 4] and rd == 1
    # weights 2,1,2,1 with U = 3: cmax = 2, U' = 2, P = 0,2,3,5 -> groups 0,1,1,2
    iso4 = {"xadj": np.zeros(5, np.int64), "adjncy": np.zeros(0, np.int32),
            "adjwgt": np.zeros(0, np.int32), "vwgt": np.array([2, 1, 2, 1], np.int32)}
    lab, _ = oracle.cluster(iso4, 3, 3, 4, 1)
    assert list(lab) == [0, 1, 1, 3]
    # mixed with an edge (1-3): isolated 0, 2, 4 form one group when U = 3;
    # 1 and 3 keep swapping labels (S = 1) and are not touched by the packing
    g = mk(5, [(1, 3)])
    lab, _ = oracle.cluster(g, 3, 2, 1, 1)
    assert lab[0] == lab[2] == lab[4] == 0 and {lab[1], lab[3]} == {1, 3}
    # with a constraint partition the packing is per block
    cp = np.array([0, 1, 1, 0, 1], np.int32)
    lab, _ = oracle.cluster(iso5, 5, 2, 1, 1, constraint_part=cp)
    assert list(lab) == [0, 1, 1, 0, 1]


def test_vcycle_constraint_keeps_clusters_inside_blocks():
    g = I.to_numpy(I.random_graph(200, 800, seed=9))
    cp = (np.arange(200) * 7919 % 3).astype(np.int32)
    lab, _ = oracle.cluster(g, 30, 5, 4, 4, constraint_part=cp)
    for L in np.unique(lab):
        assert len(np.unique(cp[lab == L])) == 1


# ---------------------------------------------------------------- Sec. III.A refinement

def test_refine_k1_never_moves():
    g = I.to_numpy(I.random_graph(100, 300, seed=2))
    p, ct, bw, rd = oracle.refine(g, 1, 0.03, 5, 4, 3, np.zeros(100, np.int32))
    assert (p == 0).all() and ct == 0 and rd == 1 and list(bw) == [100]


def test_overloaded_block_moves_even_without_gain():
    # Path 0-1-2-3, unit weights, k = 2, eps = 0: L_max = 2.  Start [0,0,0,1]:
    # block 0 (weight 3) is overloaded.  Node 2 sees block 1 (eligible: 1+1 <= 2)
    # with gain 1 - 1 = 0 and moves because its block is overloaded; node 3
    # cannot enter block 0.  Round 2 has no eligible move.
    g = mk(4, [(0, 1), (1, 2), (2, 3)])
    p, rd, mv = oracle.refine_bound(g, 2, 2, 5, 1, 1, np.array([0, 0, 0, 1]), return_moves=True)
    assert list(p) == [0, 0, 1, 1] and rd == 2 and list(mv) == [1, 0]


@pytest.mark.parametrize("w14,expect", [(3, [1, 0, 0, 1, 2]), (5, [0, 2, 0, 1, 2])])
def test_overloaded_departures_stop_at_the_excess(w14, expect):
    # k = 3, c(V) = 5, eps = 0: L_max = 2.  Block 0 = {0,1,2} has excess 1.
    # Node 0 wants block 1 (gain 2-1 = 1); node 1 wants block 2 (gain w14 - 2).
    # Departures in (gain desc, id asc) order are admitted while the weight
    # departed before them is < 1, so exactly one leaves: node 0 on a gain tie
    # (w14 = 3), node 1 when its gain is larger (w14 = 5).
    g = mk(5, [(0, 3, 2), (1, 4, w14), (0, 1, 1), (1, 2, 1)])
    p, rd = oracle.refine_bound(g, 3, 2, 1, 1, 1, np.array([0, 0, 0, 1, 2]))
    assert list(p) == expect


def test_refine_keeps_feasible_input_feasible_and_reduces_overload():
    g = I.to_numpy(I.random_graph(400, 2000, seed=21, max_w=7, max_c=6))
    k = 5
    B = oracle.lmax(int(g["vwgt"].sum()), k, 0.03)
    # feasible start (round robin by weight) stays feasible after every round
    order = np.argsort(-g["vwgt"], kind="stable")
    p0 = np.zeros(400, np.int32)
    bw = np.zeros(k, np.int64)
    for v in order:
        b = int(np.argmin(bw))
        p0[v] = b
        bw[b] += g["vwgt"][v]
    assert bw.max() <= B
    for r in range(1, 5):
        p, _ = oracle.refine_bound(g, k, B, r, 4, 5, p0)
        assert max(brute.block_weights(g, p, k)) <= B
    # overloaded start: total overload never grows from round to round
    p0 = (np.arange(400) % 2).astype(np.int32)
    prev = None
    for r in range(0, 6):
        p, _ = oracle.refine_bound(g, k, B, r, 4, 5, p0)
        over = sum(max(0, x - B) for x in brute.block_weights(g, p, k))
        if prev is not None:
            assert over <= prev
        prev = over


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_refine_brute_force_tiny(seed):
    # n <= 9: enumerate all k^n partitions.  The converged oracle result is
    # feasible, no worse than... at least the optimum, and a local optimum of
    # the move rule (no eligible improving single move remains).
    n, k = 9, 3
    g = I.to_numpy(I.random_graph(n, 16, seed=seed, max_w=6, max_c=3))
    B = oracle.lmax(int(g["vwgt"].sum()), k, 0.2)
    opt = brute.optimal_cut(g, k, B)
    p0 = np.array([v % k for v in range(n)], np.int32)
    if max(brute.block_weights(g, p0, k)) > B:
        pytest.skip("start not feasible for this seed")
    p, ct, bw, rd = oracle.refine(g, k, 0.2, 100, 2, seed, p0)
    assert rd < 100
    assert ct == brute.cut(g, p) and list(bw) == brute.block_weights(g, p, k)
    assert max(bw) <= B
    assert opt is not None and ct >= opt
    assert brute.improving_moves(g, list(p), k, B, overload_rule=True) == []


def test_refine_without_balance_is_plain_lp_on_blocks():
    # L_max >= c(V): every neighbouring block is eligible, the rule reduces to
    # synchronous plain LP restricted to the k block labels.
    g = I.to_numpy(I.random_graph(30, 70, seed=4, max_w=3))
    p0 = np.array([v % 4 for v in range(30)], np.int32)
    lab = [int(x) for x in p0]
    for r in range(1, 4):
        lab = brute.sync_plain_lp_step(g, lab, 9, r - 1)
        got, _ = oracle.refine_bound(g, 4, 10**9, r, 1, 9, p0)
        assert list(got) == lab


# ---------------------------------------------------------------- Sec. IV.C contraction

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_contraction_equals_dense_closed_form(seed):
    n = 48
    g = I.to_numpy(I.random_graph(n, 150, seed=seed, max_w=9, max_c=7))
    lab, _ = oracle.cluster(g, 25, 3, 2, seed)
    cg, f2c = oracle.contract(g, lab)
    distinct = np.unique(lab)
    assert len(cg["vwgt"]) == len(distinct)                   # n' = #distinct ids
    assert np.array_equal(f2c, np.searchsorted(distinct, lab))  # C = q o label
    P = np.zeros((n, len(distinct)), np.int64)
    P[np.arange(n), f2c] = 1
    A = brute.dense_adjacency(g)
    A2 = P.T @ A @ P
    np.fill_diagonal(A2, 0)
    assert np.array_equal(brute.dense_adjacency(cg), A2)
    assert np.array_equal(cg["vwgt"], P.T @ g["vwgt"].astype(np.int64))
    # canonical layout: neighbours strictly ascending within each row
    for c in range(len(distinct)):
        row = cg["adjncy"][cg["xadj"][c]:cg["xadj"][c + 1]]
        assert (np.diff(row) > 0).all()
    assert oracle.validate(cg) == oracle.OK


def test_contraction_preserves_weight_totals():
    g = I.to_numpy(I.chung_lu(2048, 2.1, 8.0, seed=2))
    lab, _ = oracle.cluster(g, 40, 3, 4, 1)
    cg, f2c = oracle.contract(g, lab)
    assert cg["vwgt"].sum() == g["vwgt"].sum()
    inter = sum(int(g["adjwgt"][i]) for v in range(2048)
                for i in range(g["xadj"][v], g["xadj"][v + 1])
                if f2c[v] != f2c[g["adjncy"][i]])
    assert cg["adjwgt"].sum() == inter


def test_projection_preserves_cut_and_balance():
    # Sec. III: a partition of the coarse graph induces a partition of the fine
    # graph with the same cut and balance.
    g = I.to_numpy(I.random_graph(500, 2500, seed=13, max_w=4, max_c=3))
    lab, _ = oracle.cluster(g, 20, 3, 4, 3)
    cg, f2c = oracle.contract(g, lab)
    k = 4
    pc = (np.arange(len(cg["vwgt"])) * 2654435761 % k).astype(np.int32)
    pf = oracle.project(f2c, pc)
    assert np.array_equal(pf, pc[f2c])
    assert oracle.cut(g, pf) == oracle.cut(cg, pc) == brute.cut(g, pf)
    assert np.array_equal(oracle.block_weights(g, pf, k), oracle.block_weights(cg, pc, k))


# ---------------------------------------------------------------- initial partition + driver

def test_initial_partition_lpt_start_is_balanced():
    # With 0 refinement rounds every individual is the LPT start: placing items
    # heaviest first into the lightest block keeps max - min <= max item.
    g = I.to_numpy(I.random_graph(200, 600, seed=3, max_c=50))
    k = 6
    B = oracle.lmax(int(g["vwgt"].sum()), k, 0.03)
    part, cuts, mx, best = oracle.initial_partition(g, k, B, 4, 0, 4, 77)
    for t in range(4):
        assert cuts[t] >= 0
    bw = brute.block_weights(g, part, k)
    assert max(bw) - min(bw) <= int(g["vwgt"].max())
    assert cuts[best] == brute.cut(g, part) and mx[best] == max(bw)


def test_initial_partition_lpt_hand_example():
    # Path 0-1-2 with weights 5, 3, 3, k = 2, one individual, no refinement:
    # node 0 (heaviest) goes to block 0 (all empty, lowest id wins), then both
    # weight-3 nodes go to the lighter block 1, whatever their shuffled order.
    g = mk(3, [(0, 1), (1, 2)], vw=[5, 3, 3])
    part, cuts, mx, best = oracle.initial_partition(g, 2, 100, 1, 0, 1, 5)
    assert list(part) == [0, 1, 1] and list(cuts) == [1] and list(mx) == [6] and best == 0


def test_initial_partition_picks_the_best_feasible_individual():
    g = I.to_numpy(I.random_graph(150, 600, seed=5, max_c=9, max_w=5))
    k = 4
    B = oracle.lmax(int(g["vwgt"].sum()), k, 0.03)
    part, cuts, mx, best = oracle.initial_partition(g, k, B, 6, 4, 4, 123)
    feas = [t for t in range(6) if mx[t] <= B]
    if feas:
        assert best == min(feas, key=lambda t: (cuts[t], t))
    assert oracle.cut(g, part) == cuts[best]


def test_multilevel_config1_shape_is_deterministic_and_balanced():
    g = I.to_numpy(I.chung_lu(16384, 2.1, 16.0, seed=1))
    p = oracle.default_params(4, cluster_rounds=10, refine_rounds=10, n_stop=2000, seed=1)
    part, st = oracle.multilevel(g, p)
    part2, st2 = oracle.multilevel(g, p)
    assert np.array_equal(part, part2) and st == st2
    assert st["n"][-1] < 2000 or st["levels"] >= 2
    assert st["cut"] == oracle.cut(g, part)
    bw = oracle.block_weights(g, part, 4)
    assert bw.max() == st["maxbw"]
    if st["init_maxbw"] <= st["lmax"]:
        assert bw.max() <= st["lmax"]
    assert st["U"] == max(1, 16384 // 40)


PLANTED = [(2, 40, 1), (4, 50, 1), (8, 40, 2), (6, 64, 3), (16, 30, 1), (3, 100, 5)]


@pytest.mark.parametrize("k,s,bridges", PLANTED)
def test_multilevel_recovers_a_planted_partition(k, s, bridges):
    # A known optimum: k cliques of s nodes in a ring, `bridges` edges between
    # neighbouring cliques.  L_max = floor(1.03 s) < 2s, so a k-way partition
    # either keeps every clique in its own block (cut k * bridges) or splits a
    # clique (cut >= s - 1 > k * bridges).  With a cluster bound that admits a
    # whole clique (U = s) the multilevel scheme of Sec. IV.E finds it.
    g, clique = I.ring_of_cliques(k, s, bridges, seed=k)
    g, clique = I.to_numpy(g), clique.numpy()
    assert s - 1 > k * bridges and oracle.lmax(k * s, k, 0.03) < 2 * s
    planted = oracle.cut(g, clique.astype(np.int32))
    assert planted == k * bridges
    for seed in (1, 2, 3):
        p = oracle.default_params(k, 0.03, seed=seed, n_stop=50, U=s)
        part, st = oracle.multilevel(g, p)
        assert st["cut"] == planted and st["maxbw"] <= st["lmax"]
        blocks = [set(part[clique == c].tolist()) for c in range(k)]
        assert all(len(b) == 1 for b in blocks) and len(set().union(*blocks)) == k


def test_planted_generator_shape():
    g, clique = I.ring_of_cliques(5, 12, 2, seed=9)
    g = I.to_numpy(g)
    assert oracle.validate(g) == oracle.OK
    assert np.bincount(clique.numpy()).tolist() == [12] * 5
    assert int(g["adjwgt"].sum()) // 2 == 5 * 66 + 5 * 2  # clique edges + bridge weight
    deg_in = [sum(1 for e in range(g["xadj"][v], g["xadj"][v + 1])
                  if clique[g["adjncy"][e]] == clique[v]) for v in range(60)]
    assert deg_in == [11] * 60  # every clique complete


# ---------------------------------------------------------------- batched runs

def _lpt_by_hand(g, k, sr):
    # the LPT start of a run with seed sr written out from its definition
    n = len(g["vwgt"])
    order = sorted(range(n), key=lambda v: (-int(g["vwgt"][v]), brute.mix64(sr ^ v) >> 32, v))
    bw = [0] * k
    part = [0] * n
    for v in order:
        b = min(range(k), key=lambda x: (bw[x], x))
        part[v] = b
        bw[b] += int(g["vwgt"][v])
    return part


def test_batched_runs_start_from_their_lpt_placement():
    gs = [I.to_numpy(I.random_graph(40, 90, seed=s, max_c=7, max_w=3)) for s in (1, 2)]
    rg = [0, 1, 1, 0]
    seeds = [77, 78, 2**63 + 5, 77]
    parts, cuts, mx = oracle.refine_batched(gs, 3, 0.1, 0, 2, seeds, rg)
    for r, g in enumerate(rg):
        assert list(parts[r]) == _lpt_by_hand(gs[g], 3, seeds[r])
        assert list(oracle.lpt_start(gs[g], 3, seeds[r])) == list(parts[r])
        assert cuts[r] == brute.cut(gs[g], parts[r])
        assert mx[r] == max(brute.block_weights(gs[g], parts[r], 3))


def test_batched_runs_respect_their_own_bounds_and_report_consistently():
    gs = [I.to_numpy(I.random_graph(n, 4 * n, seed=n, max_c=9, max_w=5)) for n in (60, 200, 500)]
    k = 4
    rg = [2, 0, 1, 2, 1]
    seeds = [5, 6, 7, 8, 9]
    parts, cuts, mx = oracle.refine_batched(gs, k, 0.03, 6, 4, seeds, rg)
    for r, g in enumerate(rg):
        B = oracle.lmax(int(gs[g]["vwgt"].sum()), k, 0.03)
        bw = brute.block_weights(gs[g], parts[r], k)
        assert cuts[r] == brute.cut(gs[g], parts[r]) and mx[r] == max(bw)
        start = _lpt_by_hand(gs[g], k, seeds[r])
        if max(brute.block_weights(gs[g], start, k)) <= B:
            assert max(bw) <= B   # a feasible start stays feasible


def test_a_run_in_a_batch_equals_the_same_run_alone():
    """Sec. II.C / IV.E: the individuals of a population are independent.  A
    run's result must not depend on the other runs of its batch or on its
    position: it equals the batch holding only that run, and that equals the
    run's LPT start refined on its graph alone with its seed (the single-run
    code path)."""
    gs = [I.to_numpy(I.random_graph(n, 5 * n, seed=n + 1, max_c=6, max_w=7))
          for n in (90, 300, 160)]
    k, rounds, S = 4, 8, 3
    rg = [1, 0, 2, 1, 1, 2, 0]
    seeds = [11, 12, 13, 14, 11, 2**64 - 3, 17]
    parts, cuts, mx = oracle.refine_batched(gs, k, 0.03, rounds, S, seeds, rg)
    for r, g in enumerate(rg):
        alone, ca, ma = oracle.refine_batched([gs[g]], k, 0.03, rounds, S, [seeds[r]], [0])
        assert np.array_equal(parts[r], alone[0]) and cuts[r] == ca[0] and mx[r] == ma[0]
        B = oracle.lmax(int(gs[g]["vwgt"].sum()), k, 0.03)
        single, _ = oracle.refine_bound(gs[g], k, B, rounds, S, seeds[r],
                                        oracle.lpt_start(gs[g], k, seeds[r]))
        assert np.array_equal(parts[r], single)
    # runs 1 and 4 share graph and seed: identical results at different positions
    assert np.array_equal(parts[0], parts[4])
    # the runs really moved nodes (the equalities above are not about starts)
    assert any(not np.array_equal(parts[r], oracle.lpt_start(gs[g], k, seeds[r]))
               for r, g in enumerate(rg))


def test_initial_partition_is_the_best_of_batched_runs():
    g = I.to_numpy(I.random_graph(120, 400, seed=6, max_c=5, max_w=4))
    k, P = 4, 5
    B = oracle.lmax(int(g["vwgt"].sum()), k, 0.03)
    part, cuts, mx, best = oracle.initial_partition(g, k, B, P, 4, 4, 21)
    seeds = [brute.mix64(21 ^ ((0xD1B54A32D192ED03 * (t + 1)) & brute.M64)) for t in range(P)]
    parts, bc, bm = oracle.refine_batched([g], k, 0.03, 4, 4, seeds, [0] * P)
    assert list(cuts) == list(bc) and list(mx) == list(bm)
    assert np.array_equal(part, parts[best])


def test_input_generators_web_graph_and_population_shapes():
    # seeded input generators: symmetric CSR, weight ranges, long-range share
    g = I.to_numpy(I.web_graph(1 << 12, 2.0, 16.0, dmax=800.0, long_frac=0.05, seed=2))
    n = g["vwgt"].size
    assert n == 4096 and oracle.validate(g) == oracle.OK
    deg = np.diff(g["xadj"])
    assert deg.max() > 8 * deg.mean()               # power-law hubs
    assert abs(g["adjncy"].size / 2 / (n * 16 / 2) - 1) < 0.1
    pop = [I.to_numpy(x) for x in I.population(3, 2000, 4000, seed=5)]
    for gp in pop:
        assert 2000 <= gp["vwgt"].size <= 4000 and oracle.validate(gp) == oracle.OK
        assert gp["vwgt"].min() >= 1 and gp["vwgt"].max() <= 500
        assert gp["adjwgt"].min() >= 1 and gp["adjwgt"].max() <= 1000


def test_threads_do_not_change_results():
    """The OpenMP build splits each sub-round's propose loop over threads;
    arbitration orders proposals totally, so results equal the one-thread ones."""
    g = I.to_numpy(I.chung_lu(4096, 2.1, 8.0, seed=11))
    n = g["vwgt"].size
    prm = oracle.default_params(8, 0.03, seed=4, n_stop=300)
    p0 = (np.arange(n, dtype=np.int64) * 2654435761 % 8).astype(np.int32)
    old = oracle.get_threads()
    try:
        oracle.set_threads(1)
        want = oracle.multilevel(g, prm)
        want_r = oracle.refine(g, 8, 0.03, 6, 4, 3, p0)
        for t in (2, 5, 8):
            oracle.set_threads(t)
            got = oracle.multilevel(g, prm)
            assert np.array_equal(got[0], want[0]) and got[1] == want[1]
            got_r = oracle.refine(g, 8, 0.03, 6, 4, 3, p0)
            assert np.array_equal(got_r[0], want_r[0]) and got_r[1] == want_r[1]
            assert np.array_equal(got_r[2], want_r[2]) and got_r[3] == want_r[3]
    finally:
        oracle.set_threads(old)
