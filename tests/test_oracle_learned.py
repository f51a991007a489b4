"""Pins of the oracle's learned refinement gate (features, bf16 scorer,
gated rounds, gradient) against hand values, exact arithmetic, finite
differences and the plain refinement it reduces to."""
import numpy as np
import pytest

import oracle
from paper_1404_4797_gb300 import inputs as I


def net_const(b3):
    """bf16 network whose logit is b3 for every input."""
    p = np.zeros(oracle.MLP_NPARAM, np.float32)
    p[1312] = b3
    return to_bf16_bits(p)


def to_bf16_bits(p):
    p = np.asarray(p, np.float32)
    out = np.zeros(p.size, np.uint16)
    for i, v in enumerate(p):
        out[i] = np.float32(oracle.bf16(float(v))).view(np.uint32) >> 16
    return out


def test_bf16_round_to_nearest_even():
    assert oracle.bf16(1.0) == 1.0
    assert oracle.bf16(1.0 + 2**-8) == 1.0                # tie -> even mantissa
    assert oracle.bf16(1.0 + 3 * 2**-8) == 1.0 + 2**-6    # tie -> even (up)
    assert oracle.bf16(1.0 + 2**-8 + 2**-12) == 1.0 + 2**-7  # above the tie
    assert oracle.bf16(-3.0) == -3.0
    assert oracle.bf16(0.1) == pytest.approx(0.10009765625)


def test_log2_feature_exact_at_powers_and_linear_between():
    for e in range(0, 40):
        assert oracle.log2_feature(2**e) == e
    assert oracle.log2_feature(3) == 1.5
    assert oracle.log2_feature(6) == 2.5
    assert oracle.log2_feature(12) == 3.5
    assert oracle.log2_feature(2**20 + 2**19) == 20.5


def path4():
    # 0-1-2-3, weights 1, 2, 3
    return {"xadj": np.array([0, 1, 3, 5, 6]), "adjncy": np.array([1, 0, 2, 1, 3, 2]),
            "adjwgt": np.array([1, 1, 2, 2, 3, 3]), "vwgt": np.ones(4, np.int32)}


def test_features_by_hand():
    g = path4()
    lab = np.array([0, 0, 1, 1], np.int32)
    W = np.array([2, 2], np.int64)
    moved = np.array([0, 1, 0, 0], np.uint8)
    vb = np.array([0, 2, 2, 0], np.int64)   # best external weight seen at the last visit
    vo = np.array([1, 1, 3, 3], np.int64)   # own-block weight seen at the last visit
    x = oracle.features(g, lab, W, 2, moved, vb, vo)
    # node 1: deg 2 -> log2-feature(3) = 1.5; W/Lmax = 1; weighted degree 3:
    # (2 - 1)/3 and 1/3 in bf16; moved; neighbours 0 and 2 did not move
    assert x[1, 0] == 1.5 and x[1, 1] == 1.0
    assert x[1, 2] == oracle.bf16(1.0 / 3.0) and x[1, 5] == oracle.bf16(1.0 / 3.0)
    assert x[1, 3] == 1.0 and x[1, 4] == 0.0
    # node 0: one neighbour (1, which moved), weighted degree 1: gain -1, own share 1
    assert list(x[0]) == [1.0, 1.0, -1.0, 0.0, 1.0, 1.0]
    # node 3: weighted degree 3, gain (0 - 3)/3, own share 1, neighbour 2 did not move
    assert x[3, 2] == -1.0 and x[3, 4] == 0.0 and x[3, 5] == 1.0
    # before any visit the visit features are 0; W / L_max of an overloaded block
    x2 = oracle.features(g, lab, np.array([3, 1], np.int64), 2, None)
    assert x2[0, 1] == 1.5 and x2[2, 1] == 0.5
    assert np.all(x2[:, 2] == 0) and np.all(x2[:, 5] == 0)


def test_visit_features_record_what_the_visit_saw():
    # With one sub-round every node of round 0 is visited against the start
    # state, so the features before round 1 carry, per node, the weight to its
    # start block and to the best eligible other block at the start (brute
    # force here), divided by its weighted degree.
    g = I.to_numpy(I.random_graph(300, 1200, seed=4, max_w=7, max_c=3))
    n, k, eps = 300, 6, 0.03
    p0 = (np.arange(n, dtype=np.int64) * 2654435761 % k).astype(np.int32)
    _, moves, _, tx, _ = oracle.refine_learned(g, k, eps, 2, 1, 13, p0, net_const(8.0), 0.0,
                                               3, trace=True)
    assert len(moves) == 2
    lmax = oracle.lmax(int(g["vwgt"].sum()), k, eps)
    W0 = np.bincount(p0, weights=g["vwgt"], minlength=k).astype(np.int64)
    for v in range(n):
        row = range(g["xadj"][v], g["xadj"][v + 1])
        if len(row) == 0:
            continue
        acc = np.zeros(k, np.int64)
        for i in row:
            acc[p0[g["adjncy"][i]]] += g["adjwgt"][i]
        own = p0[v]
        wd = int(acc.sum())
        elig = [b for b in range(k) if b != own and acc[b] > 0 and W0[b] + g["vwgt"][v] <= lmax]
        wb = max((int(acc[b]) for b in elig), default=0)
        assert tx[1][v, 5] == oracle.bf16(float(np.float32(acc[own]) / np.float32(wd)))
        assert tx[1][v, 2] == oracle.bf16(float(np.float32(wb - acc[own]) / np.float32(wd)))


def test_mlp_forward_exact_small_values():
    rng = np.random.default_rng(3)
    # parameters and inputs small dyadic numbers: every fmaf is exact
    p = rng.integers(-4, 5, oracle.MLP_NPARAM).astype(np.float32) / 8
    X = rng.integers(0, 5, (50, 6)).astype(np.float32) / 4
    net = to_bf16_bits(p)
    z = oracle.mlp_score(X, net)
    W1 = p[0:192].reshape(32, 6).astype(np.float64)
    b1 = p[192:224].astype(np.float64)
    W2 = p[224:1248].reshape(32, 32).astype(np.float64)
    b2 = p[1248:1280].astype(np.float64)
    W3 = p[1280:1312].astype(np.float64)
    b3 = float(p[1312])
    h1 = np.maximum(X.astype(np.float64) @ W1.T + b1, 0)
    assert np.all(h1 * 128 == np.round(h1 * 128))  # exact in bf16 range used
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    want = h2 @ W3 + b3
    # hidden values stay within bf16's 8 significant bits here
    h1b = np.array([[oracle.bf16(float(v)) for v in r] for r in h1])
    assert np.array_equal(h1b, h1)
    h2b = np.array([[oracle.bf16(float(v)) for v in r] for r in h2])
    want = h2b @ W3 + b3
    assert np.array_equal(z.astype(np.float64), want)


def test_mlp_forward_relu_and_bias_by_hand():
    p = np.zeros(oracle.MLP_NPARAM, np.float32)
    p[0] = 1.0        # W1[0][0]
    p[192] = -0.5     # b1[0]
    p[224] = 2.0      # W2[0][0]
    p[1280] = 3.0     # W3[0]
    p[1312] = 0.25    # b3
    net = to_bf16_bits(p)
    X = np.array([[0.25, 9, 9, 9, 9, 9], [1.5, 0, 0, 0, 0, 0]], np.float32)
    z = oracle.mlp_score(X, net)
    assert z[0] == 0.25                       # relu(0.25 - 0.5) = 0
    assert z[1] == 0.25 + 3 * 2 * 1.0         # relu(1.0) * 2 * 3


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    X = rng.random((40, 6)).astype(np.float32)
    y = (rng.random(40) < 0.3).astype(np.uint8)
    p = (rng.standard_normal(oracle.MLP_NPARAM) * 0.4).astype(np.float32)
    loss, g = oracle.mlp_loss_grad(X, y, p)
    assert loss > 0
    for i in [0, 7, 191, 192, 223, 224, 700, 1247, 1248, 1279, 1280, 1311, 1312]:
        h = 1e-2
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(X, y, pp)[0] - oracle.mlp_loss_grad(X, y, pm)[0]) / (
            float(pp[i]) - float(pm[i]))
        assert g[i] == pytest.approx(fd, rel=2e-2, abs=2e-4), i


def test_loss_by_hand_for_constant_logit():
    X = np.zeros((4, 6), np.float32)
    y = np.array([1, 0, 0, 1], np.uint8)
    p = np.zeros(oracle.MLP_NPARAM, np.float32)
    loss, g = oracle.mlp_loss_grad(X, y, p)
    assert loss == pytest.approx(np.log(2))
    assert g[1312] == pytest.approx(0.0)      # mean(sigmoid(0) - y) = 0.5 - 0.5
    y = np.array([1, 1, 1, 1], np.uint8)
    assert oracle.mlp_loss_grad(X, y, p)[1][1312] == pytest.approx(-0.5)


def _exact_net(rng):
    """A network on which bf16 rounding changes nothing: weights in {-1, 0, 1}
    (second layer mostly zero), small integer biases, inputs in {0, 0.5, 1, 2},
    so every parameter and every hidden output is a small dyadic number that
    bf16 represents exactly."""
    p = np.zeros(oracle.MLP_NPARAM, np.float32)
    p[0:192] = rng.integers(-1, 2, 192)
    p[192:224] = rng.integers(-2, 3, 32)
    p[224:1248] = rng.integers(-1, 2, 1024) * (rng.random(1024) < 0.1)
    p[1248:1280] = rng.integers(-1, 2, 32)
    p[1280:1312] = rng.integers(-1, 2, 32) * 0.5
    p[1312] = 0.25
    X = rng.choice(np.array([0.0, 0.5, 1.0, 2.0], np.float32), (30, 6))
    y = (rng.random(30) < 0.4).astype(np.uint8)
    return p, X, y


def test_bf16_training_equals_float_training_where_rounding_is_exact():
    # where nothing rounds, the BF16-in loss and straight-through gradient are
    # the float network's loss and gradient (pinned by finite differences above)
    rng = np.random.default_rng(8)
    p, X, y = _exact_net(rng)
    lb, gb = oracle.mlp_loss_grad(X, y, p, bf16_in=True)
    lf, gf = oracle.mlp_loss_grad(X, y, p)
    assert lb == pytest.approx(lf, rel=1e-12) and lb > 0
    assert np.allclose(gb, gf, rtol=1e-9, atol=1e-12)
    assert np.count_nonzero(gf) > 100


def test_bf16_training_rounds_parameters_and_hidden_outputs():
    X = np.array([[1, 0, 0, 0, 0, 0]], np.float32)
    y = np.array([1], np.uint8)
    # parameter rounding: W3[0] = 1 + 2^-10 is not a bf16 value and rounds to 1
    p = np.zeros(oracle.MLP_NPARAM, np.float32)
    p[0] = 1.0                     # W1[0][0]
    p[224] = 1.0                   # W2[0][0]
    p[1280] = 1.0 + 2.0 ** -10     # W3[0]
    q = p.copy()
    q[1280] = 1.0
    lb, gb = oracle.mlp_loss_grad(X, y, p, bf16_in=True)
    lq, gq = oracle.mlp_loss_grad(X, y, q)
    assert lb == lq and np.array_equal(gb, gq)
    # z = 1 by hand: loss log(1 + e^-1), dL/db3 = sigmoid(1) - 1, dL/dW3[0] = dz * h2 = dz
    dz = 1.0 / (1.0 + np.exp(-1.0)) - 1.0
    assert lb == pytest.approx(np.log1p(np.exp(-1.0)), rel=1e-12)
    assert gb[1312] == pytest.approx(dz, rel=1e-12) and gb[1280] == pytest.approx(dz, rel=1e-12)
    # hidden-output rounding: b1[0] = 2^-9 makes a1 = 1 + 2^-9, which the
    # forward rounds to 1 (a quarter of a bf16 step), so z stays exactly 1
    p2 = np.zeros(oracle.MLP_NPARAM, np.float32)
    p2[0], p2[192], p2[224], p2[1280] = 1.0, 2.0 ** -9, 1.0, 1.0
    l2, g2 = oracle.mlp_loss_grad(X, y, p2, bf16_in=True)
    assert l2 == lb and g2[1280] == gb[1280] and g2[1312] == gb[1312]
    # dL/dW2[0][0] = d2 * h1 = dz * W3[0] * h1 takes the rounded h1 = 1
    assert g2[224] == pytest.approx(dz, rel=1e-12)
    assert oracle.mlp_loss_grad(X, y, p2)[0] != l2   # the float network sees 1 + 2^-9


GRAPHS = {
    "chunglu": lambda: I.to_numpy(I.chung_lu(2048, 2.1, 8.0, seed=3)),
    "weighted": lambda: I.to_numpy(I.random_graph(3000, 12000, seed=5, max_w=20, max_c=9)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_learned_without_net_is_plain_refinement(name):
    g = GRAPHS[name]()
    n = g["vwgt"].size
    p0 = (np.arange(n, dtype=np.int64) * 2654435761 % 8).astype(np.int32)
    want, _, _, rd = oracle.refine(g, 8, 0.03, 6, 4, 21, p0)
    got, moves, visited, _, _ = oracle.refine_learned(g, 8, 0.03, 6, 4, 21, p0, None)
    assert np.array_equal(got, want) and len(moves) == rd
    deg = np.diff(g["xadj"])
    assert visited == rd * int(np.sum(deg > 0))
    # a network that admits everyone gives the same result
    got2, moves2, visited2, _, _ = oracle.refine_learned(g, 8, 0.03, 6, 4, 21, p0,
                                                         net_const(8.0), 0.0, 3)
    assert np.array_equal(got2, want) and visited2 == visited


@pytest.mark.parametrize("name", list(GRAPHS))
def test_gate_that_admits_nobody_visits_full_rounds_only(name):
    g = GRAPHS[name]()
    n = g["vwgt"].size
    k, eps = 8, 0.03
    p0 = (np.arange(n, dtype=np.int64) * 2654435761 % k).astype(np.int32)
    got, moves, visited, tx, ty = oracle.refine_learned(g, k, eps, 7, 4, 21, p0,
                                                        net_const(-8.0), 0.0, 3, trace=True)
    deg = np.diff(g["xadj"])
    r = len(moves)
    assert r >= 3  # gated rounds without moves do not end the run
    full = [i for i in range(r) if i == 0 or i % 3 == 2 or i == 6]
    assert visited == len(full) * int(np.sum(deg > 0))
    for i in range(r):
        if i not in full:
            assert moves[i] == 0
    # balance holds; round 0 sees the start state; moved flags match the moves
    lmax = oracle.lmax(int(g["vwgt"].sum()), k, eps)
    assert np.all(oracle.block_weights(g, got, k) <= lmax)
    W0 = oracle.block_weights(g, p0, k)
    assert np.array_equal(tx[0], oracle.features(g, p0, W0, lmax, np.zeros(n, np.uint8)))
    assert ty.shape == (r, n)
    for i in range(r):
        assert int(ty[i].sum()) == moves[i]
        if i > 0:
            assert np.array_equal(tx[i][:, 3], ty[i - 1].astype(np.float32))
