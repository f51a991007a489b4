"""Learned refinement gate on the GPU against the CPU oracle: scorer and
gated refinement bit for bit (partition, rounds, visited nodes, traces);
gradient within 1e-3 of the oracle's float64 gradient; training lowers the
loss; the trace -> train -> threshold -> gated-refinement pipeline."""
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


def bits_of(p):
    """bf16 bit patterns (uint16 numpy) of float32 parameters via the oracle's rounding."""
    p = np.asarray(p, np.float32)
    r = np.array([oracle.bf16(float(v)) for v in p], np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def dev_bits(b):
    return torch.from_numpy(b.view(np.int16).copy()).cuda()


def random_net(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(oracle.MLP_NPARAM) * scale).astype(np.float32)


GRAPHS = {
    "chunglu2k": lambda: I.chung_lu(2048, 2.1, 8.0, seed=3),
    "weighted": lambda: I.random_graph(3000, 12000, seed=5, max_w=20, max_c=9),
    "rmat14": lambda: I.rmat(14, 16, seed=2),
}


def test_score_matches_oracle_bit_for_bit():
    rng = np.random.default_rng(1)
    X = rng.random((5000, 6)).astype(np.float32) * 4
    X = np.array([[oracle.bf16(float(v)) for v in r] for r in X], np.float32)
    for seed in (1, 2):
        net = bits_of(random_net(seed))
        want = oracle.mlp_score(X, net)
        got = S.sclap_mlp_score(torch.from_numpy(X).cuda(), dev_bits(net)).cpu().numpy()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_without_net_equals_plain_refinement(name):
    g = GRAPHS[name]()
    n = g["vwgt"].numel()
    p0 = (torch.arange(n, dtype=torch.int64) * 2654435761 % 8).to(torch.int32).cuda()
    want, cut_w, _, rd_w = S.sclap_refine(I.to_device(g, "cuda"), 8, 0.03, 6, 4, 21, p0)
    got, cut_g, _, rd_g, vis, _, _ = S.sclap_refine_learned(I.to_device(g, "cuda"), 8, 0.03, 6,
                                                            4, 21, p0)
    assert torch.equal(got, want) and cut_g == cut_w and rd_g == rd_w
    deg = np.diff(I.to_numpy(g)["xadj"])
    assert vis == rd_g * int(np.sum(deg > 0))


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("k", [4, 16, 100])
def test_gated_refinement_matches_oracle(name, k):
    g = GRAPHS[name]()
    gn = I.to_numpy(g)
    n = gn["vwgt"].size
    p0 = (np.arange(n, dtype=np.int64) * 2654435761 % k).astype(np.int32)
    net = bits_of(random_net(7))
    # threshold at the median start-of-run logit: about half the nodes gated out
    lmax = oracle.lmax(int(gn["vwgt"].sum()), k, 0.03)
    x0 = oracle.features(gn, p0, oracle.block_weights(gn, p0, k), lmax, None)
    z_min = float(np.median(oracle.mlp_score(x0, net)))
    want, mv_w, vis_w, tx_w, ty_w = oracle.refine_learned(gn, k, 0.03, 8, 4, 13, p0, net, z_min,
                                                          3, trace=True)
    got, cut, bw, rd, vis, tx, ty = S.sclap_refine_learned(
        I.to_device(g, "cuda"), k, 0.03, 8, 4, 13, torch.from_numpy(p0).cuda(), dev_bits(net),
        z_min, 3, trace=True)
    assert rd == len(mv_w) and vis == vis_w
    assert np.array_equal(got.cpu().numpy(), want)
    assert np.array_equal(tx.cpu().numpy().view(np.uint32), tx_w.view(np.uint32))
    assert np.array_equal(ty.cpu().numpy(), ty_w)
    assert cut == oracle.cut(gn, want)


@pytest.mark.parametrize("bf16_in", [False, True])
def test_loss_gradient_matches_oracle(bf16_in):
    rng = np.random.default_rng(4)
    X = (rng.random((20000, 6)) * 3).astype(np.float32)
    if bf16_in:  # trace features are bf16 values
        X = np.array([[oracle.bf16(float(v)) for v in row] for row in X], np.float32)
    y = (rng.random(20000) < 0.2).astype(np.uint8)
    p = random_net(9, 0.3)
    loss_w, g_w = oracle.mlp_loss_grad(X, y, p, bf16_in=bf16_in)
    loss_g, g_g = S.sclap_mlp_loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(),
                                        torch.from_numpy(p).cuda(), bf16_in=bf16_in)
    g_g = g_g.cpu().numpy().astype(np.float64)
    assert loss_g == pytest.approx(loss_w, rel=1e-3)
    assert np.max(np.abs(g_g - g_w)) <= 1e-3 * np.max(np.abs(g_w))
    assert np.linalg.norm(g_g - g_w) <= 1e-3 * np.linalg.norm(g_w)
    if bf16_in:  # the rounding matters for this network
        assert not np.allclose(g_w, oracle.mlp_loss_grad(X, y, p)[1], rtol=1e-4)


def test_training_lowers_the_loss():
    rng = np.random.default_rng(6)
    X = rng.random((30000, 6)).astype(np.float32)
    y = ((X[:, 0] + 0.5 * X[:, 3]) > 0.9).astype(np.uint8)
    p0 = random_net(3, 0.2)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    l0, _ = S.sclap_mlp_loss_grad(Xd, yd, torch.from_numpy(p0).cuda(), bf16_in=True)
    p1, l1 = S.sclap_mlp_train(Xd, yd, torch.from_numpy(p0).cuda(), 8, 256, 0.5, 5)
    assert l1 < 0.6 * l0 and l1 < 0.4
    # training reports the BF16-in loss of the network inference will run
    lw, _ = oracle.mlp_loss_grad(X, y, p1.cpu().numpy(), bf16_in=True)
    assert l1 == pytest.approx(lw, rel=1e-3)


def test_trace_train_threshold_gate_pipeline():
    g = I.rmat(14, 16, seed=5)
    gn = I.to_numpy(g)
    gd = I.to_device(g, "cuda")
    n, k = gn["vwgt"].size, 16
    xs, ys = [], []
    for seed in (1, 2, 3):  # traces of plain refinement
        p0 = torch.from_numpy(((np.arange(n) * 2654435761 + seed) % k).astype(np.int32)).cuda()
        _, _, _, rd, _, tx, ty = S.sclap_refine_learned(gd, k, 0.03, 6, 4, seed, p0, trace=True)
        xs.append(tx.reshape(-1, 6))
        ys.append(ty.reshape(-1))
    X, Y = torch.cat(xs), torch.cat(ys)
    prm, loss = S.sclap_mlp_train(X, Y, torch.from_numpy(random_net(2, 0.2)).cuda(), 4, 1024,
                                  0.5, 9)
    net = S.bf16_bits(prm)
    z = S.sclap_mlp_score(X, net)
    zm = z[Y.bool()]
    z_min = float(torch.sort(zm).values[int(0.01 * zm.numel())])  # move recall >= 0.99
    for seed in (17, 18):  # evaluation seeds
        p0 = ((np.arange(n) * 2654435761 + seed) % k).astype(np.int32)
        want, mv, vis_w, _, _ = oracle.refine_learned(gn, k, 0.03, 6, 4, seed, p0,
                                                      net.cpu().numpy().view(np.uint16),
                                                      z_min, 3)
        got, cut, bw, rd, vis, _, _ = S.sclap_refine_learned(gd, k, 0.03, 6, 4, seed,
                                                             torch.from_numpy(p0).cuda(), net,
                                                             z_min, 3)
        assert np.array_equal(got.cpu().numpy(), want) and vis == vis_w and rd == len(mv)
        lmax = oracle.lmax(int(gn["vwgt"].sum()), k, 0.03)
        assert int(bw.max()) <= lmax


def test_pack_bf16_matches_oracle_rounding():
    rng = np.random.default_rng(5)
    p = (rng.standard_normal(oracle.MLP_NPARAM) * 3).astype(np.float32)
    # exact ties at both parities, values just above a tie, signed zero
    p[:6] = np.array([1.0 + 2**-8, 1.0 + 3 * 2**-8, 1.0 + 2**-8 + 2**-12, -(1.0 + 2**-8),
                      -0.0, 3.0e38], np.float32)
    got = S.bf16_bits(torch.from_numpy(p).cuda()).cpu().numpy().view(np.uint16)
    assert np.array_equal(got, bits_of(p))
