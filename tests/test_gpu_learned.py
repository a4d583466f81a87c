"""Learned proposal + certification on the GPU against the float64 / integer
oracles. Winner sets must match exactly; the FP32 model within 1e-4."""
import numpy as np
import pytest
import torch

import oracle
import oracle.mlp as M
import workloads as W
from helpers import fig1, mcgarvey_ballots, topk_tie_counterexample

pytestmark = pytest.mark.gpu

S = None


@pytest.fixture(scope="module", autouse=True)
def lib():
    global S
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_12976_gb300 as mod
    S = mod
    yield mod
    assert S.context().status() == S.OK


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def _elections():
    out = []
    _, mu, _, _ = fig1()
    b = mcgarvey_ballots(mu)
    out.append((b, 4))
    g = topk_tie_counterexample()
    out.append((g["ballots"], g["m"]))
    out.append((np.zeros((0, 6), np.int32), 6))
    out.append((np.array([[0]], np.int32), 1))
    out.append((W.impartial(3, 7, 2, 2), 2))
    for t, (m, n, k, phi) in enumerate([(40, 500, 40, 0.9), (150, 2000, 12, 0.85), (300, 900, 30, 1.0),
                                        (777, 3000, 25, 0.95), (64, 1000, 64, 0.8), (2052, 2500, 30, 0.9)]):
        out.append((W.mallows(50 + t, n, m, k, phi, W.permutation(50 + t, m)), m))
    return out


@pytest.mark.parametrize("case", range(11))
def test_features_match_oracle(case):
    r, m = _elections()[case]
    d = oracle.tally(r, m)
    f = S.schulze_features(cu(d), r.shape[0])
    np.testing.assert_allclose(f.cpu().numpy(), M.features(d, r.shape[0]), rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("m", [300, 301])
@pytest.mark.parametrize("scale", [1, 20, 1 << 19])
def test_features_every_count_width_matches_oracle(m, scale):
    """The features pass counts two entries per instruction (16-bit lanes)
    for n <= 32766, one at a time with 32-bit partial sums below 2^29 and
    with 64-bit sums above; a tally scaled by `scale` (with n scaled alike,
    so entries stay in [0, n]) takes each of the three, with rows of d
    16-byte aligned (m = 300) or not (m = 301)."""
    r = W.mallows(77, 1100, m, 30, 0.9, W.permutation(77, m))
    d = oracle.tally(r, m).astype(np.int64) * scale
    n = r.shape[0] * scale
    f = S.schulze_features(cu(d), n)
    np.testing.assert_allclose(f.cpu().numpy(), M.features(d, n), rtol=1e-6, atol=1e-7)


def test_features_of_an_unaligned_tally():
    """d one element past a 16-byte boundary with m a multiple of 4: the
    features pass copies it element by element and matches the oracle."""
    m = 300
    r = W.mallows(78, 900, m, 25, 0.9, W.permutation(78, m))
    d = oracle.tally(r, m)
    buf = torch.full((m * m + 1,), -9, dtype=torch.int32, device="cuda")
    t = buf[1:].view(m, m)
    assert t.data_ptr() % 16 != 0
    t.copy_(cu(d))
    f = S.schulze_features(t, r.shape[0])
    np.testing.assert_allclose(f.cpu().numpy(), M.features(d, r.shape[0]), rtol=1e-6, atol=1e-7)


def test_mlp_forward_matches_oracle():
    rs = np.random.Generator(np.random.PCG64(1))
    theta = W.mlp_init(3)
    X = rs.normal(size=(1000, 16)).astype(np.float32)
    s = S.schulze_mlp_forward(torch.from_numpy(theta).cuda(), torch.from_numpy(X).cuda())
    want, _ = M.forward(theta.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(s.cpu().numpy(), want, rtol=1e-4, atol=1e-5)


def _train_batch(seed, E=6):
    rs = np.random.Generator(np.random.PCG64(seed))
    feats, labels, seg = [], [], [0]
    for e in range(E):
        m = int(rs.integers(20, 200))
        r = W.mallows(seed * 100 + e, int(rs.integers(100, 800)), m, int(rs.integers(3, 20)), 0.9,
                      W.permutation(e, m))
        d = oracle.tally(r, m)
        feats.append(M.features(d, r.shape[0]))
        labels.append(oracle.winners(oracle.strongest_paths(d)))
        seg.append(seg[-1] + m)
    return (np.concatenate(feats).astype(np.float32), np.concatenate(labels).astype(np.int32),
            np.array(seg, np.int32))


def test_train_step_matches_oracle_and_is_deterministic():
    X, lab, seg = _train_batch(4)
    theta0 = W.mlp_init(5)
    lr = 1e-2
    want_loss, want_g, _ = M.loss_and_grad(theta0.astype(np.float64), X.astype(np.float64), lab, seg)
    want_theta, want_m1, want_m2 = M.adam(theta0.astype(np.float64), want_g, np.zeros(M.NPARAM),
                                          np.zeros(M.NPARAM), 1, lr)
    outs = []
    for _ in range(2):
        p = torch.from_numpy(theta0.copy()).cuda()
        m1 = torch.zeros(M.NPARAM, device="cuda")
        m2 = torch.zeros(M.NPARAM, device="cuda")
        loss, g = S.schulze_mlp_train_step(p, m1, m2, 1, torch.from_numpy(X).cuda(), cu(lab), cu(seg), lr)
        torch.cuda.synchronize()
        outs.append((loss.item(), g.cpu().numpy(), p.cpu().numpy(), m1.cpu().numpy(), m2.cpu().numpy()))
    loss, g, p, m1, m2 = outs[0]
    assert loss == pytest.approx(want_loss, rel=1e-5)
    scale = np.abs(want_g).max()
    np.testing.assert_allclose(g, want_g, rtol=1e-4, atol=1e-4 * scale)
    np.testing.assert_allclose(m1, want_m1, rtol=1e-4, atol=1e-5 * scale)
    # the first Adam step moves every parameter by about lr * sign(g) where g is not tiny
    big = np.abs(want_g) > 1e-3 * scale
    np.testing.assert_allclose(p[big], want_theta[big], rtol=1e-4, atol=1e-6)
    for a, b in zip(outs[0], outs[1]):  # same inputs, same bits
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


def test_training_reduces_the_loss():
    X, lab, seg = _train_batch(7, E=16)
    p = torch.from_numpy(W.mlp_init(8)).cuda()
    m1, m2 = torch.zeros(M.NPARAM, device="cuda"), torch.zeros(M.NPARAM, device="cuda")
    Xd, ld, sd = torch.from_numpy(X).cuda(), cu(lab), cu(seg)
    losses = []
    for step in range(1, 201):
        loss, _ = S.schulze_mlp_train_step(p, m1, m2, step, Xd, ld, sd, 3e-3)
        losses.append(loss.item())
    assert losses[-1] < 0.6 * losses[0]


@pytest.mark.parametrize("case", range(10))
def test_certify_true_and_false_proposals(case):
    r, m = _elections()[case]
    d = oracle.tally(r, m)
    want = oracle.winners(oracle.strongest_paths(d))
    dd = cu(d)
    win_ids = np.flatnonzero(want)
    losers = np.flatnonzero(want == 0)
    # a winner proposed first: exact winner set
    w, res = S.schulze_certify(dd, r.shape[0], cu(win_ids[:1]))
    res = res.cpu().numpy()
    if res[0] == 1:
        np.testing.assert_array_equal(w.cpu().numpy(), want)
    else:  # only allowed when the winner has no outgoing edge (edge-less profiles)
        assert oracle.weights(d)[win_ids[0]].max() == 0
    # losers only: never certified
    if losers.size:
        _, res2 = S.schulze_certify(dd, r.shape[0], cu(losers[:4]))
        assert res2.cpu().numpy()[0] == 0
        # a loser then a winner: the second proposal certifies
        w3, res3 = S.schulze_certify(dd, r.shape[0], cu(np.array([losers[0], win_ids[0]])))
        res3 = res3.cpu().numpy()
        if res3[0] == 1:
            assert res3[1] == 1
            np.testing.assert_array_equal(w3.cpu().numpy(), want)


@pytest.mark.parametrize("case", range(10))
def test_winners_fast_exact(case):
    r, m = _elections()[case]
    d = oracle.tally(r, m)
    want = oracle.winners(oracle.strongest_paths(d))
    for params in (None, torch.from_numpy(W.mlp_init(9)).cuda()):
        w, stats = S.schulze_winners_fast(cu(d), r.shape[0], params, top=4)
        np.testing.assert_array_equal(w.cpu().numpy(), want)
        assert stats[1] in (0, 1)
        assert (stats[0] >= 0) == (stats[1] == 0)


def test_winners_fast_large_election_against_closure():
    e = W.large_topk(seed=31, n=20000, m=4096, k=50)
    ranks = cu(e.ranks)
    out = S.schulze_run(ranks, e.m)
    w, stats = S.schulze_winners_fast(out["d"], e.n, None, top=4)
    assert torch.equal(w, out["winners"])
    assert stats[1] == 0  # the Copeland proposal certified: no closure needed


@pytest.fixture(scope="module")
def trained_params():
    """A proposal network trained by the library on 192 GPU-solved elections
    drawn like the training set of the learned-proposal workload (m in
    [256, 2048], top-k Mallows), eight epochs: small, but trained."""
    from paper_2505_12976_gb300 import learned as L
    data = L.Dataset("cuda")
    tb = W.learned_train(E=192, seed=4242)
    for e in range(tb.E):
        data.add(cu(tb.election(e).ranks), int(tb.m[e]))
    tr = L.Trainer(W.mlp_init(11), seed=12)
    hist = tr.train(data, epochs=8, elections_per_step=32, lr=3e-3)
    assert hist[-1] < hist[0]
    return tr.params


def test_learned_eval_elections_match_oracle(trained_params):
    """Evaluation elections of the learned-proposal workload at full size
    (m = 8192, n = 20000, top-50 Mallows(0.9)), eight of them: the winners
    from trained proposals equal the oracle's. The oracle works on the
    listed candidates A only: an unlisted candidate is preferred to nobody,
    so it has no outgoing edge, every listed one beats it, and paths between
    listed candidates never leave A (Sect. 2.1 definitions); the tally of
    the ballots relabeled to A is d[A, A], checked against the GPU's."""
    ev = W.learned_eval(E=8)
    for e in range(ev.E):
        r, m, n = ev.election(e).ranks, int(ev.m[e]), int(ev.n[e])
        d = S.schulze_tally(cu(r), m)
        A = np.unique(r)
        idx = np.full(m, -1, np.int32)
        idx[A] = np.arange(A.size, dtype=np.int32)
        dA = oracle.tally(idx[r], A.size)
        np.testing.assert_array_equal(d.cpu().numpy()[np.ix_(A, A)], dA)
        want = np.zeros(m, np.int32)
        want[A] = oracle.winners(oracle.strongest_paths(dA, nthreads=8))
        for params in (trained_params, None):
            w, stats = S.schulze_winners_fast(d, n, params, top=4)
            np.testing.assert_array_equal(w.cpu().numpy(), want)
            assert stats[1] in (0, 1)


def test_winners_fast_dense_profile_uses_propagation():
    """A dense profile whose warm set is too large to certify (every one of
    2200 candidates has an outgoing edge): the paper's propagation decides,
    exactly, instead of the closure."""
    m, n, k = 2200, 1500, 2200
    r = W.impartial(77, n, m, k)
    d = S.schulze_tally(cu(r), m)
    want = oracle.winners(oracle.strongest_paths(d.cpu().numpy(), nthreads=8))
    w, stats = S.schulze_winners_fast(d, n, None, top=4)
    assert stats[1] == 2, stats
    np.testing.assert_array_equal(w.cpu().numpy(), want)


def test_trained_proposals_gain_over_copeland():
    """What the trained network gains over the method without it (the
    Copeland score wins - losses as the proposer). Trained by the library on
    2000 GPU-solved elections of the learned workload's training model,
    twenty epochs (training is deterministic, so the counts below repeat).
    Evaluated on near-uniform profiles (Mallows phi 0.99, 0.995, 1.0; m 300
    and 1000; 2000 top-30 ballots), where the top of the majority graph has
    cycles and Copeland's first choice is sometimes not a Schulze winner:
    the network's first choice must be a winner at least as often, and must
    be right on some elections where Copeland's is not. Winner sets from both
    proposers stay exact (the closure judges; the oracle judges the m = 300
    ones). The counts are printed."""
    from paper_2505_12976_gb300 import learned as L
    data = L.Dataset("cuda")
    for c0 in range(0, 2000, 256):
        tb = W.learned_train(E=min(256, 2000 - c0), seed=W.SEED_BASE + 4 + 7919 * c0)
        for e in range(tb.E):
            data.add(cu(tb.election(e).ranks), int(tb.m[e]))
    tr = L.Trainer(W.mlp_init(), seed=W.SEED_BASE + 6)
    tr.train(data, epochs=20, elections_per_step=64, lr=3e-3)
    tally = {"E": 0, "mlp_hit1": 0, "cop_hit1": 0, "cop_miss": 0, "mlp_hit1_where_cop_misses": 0}
    for phi in (0.99, 0.995, 1.0):
        for s in range(32):
            m = 300 if s % 2 else 1000
            r = W.mallows(5000 + s, 2000, m, 30, phi, W.permutation(77 + s, m))
            out = S.schulze_run(cu(r), m)
            win = out["winners"].cpu().numpy()
            if m == 300:
                np.testing.assert_array_equal(win, oracle.winners(oracle.strongest_paths(oracle.tally(r, m))))
            d, n = out["d"], r.shape[0]
            mlp = S.schulze_mlp_forward(tr.params, S.schulze_features(d, n)).cpu().numpy()
            dn = d.cpu().numpy()
            cop = ((dn > dn.T).sum(1) - (dn < dn.T).sum(1)).astype(np.float64)
            hit_m, hit_c = bool(win[np.argmax(mlp)]), bool(win[np.argmax(cop)])
            tally["E"] += 1
            tally["mlp_hit1"] += hit_m
            tally["cop_hit1"] += hit_c
            tally["cop_miss"] += not hit_c
            tally["mlp_hit1_where_cop_misses"] += hit_m and not hit_c
            for params in (tr.params, None):
                w, _ = S.schulze_winners_fast(d, n, params, top=4)
                np.testing.assert_array_equal(w.cpu().numpy(), win)
    print("proposal first-choice hits on near-uniform profiles:", tally)
    assert tally["mlp_hit1"] >= tally["cop_hit1"]
    assert tally["cop_miss"] == 0 or tally["mlp_hit1_where_cop_misses"] >= 1
