"""Pins of the float64 proposal-model reference (no GPU needed): features
against hand-derived values of the Fig. 1 profile and counting identities,
gradients against central finite differences, the loss against its closed
form for equal scores, and the first Adam step against its closed form."""
import numpy as np
import pytest

import oracle
import oracle.mlp as M
import workloads as W
from helpers import fig1, mcgarvey_ballots


def test_features_of_fig1_profile():
    """Fig. 1 realised by 42 ballots: d = 21 + margin / 2 on every pair."""
    _, mu, _, _ = fig1()
    ballots = mcgarvey_ballots(mu)
    d = oracle.tally(ballots, 4)
    f = M.features(d, 42)
    # a: beats b (23-19) and c (24-18), loses to d (20-22)
    np.testing.assert_allclose(f[0, :3], [2 / 3, 1 / 3, 0.0])
    np.testing.assert_allclose(f[0, 5:9], [24 / 42, 22 / 42, 0.0, 2 / 42])
    # b: out edge b->c 26, in edges a->b 23, d->b 27: the loser filter fires (Sect. 4)
    np.testing.assert_allclose(f[1, 5:8], [26 / 42, 27 / 42, 1.0])
    # full rankings: row + column sums = n (m - 1)
    np.testing.assert_allclose(f[:, 3] + f[:, 4], 1.0)
    # margins of a: +4, +6, -2
    np.testing.assert_allclose(f[0, 11:13], [-2 / 42, 6 / 42])
    # Borda order of the rows: a 67, b 60, c 59, d 66 -> ranks 0, 2, 3, 1
    np.testing.assert_allclose(f[:, 14] * 3, [0, 2, 3, 1])


@pytest.mark.parametrize("seed", range(4))
def test_feature_identities(seed):
    r = W.mallows(seed, 200, 25, 6, 0.8, W.permutation(seed, 25))
    d = oracle.tally(r, 25)
    f = M.features(d, 200)
    np.testing.assert_allclose(f[:, 0] + f[:, 1] + f[:, 2], 1.0)
    win = oracle.winners(oracle.strongest_paths(d))
    assert np.all(win[f[:, 7] == 1] == 0)  # the loser filter never hits a winner
    w = oracle.weights(d)
    np.testing.assert_allclose(f[:, 5], w.max(axis=1) / 200)
    np.testing.assert_allclose(f[:, 6], w.max(axis=0) / 200)
    # relabeling permutes the per-candidate features
    pi = np.random.Generator(np.random.PCG64(seed)).permutation(25).astype(np.int32)
    f2 = M.features(oracle.tally(pi[r], 25), 200)
    np.testing.assert_allclose(f2[pi], f, atol=1e-12)


def _toy(seed, E=3):
    rs = np.random.Generator(np.random.PCG64(seed))
    sizes = rs.integers(3, 9, E)
    seg = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    X = rs.normal(size=(int(seg[-1]), 16))
    labels = np.zeros(int(seg[-1]), np.int32)
    for e in range(E):
        labels[seg[e] + rs.integers(0, sizes[e], 1 + (e % 2))] = 1
    theta = W.mlp_init(seed).astype(np.float64) + rs.normal(0, 0.05, M.NPARAM)
    return theta, X, labels, seg


@pytest.mark.parametrize("seed", range(3))
def test_gradient_matches_central_differences(seed):
    theta, X, labels, seg = _toy(seed)
    loss, g, _ = M.loss_and_grad(theta, X, labels, seg)
    rs = np.random.Generator(np.random.PCG64(100 + seed))
    idx = np.concatenate([rs.choice(M.NPARAM - 1, 60, replace=False), [M.OFF_B3]])
    h = 1e-6
    for t in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[t] += h
        tm[t] -= h
        num = (M.loss_and_grad(tp, X, labels, seg)[0] - M.loss_and_grad(tm, X, labels, seg)[0]) / (2 * h)
        assert abs(num - g[t]) <= 1e-7 + 1e-5 * abs(num), (t, num, g[t])


def test_loss_closed_form_for_equal_scores():
    """All scores equal: softmax is uniform, so the loss is log(m_e) averaged
    over elections whatever the number of winners."""
    theta = np.zeros(M.NPARAM)
    theta[M.OFF_B3] = 0.7
    seg = np.array([0, 5, 12, 14])
    labels = np.array([1, 0, 0, 0, 0, 0, 1, 1, 0, 0, 0, 0, 1, 1])
    X = np.random.Generator(np.random.PCG64(1)).normal(size=(14, 16))
    loss, g, ds = M.loss_and_grad(theta, X, labels, seg)
    assert loss == pytest.approx((np.log(5) + np.log(7) + np.log(2)) / 3, rel=1e-12)
    # d loss / d b3 = sum of (p - t) / E = 0
    assert g[M.OFF_B3] == pytest.approx(0.0, abs=1e-12)


def test_first_adam_step_closed_form():
    """At step 1 the bias-corrected moments are g and g^2: the step is
    lr * g / (|g| + eps)."""
    rs = np.random.Generator(np.random.PCG64(2))
    theta = rs.normal(size=M.NPARAM)
    g = rs.normal(size=M.NPARAM)
    t1, m1, m2 = M.adam(theta, g, np.zeros(M.NPARAM), np.zeros(M.NPARAM), 1, 1e-3)
    np.testing.assert_allclose(t1, theta - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(m2, 0.001 * g * g)
