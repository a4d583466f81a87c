"""Float64 reference of the learned winner proposal -- TEST INFRASTRUCTURE ONLY.

The proposal model is an engineering addition on top of the Schulze method:
the paper has no learned component. Its only link to the paper is that some
of the per-candidate features restate quantities the paper uses: the
dominance relation of Sect. 2.1 (Copeland wins and losses) and the loser
filter of Sect. 4 (largest incoming against largest outgoing edge weight).
Exactness of the winners never depends on the model: every proposal is
certified by widest paths (Sect. 2.1 definitions), with the full closure as
the fallback.

Plain numpy, float64, written step by step; no blocking, fusion or reordering.
"""
from __future__ import annotations

import numpy as np

NFEAT = 16
H = 64
# flat parameter layout: W1 [64][16], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1]
OFF_W1, OFF_B1 = 0, 1024
OFF_W2, OFF_B2 = 1088, 5184
OFF_W3, OFF_B3 = 5248, 5312
NPARAM = 5313


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    W1 = theta[OFF_W1:OFF_B1].reshape(H, NFEAT)
    b1 = theta[OFF_B1:OFF_W2]
    W2 = theta[OFF_W2:OFF_B2].reshape(H, H)
    b2 = theta[OFF_B2:OFF_W3]
    W3 = theta[OFF_W3:OFF_B3]
    b3 = theta[OFF_B3]
    return W1, b1, W2, b2, W3, b3


def features(d, n):
    """16 features per candidate from the tally d (int [m, m]) and n ballots.

    For candidate c, over j != c, with w the winning-votes weights:
      0 Copeland wins / (m-1)          #{j: d[c][j] > d[j][c]}
      1 Copeland losses / (m-1)        #{j: d[j][c] > d[c][j]}
      2 ties / (m-1)                   #{j: d[c][j] == d[j][c]}
      3 sum_j d[c][j] / (n (m-1))      (a Borda-like score)
      4 sum_j d[j][c] / (n (m-1))
      5 max_j w[c][j] / n              (heaviest outgoing edge)
      6 max_j w[j][c] / n              (heaviest incoming edge)
      7 1 if 6 > 5 else 0              (the loser filter of Sect. 4)
      8 (max_j w[c][j] - max_j w[j][c]) / n
      9 sum_j w[c][j] / (n (m-1))
     10 sum_j w[j][c] / (n (m-1))
     11 min_j (d[c][j] - d[j][c]) / n  (worst pairwise margin)
     12 max_j (d[c][j] - d[j][c]) / n  (best pairwise margin)
     13 max_j d[c][j] / n
     14 #{j: rowsum_d[j] > rowsum_d[c]} / (m-1)   (rank by feature 3, 0 = best)
     15 #{j: wins[j] - losses[j] > wins[c] - losses[c]} / (m-1)
    With m == 1 the per-pair features are 0; n == 0 counts as n = 1.
    """
    d = np.asarray(d, dtype=np.int64)
    m = d.shape[0]
    nn = float(max(int(n), 1))
    mm = float(max(m - 1, 1))
    f = np.zeros((m, NFEAT), dtype=np.float64)
    wins = np.zeros(m, np.int64)
    losses = np.zeros(m, np.int64)
    rowsum = np.zeros(m, np.int64)
    for c in range(m):
        others = [j for j in range(m) if j != c]
        if not others:
            continue
        dcj = d[c, others]
        djc = d[others, c]
        wout = np.where(dcj > djc, dcj, 0)
        win = np.where(djc > dcj, djc, 0)
        wins[c] = int(np.sum(dcj > djc))
        losses[c] = int(np.sum(djc > dcj))
        rowsum[c] = int(np.sum(dcj))
        f[c, 0] = wins[c] / mm
        f[c, 1] = losses[c] / mm
        f[c, 2] = np.sum(dcj == djc) / mm
        f[c, 3] = np.sum(dcj) / (nn * mm)
        f[c, 4] = np.sum(djc) / (nn * mm)
        f[c, 5] = wout.max() / nn
        f[c, 6] = win.max() / nn
        f[c, 7] = 1.0 if win.max() > wout.max() else 0.0
        f[c, 8] = (wout.max() - win.max()) / nn
        f[c, 9] = np.sum(wout) / (nn * mm)
        f[c, 10] = np.sum(win) / (nn * mm)
        f[c, 11] = np.min(dcj - djc) / nn
        f[c, 12] = np.max(dcj - djc) / nn
        f[c, 13] = dcj.max() / nn
    cope = wins - losses
    for c in range(m):
        if m > 1:
            f[c, 14] = np.sum(rowsum > rowsum[c]) / mm
            f[c, 15] = np.sum(cope > cope[c]) / mm
    return f


def forward(theta, X):
    """scores [N] and the activations (z1, h1, z2, h2) of the 16-64-64-1 ReLU MLP."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ W3 + b3
    return s, (z1, h1, z2, h2)


def loss_and_grad(theta, X, labels, seg_off):
    """Listwise softmax cross-entropy, averaged over elections.

    Election e owns candidates seg_off[e] .. seg_off[e+1]-1; its target puts
    equal mass on its winners (labels == 1). Returns (loss, grad [NPARAM],
    dscore [N])."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    s, (z1, h1, z2, h2) = forward(theta, X)
    labels = np.asarray(labels)
    E = len(seg_off) - 1
    ds = np.zeros_like(s)
    loss = 0.0
    for e in range(E):
        a, b = int(seg_off[e]), int(seg_off[e + 1])
        se = s[a:b]
        t = labels[a:b].astype(np.float64)
        t = t / t.sum()
        mx = se.max()
        lse = mx + np.log(np.sum(np.exp(se - mx)))
        logp = se - lse
        loss += -np.sum(t * logp)
        ds[a:b] = (np.exp(logp) - t) / E
    loss /= E
    gW3 = h2.T @ ds
    gb3 = ds.sum()
    dh2 = np.outer(ds, W3) * (z2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g, ds


def adam(theta, g, m1, m2, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) at 1-based `step`; returns new
    (theta, m1, m2)."""
    m1 = beta1 * np.asarray(m1, np.float64) + (1 - beta1) * g
    m2 = beta2 * np.asarray(m2, np.float64) + (1 - beta2) * g * g
    mhat = m1 / (1 - beta1 ** step)
    vhat = m2 / (1 - beta2 ** step)
    theta = np.asarray(theta, np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m1, m2
