"""Pins of the CPU oracle to the paper and to mathematics (no GPU needed).

Each test fixes the oracle against something other than itself: the worked
example of Fig. 1, McGarvey's construction, brute-force path enumeration,
max-min Dijkstra, counting identities of the tally, the NL-hardness family
of Sect. 3, the Schwartz-set refinement and the loser filter of Sect. 4.
"""
import itertools

import numpy as np
import pytest

import oracle
import workloads as W
from helpers import (brute_force_widths, fig1, mcgarvey_ballots, nl_reduction, random_digraph, reachable,
                     schwartz_set, topk_tie_counterexample)


# ---------------------------------------------------------------- Fig. 1

def test_fig1_widest_path_table():
    """Closure of the Fig. 1 graph equals the table printed beside it."""
    names, mu, p_paper, win = fig1()
    p = oracle.closure(mu)
    np.testing.assert_array_equal(p, p_paper)
    assert list(np.flatnonzero(oracle.winners(p))) == win == [0]


def test_fig1_from_margins_matrix():
    """d holding the margins on each edge and 0 on its reverse gives the same
    weights and the same table (edge weight = count where it beats the reverse)."""
    _, mu, p_paper, _ = fig1()
    np.testing.assert_array_equal(oracle.weights(mu), mu)
    np.testing.assert_array_equal(oracle.strongest_paths(mu), p_paper)


def test_fig1_mcgarvey_end_to_end():
    """Fig. 1 realised by 42 linear orders (McGarvey): the tally reproduces the
    margins, and winning-vote widths are (n + margin width) / 2 (Sect. 2.1)."""
    _, mu, p_paper, win = fig1()
    ballots = mcgarvey_ballots(mu)
    n, m = ballots.shape
    assert n == int(mu.sum()) == 42
    d = oracle.tally(ballots, m)
    # the margins of the figure, recovered from the counts
    np.testing.assert_array_equal(oracle.weights_margin(d), mu)
    off = ~np.eye(m, dtype=bool)
    assert (d + d.T)[off].tolist() == [n] * (m * m - m)
    np.testing.assert_array_equal(d, [[0, 23, 24, 20], [19, 0, 26, 15], [18, 16, 0, 25], [22, 27, 17, 0]])
    p = oracle.strongest_paths(d)
    expect = np.where(off, (n + p_paper) // 2, 0)
    np.testing.assert_array_equal(p, expect)
    assert list(np.flatnonzero(oracle.winners(p))) == win
    order, bb = oracle.ranking(p)
    assert bb.tolist() == [0, 2, 3, 1]
    assert order.tolist() == [0, 3, 1, 2]  # a, d, b, c
    # margin-weighted closure reproduces the printed table itself
    np.testing.assert_array_equal(oracle.closure(oracle.weights_margin(d)), p_paper)


def test_topk_tie_counterexample_golden():
    g = topk_tie_counterexample()
    d = oracle.tally(g["ballots"], g["m"])
    np.testing.assert_array_equal(d, g["d"])
    p = oracle.strongest_paths(d)
    np.testing.assert_array_equal(p, g["p"])
    assert list(np.flatnonzero(oracle.winners(p))) == g["winners"]
    order, bb = oracle.ranking(p)
    assert bb.tolist() == g["beaten_by"]
    assert order.tolist() == g["ranking"]
    # R = {p(a,b) >= p(b,a)} is not transitive here: 1 R 0, 0 R 2, not 1 R 2
    R = p >= p.T
    assert R[1, 0] and R[0, 2] and not R[1, 2]


# ------------------------------------------------------- brute force

def _small_profiles():
    rs = np.random.Generator(np.random.PCG64(7))
    out = []
    for t in range(60):
        m = int(rs.integers(1, 8))
        n = int(rs.integers(0, 12))
        k = int(rs.integers(0, m + 1))
        kind = t % 3
        if kind == 0:
            r = W.impartial(1000 + t, n, m, k)
        elif kind == 1:
            r = W.mallows(1000 + t, n, m, k, float(rs.uniform(0.3, 1.0)), W.permutation(t, m))
        else:
            r = W.mallows(1000 + t, n, m, k, 1.0)
        out.append((r, m))
    return out


@pytest.mark.parametrize("case", range(60))
def test_closure_equals_brute_force_paths(case):
    r, m = _small_profiles()[case]
    d = oracle.tally(r, m)
    w = oracle.weights(d)
    np.testing.assert_array_equal(oracle.closure(w), brute_force_widths(w))


def test_closure_brute_force_random_weights():
    """Arbitrary nonnegative weight matrices (not only tournaments)."""
    rs = np.random.Generator(np.random.PCG64(11))
    for _ in range(40):
        m = int(rs.integers(2, 8))
        w = rs.integers(0, 6, size=(m, m)).astype(np.int32)
        w[rs.random((m, m)) < 0.4] = 0
        np.fill_diagonal(w, 0)
        np.testing.assert_array_equal(oracle.closure(w), brute_force_widths(w))


# ---------------------------------------------------- Dijkstra rows

def test_dijkstra_rows_and_columns_match_closure():
    e = W.large_topk(seed=5, n=400, m=160, k=12)
    d = oracle.tally(e.ranks, e.m)
    w = oracle.weights(d)
    p = oracle.closure(w)
    for s in (0, 1, 77, 159):
        np.testing.assert_array_equal(oracle.widest_from(w, s), p[s])
        np.testing.assert_array_equal(oracle.widest_to(w, s), p[:, s])


def test_dijkstra_batched_rows_and_columns():
    """The batched form (sources spread over threads) gives the same rows and
    columns as the closure."""
    e = W.large_topk(seed=6, n=500, m=140, k=15)
    w = oracle.weights(oracle.tally(e.ranks, e.m))
    p = oracle.closure(w)
    src = [0, 3, 70, 139, 3]
    np.testing.assert_array_equal(oracle.widest_many(w, src, nthreads=4), p[src])
    np.testing.assert_array_equal(oracle.widest_many(w, src, transpose=True, nthreads=4), p[:, src].T)
    assert oracle.widest_many(w, []).shape == (0, e.m)


def test_dijkstra_brute_force():
    rs = np.random.Generator(np.random.PCG64(12))
    for _ in range(30):
        m = int(rs.integers(2, 8))
        w = rs.integers(0, 9, size=(m, m)).astype(np.int32)
        w[rs.random((m, m)) < 0.5] = 0
        np.fill_diagonal(w, 0)
        bf = brute_force_widths(w)
        for s in range(m):
            np.testing.assert_array_equal(oracle.widest_from(w, s), bf[s])
            np.testing.assert_array_equal(oracle.widest_to(w, s), bf[:, s])


# --------------------------------------------------- tally identities

@pytest.mark.parametrize("m,n,seed", [(2, 5, 1), (7, 40, 2), (33, 200, 3), (64, 1000, 4)])
def test_full_ranking_identities(m, n, seed):
    r = W.impartial(seed, n, m, m)
    d = oracle.tally(r, m)
    off = ~np.eye(m, dtype=bool)
    assert np.all((d + d.T)[off] == n)
    assert np.all(np.diag(d) == 0)
    # row sums are Borda scores: position q earns m - 1 - q points
    borda = np.zeros(m, dtype=np.int64)
    for row in r:
        for q, c in enumerate(row):
            borda[c] += m - 1 - q
    np.testing.assert_array_equal(d.sum(axis=1), borda)


@pytest.mark.parametrize("m,n,k,seed", [(5, 30, 2, 1), (40, 300, 7, 2), (100, 500, 1, 3), (50, 100, 49, 4)])
def test_topk_identities(m, n, k, seed):
    r = W.mallows(seed, n, m, k, 0.85, W.permutation(seed, m))
    d = oracle.tally(r, m)
    listed = np.zeros((n, m), dtype=bool)
    listed[np.repeat(np.arange(n), k), r.reshape(-1)] = True
    either = (listed[:, :, None] | listed[:, None, :]).sum(axis=0)
    off = ~np.eye(m, dtype=bool)
    np.testing.assert_array_equal((d + d.T)[off], either[off])
    # a listed candidate at position q is preferred to the m - 1 - q others
    rowsum = np.zeros(m, dtype=np.int64)
    for row in r:
        for q, c in enumerate(row):
            rowsum[c] += m - 1 - q
    np.testing.assert_array_equal(d.sum(axis=1), rowsum)
    # voter order does not matter, and tallies add over disjoint electorates
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(n)
    np.testing.assert_array_equal(oracle.tally(r[perm], m), d)
    h = n // 2
    np.testing.assert_array_equal(oracle.tally(r[:h], m) + oracle.tally(r[h:], m), d)


@pytest.mark.parametrize("case", ["full", "topk", "topk_one", "no_ballots", "empty_ballots", "one_candidate"])
def test_tally_entry_counts_like_the_tally(case):
    """The voter-by-voter count of one entry (used for sampled checks of
    profiles too large for the whole tally) equals the whole tally entry by
    entry, unlisted candidates included, and vanishes where nobody votes."""
    if case == "full":
        m, r = 9, W.mallows(31, 70, 9, 9, 0.8, W.permutation(31, 9))
    elif case == "topk":
        m, r = 14, W.mallows(32, 90, 14, 4, 0.9, W.permutation(32, 14))
    elif case == "topk_one":
        m, r = 6, W.impartial(33, 25, 6, 1)
    elif case == "no_ballots":
        m, r = 5, np.zeros((0, 3), np.int32)
    elif case == "empty_ballots":
        m, r = 5, np.zeros((7, 0), np.int32)
    else:
        m, r = 1, np.zeros((4, 1), np.int32)
    d = oracle.tally(r, m)
    got = np.array([[oracle.tally_entry(r, m, i, j) for j in range(m)] for i in range(m)])
    np.testing.assert_array_equal(got, d)
    if case in ("no_ballots", "empty_ballots"):
        assert not got.any()
    if case.startswith("topk"):
        unlisted = np.setdiff1d(np.arange(m), np.unique(r))
        for a in unlisted:  # an unlisted candidate is preferred to nobody
            assert not got[a].any()


def test_tally_entry_hand_derived():
    """Entries fixed by hand rather than by the tally: the tie counterexample
    (ballots [0, 2] and [2, 1] over three candidates) and Fig. 1 realised by
    McGarvey's construction (d[a][b] = 21 + mu(a, b) / 2 off the diagonal)."""
    g = topk_tie_counterexample()
    for i in range(g["m"]):
        for j in range(g["m"]):
            assert oracle.tally_entry(g["ballots"], g["m"], i, j) == g["d"][i][j], (i, j)
    _, mu, _, _ = fig1()
    ballots = mcgarvey_ballots(mu)
    n = ballots.shape[0]
    for i in range(4):
        for j in range(4):
            want = 0 if i == j else (n + int(mu[i, j]) - int(mu[j, i])) // 2
            assert oracle.tally_entry(ballots, 4, i, j) == want, (i, j)


def test_unlisted_candidates_tie():
    """k = m - 1 lists all but one candidate: same as the full ranking with the
    missing one appended last."""
    r = W.impartial(9, 50, 6, 5)
    full = np.concatenate([r, np.array([[c for c in range(6) if c not in row] for row in r], np.int32)], 1)
    np.testing.assert_array_equal(oracle.tally(r, 6), oracle.tally(full, 6))


def test_validation_rejects_bad_ballots():
    assert oracle.validate(np.array([[0, 1], [1, 1]], np.int32), 3) == oracle.EDATA
    assert oracle.validate(np.array([[0, 3]], np.int32), 3) == oracle.EDATA
    assert oracle.validate(np.array([[0, -1]], np.int32), 3) == oracle.EDATA
    assert oracle.validate(np.array([[2, 0]], np.int32), 3) == oracle.OK
    with pytest.raises(oracle.OracleError):
        oracle.tally(np.array([[0, 0]], np.int32), 2)


# ------------------------------------------------ winners / ranking

def _profiles_mid():
    out = []
    for t in range(24):
        m = [3, 5, 8, 13, 20, 31][t % 6]
        n = [1, 2, 7, 30, 101][t % 5]
        k = [m, max(1, m // 3), m - 1, 1][t % 4]
        phi = [0.5, 0.9, 1.0][t % 3]
        out.append((W.mallows(500 + t, n, m, k, phi, W.permutation(t, m)), m))
    return out


@pytest.mark.parametrize("case", range(24))
def test_winner_and_ranking_invariants(case):
    r, m = _profiles_mid()[case]
    d = oracle.tally(r, m)
    p = oracle.strongest_paths(d)
    win = oracle.winners(p)
    order, bb = oracle.ranking(p)
    beats = p > p.T
    # strict relation is transitive
    for a, b, c in itertools.permutations(range(m), 3):
        if beats[a, b] and beats[b, c]:
            assert beats[a, c]
    assert win.sum() >= 1
    np.testing.assert_array_equal(win, (bb == 0).astype(np.int32))
    np.testing.assert_array_equal(bb, beats.sum(axis=0))
    assert sorted(order.tolist()) == list(range(m))
    where = np.empty(m, int)
    where[order] = np.arange(m)
    for a, b in zip(*np.nonzero(beats)):
        assert where[a] < where[b]  # linear extension
    # winners lie in the Schwartz set (Schulze refines it, Sect. 2.1)
    assert set(np.flatnonzero(win)) <= schwartz_set(d)
    # loser filter of Sect. 4: a heavier incoming than outgoing edge loses
    w = oracle.weights(d)
    for c in range(m):
        if w[:, c].max() > w[c, :].max():
            assert win[c] == 0


@pytest.mark.parametrize("seed", range(8))
def test_condorcet_winner_is_unique_winner(seed):
    m, n = 12, 51
    r = W.mallows(seed, n, m, m, 0.4)  # concentrated around the identity
    d = oracle.tally(r, m)
    cw = [c for c in range(m) if all(d[c, j] > d[j, c] for j in range(m) if j != c)]
    assert len(cw) == 1
    win = oracle.winners(oracle.strongest_paths(d))
    assert np.flatnonzero(win).tolist() == cw


def test_margin_and_winning_votes_agree_on_full_rankings():
    for seed in range(10):
        m, n = 9, 20 + seed
        r = W.mallows(seed, n, m, m, 0.95, W.permutation(seed, m))
        d = oracle.tally(r, m)
        pw = oracle.closure(oracle.weights(d))
        pm = oracle.closure(oracle.weights_margin(d))
        np.testing.assert_array_equal(oracle.winners(pw), oracle.winners(pm))
        np.testing.assert_array_equal(oracle.ranking(pw)[1], oracle.ranking(pm)[1])


def test_relabeling_commutes():
    r = W.mallows(3, 60, 15, 6, 0.8, W.permutation(3, 15))
    m = 15
    pi = np.random.Generator(np.random.PCG64(3)).permutation(m).astype(np.int32)
    d = oracle.tally(r, m)
    d2 = oracle.tally(pi[r], m)
    inv = np.argsort(pi)
    np.testing.assert_array_equal(d2, d[np.ix_(inv, inv)])
    p, p2 = oracle.strongest_paths(d), oracle.strongest_paths(d2)
    np.testing.assert_array_equal(p2, p[np.ix_(inv, inv)])
    np.testing.assert_array_equal(oracle.winners(p2), oracle.winners(p)[inv])
    np.testing.assert_array_equal(oracle.ranking(p2)[1], oracle.ranking(p)[1][inv])


# ------------------------------------------- NL-hardness family

@pytest.mark.parametrize("seed", range(40))
def test_nl_reduction_family(seed):
    """a is the unique Schulze winner iff b is reachable from a (Sect. 3)."""
    rs = np.random.Generator(np.random.PCG64(seed))
    nv = int(rs.integers(2, 7))
    edges = random_digraph(rs, nv, float(rs.uniform(0.15, 0.6)))
    a, b = (int(x) for x in rs.choice(nv, 2, replace=False))
    mu = nl_reduction(nv, edges, a, b)
    win = oracle.winners(oracle.strongest_paths(mu))
    adj = {}
    for u, v in edges:
        adj.setdefault(u, []).append(v)
    if reachable(adj, a, b):
        assert np.flatnonzero(win).tolist() == [a]
    else:
        assert win[a] == 0


def test_nl_reduction_via_ballots():
    """Same family end to end: McGarvey ballots -> tally -> closure."""
    rs = np.random.Generator(np.random.PCG64(99))
    hits = 0
    for t in range(6):
        nv = 4
        edges = random_digraph(rs, nv, 0.4)
        a, b = 0, 3
        mu = nl_reduction(nv, edges, a, b)
        ballots = mcgarvey_ballots(mu)
        d = oracle.tally(ballots, mu.shape[0])
        np.testing.assert_array_equal(oracle.weights_margin(d), mu)
        win = oracle.winners(oracle.strongest_paths(d))
        adj = {}
        for u, v in edges:
            adj.setdefault(u, []).append(v)
        if reachable(adj, a, b):
            hits += 1
            assert np.flatnonzero(win).tolist() == [a]
        else:
            assert win[a] == 0


# ------------------------------------------------ degenerate inputs

def test_degenerate_inputs():
    for m in (1, 2, 5):
        for r in (np.zeros((0, m), np.int32), np.zeros((4, 0), np.int32)):
            d, p, win, order, bb = oracle.schulze(r, m)
            assert not d.any() and not p.any()
            assert win.tolist() == [1] * m
            assert order.tolist() == list(range(m))
    d, p, win, order, bb = oracle.schulze(np.array([[0]], np.int32), 1)
    assert win.tolist() == [1] and order.tolist() == [0]
    # all voters identical: unique winner ballot[0]; ranking = ballot then the rest by id
    ballot = np.array([4, 1, 6], np.int32)
    r = np.tile(ballot, (9, 1))
    d, p, win, order, bb = oracle.schulze(r, 8)
    assert np.flatnonzero(win).tolist() == [4]
    assert order.tolist() == [4, 1, 6, 0, 2, 3, 5, 7]


# ----------------------------------------------- weak orders, position form

def test_tally_positions_hand_derived():
    """Three weak orders over (a, b, c, d): a ~ b > c > d; all tied;
    d > b ~ c > a. A tied pair counts for neither candidate (Sect. 2.1)."""
    pos = np.array([[0, 0, 1, 2], [0, 0, 0, 0], [5, 1, 1, 0]], np.int32)
    want = np.zeros((4, 4), np.int32)
    for i, j in [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3),   # first ballot
                 (3, 1), (3, 2), (3, 0), (1, 0), (2, 0)]:  # third ballot
        want[i, j] += 1
    np.testing.assert_array_equal(oracle.tally_positions(pos), want)


@pytest.mark.parametrize("seed", range(4))
def test_tally_positions_equals_order_form(seed):
    """Order-form ballots (unlisted candidates at position k) give the same
    counts through the position form as through the order-form tally."""
    m, n, k = 11, 40, 6
    r = W.mallows(seed, n, m, k, 0.8, W.permutation(seed, m))
    pos = np.full((n, m), k, np.int32)
    for v in range(n):
        pos[v, r[v]] = np.arange(k)
    np.testing.assert_array_equal(oracle.tally_positions(pos), oracle.tally(r, m))


@pytest.mark.parametrize("seed", range(6))
def test_tally_positions_tie_splitting(seed):
    """Breaking one tie (i ~ j on ballot v) both ways: d(i ahead) + d(j
    ahead) = 2 d(tied) + e_ij + e_ji, every other count unchanged."""
    rs = np.random.Generator(np.random.PCG64(seed))
    m, n = 8, 25
    pos = rs.integers(0, 4, size=(n, m)).astype(np.int32)  # many ties
    v = int(rs.integers(0, n))
    pos[v] = rs.permutation(m)  # ballot v: strict except candidates 1 ~ 5
    pos[v, 5] = pos[v, 1]
    base = oracle.tally_positions(pos)
    p1, p2 = 2 * pos, 2 * pos
    p1[v, 5] += 1  # 1 ahead of 5, every other relation of ballot v kept
    p2[v, 1] += 1  # 5 ahead of 1
    e = np.zeros((m, m), np.int64)
    e[1, 5] = e[5, 1] = 1
    np.testing.assert_array_equal(oracle.tally_positions(p1).astype(np.int64) + oracle.tally_positions(p2),
                                  2 * base.astype(np.int64) + e)


def test_tally_positions_rejects_out_of_range():
    with pytest.raises(oracle.OracleError):
        oracle.tally_positions(np.array([[0, 65535]], np.int32))
    with pytest.raises(oracle.OracleError):
        oracle.tally_positions(np.array([[-1, 0]], np.int32))


# ------------------------------------- top-k ranking by iterated removal

def _levels_brute_force(d, k_top, margin=False):
    """Levels from the definition: brute-force widest paths (simple-path
    enumeration) on the weights of the remaining candidates, winners by
    Sect. 2.1, removed, repeated."""
    d = np.asarray(d, np.int64)
    m = d.shape[0]
    level = np.zeros(m, np.int32)
    t = placed = 0
    while placed < min(m, k_top):
        rem = np.flatnonzero(level == 0)
        ds = d[np.ix_(rem, rem)]
        w = np.where(ds > ds.T, ds - ds.T if margin else ds, 0)
        np.fill_diagonal(w, 0)
        p = brute_force_widths(w)
        t += 1
        for a, c in enumerate(rem):
            if all(p[a, b] >= p[b, a] for b in range(len(rem)) if b != a):
                level[c] = t
                placed += 1
    return level, t


@pytest.mark.parametrize("seed", range(30))
def test_ranking_iterated_matches_brute_force(seed):
    rs = np.random.Generator(np.random.PCG64(500 + seed))
    m = int(rs.integers(2, 8))
    n = int(rs.integers(1, 12))
    k = int(rs.integers(1, m + 1))
    r = W.mallows(700 + seed, n, m, k, 0.7 + 0.3 * rs.random(), W.permutation(seed, m))
    d = oracle.tally(r, m)
    for k_top in (1, 2, m):
        for margin in (False, True):
            got = oracle.ranking_iterated(d, k_top, margin)
            want = _levels_brute_force(d, k_top, margin)
            np.testing.assert_array_equal(got[0], want[0])
            assert got[1] == want[1]


def test_ranking_iterated_identical_voters_and_fig1():
    """Identical full ballots: one candidate per level, in ballot order. Fig. 1:
    a alone on the first level (the paper's winner)."""
    m = 9
    ballot = np.random.Generator(np.random.PCG64(1)).permutation(m).astype(np.int32)
    d = oracle.tally(np.tile(ballot, (5, 1)), m)
    level, nl = oracle.ranking_iterated(d)
    assert nl == m
    np.testing.assert_array_equal(level[ballot], np.arange(1, m + 1))
    _, mu, _, win = fig1()
    level, _ = oracle.ranking_iterated(oracle.tally(mcgarvey_ballots(mu), 4), 1)
    assert np.flatnonzero(level == 1).tolist() == win
    assert np.count_nonzero(level) == 1


# ---------------------------- the paper's vertex-centric winners algorithm

@pytest.mark.parametrize("seed", range(40))
def test_pregel_winners_match_closure(seed):
    """Alg. 1-4 (Sect. 4) find exactly the winners of the widest-path
    definition (Sect. 2.1), on tallies (both edge weights) and on random
    weighted digraphs with ties and 2-cycles; every while-loop iteration
    decides at least one vertex."""
    rs = np.random.Generator(np.random.PCG64(900 + seed))
    m = int(rs.integers(1, 30))
    r = W.mallows(900 + seed, int(rs.integers(1, 50)), m, int(rs.integers(1, m + 1)), 0.5 + 0.5 * rs.random(),
                  W.permutation(seed, m))
    d = oracle.tally(r, m)
    g = rs.integers(1, int(rs.integers(1, 6)) + 1, size=(m, m)).astype(np.int32) * (rs.random((m, m)) < rs.random())
    np.fill_diagonal(g, 0)
    for w in (oracle.weights(d), oracle.weights_margin(d), g.astype(np.int32)):
        win, it, _ = oracle.winners_pregel(w)
        np.testing.assert_array_equal(win, oracle.winners(oracle.closure(w)))
        assert it <= m


def test_pregel_fig1_and_nl_family():
    """Fig. 1: a alone, in one iteration. The NL-hardness family of Sect. 3:
    a is the unique winner iff b is reachable from a."""
    _, mu, _, win = fig1()
    got, it, _ = oracle.winners_pregel(mu)
    assert np.flatnonzero(got).tolist() == win and it == 1
    for seed in range(30):
        rs = np.random.Generator(np.random.PCG64(300 + seed))
        nv = int(rs.integers(2, 7))
        edges = random_digraph(rs, nv, float(rs.uniform(0.15, 0.6)))
        a, b = (int(x) for x in rs.choice(nv, 2, replace=False))
        mu = nl_reduction(nv, edges, a, b)
        got, _, _ = oracle.winners_pregel(oracle.weights(mu))
        adj = {}
        for u, v in edges:
            adj.setdefault(u, []).append(v)
        if reachable(adj, a, b):
            assert np.flatnonzero(got).tolist() == [a]
        else:
            assert got[a] == 0
