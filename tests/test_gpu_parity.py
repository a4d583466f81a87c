"""CUDA path against the CPU oracle, element by element (bit-exact: every
quantity is an integer)."""
import os

import numpy as np
import pytest
import torch

import oracle
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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def eq(a, b, what=""):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    bad = np.argwhere(a != b)
    assert bad.size == 0, f"{what}: {len(bad)} mismatches, first {bad[:5].tolist()} " \
                          f"gpu={a[tuple(bad[0])]} oracle={b[tuple(bad[0])]}"


# --------------------------------------------------------- paper pins

@pytest.mark.parametrize("flags", [1, 2])
def test_fig1_table_on_gpu(flags):
    _, mu, p_paper, win = fig1()
    p = S.schulze_strongest_paths(cu(mu), bound=12, flags=flags)
    eq(host(p), p_paper, "fig1 widths")
    assert np.flatnonzero(host(S.schulze_winners(p))).tolist() == win


def test_fig1_mcgarvey_on_gpu():
    _, mu, p_paper, _ = fig1()
    ballots = mcgarvey_ballots(mu)
    out = S.schulze_run(cu(ballots), 4)
    d, p, win, order, bb = oracle.schulze(ballots, 4)
    eq(host(out["d"]), d)
    eq(host(out["p"]), p)
    assert host(out["order"]).tolist() == [0, 3, 1, 2]
    assert host(out["beaten_by"]).tolist() == [0, 2, 3, 1]


def test_topk_tie_counterexample_on_gpu():
    g = topk_tie_counterexample()
    for flags in (S.F_TALLY_DENSE, S.F_TALLY_SPARSE, S.F_TALLY_SPARSE | S.F_TALLY_GROUPED):
        out = S.schulze_run(cu(g["ballots"]), g["m"], flags=flags)
        eq(host(out["d"]), g["d"])
        eq(host(out["p"]), g["p"])
        assert np.flatnonzero(host(out["winners"])).tolist() == g["winners"]
        assert host(out["order"]).tolist() == g["ranking"]
        assert host(out["beaten_by"]).tolist() == g["beaten_by"]


# ------------------------------------------------------------- tally

TALLY_CASES = []
for m in (1, 2, 3, 7, 31, 32, 33, 63, 64, 65, 127, 129, 300):
    for n in (0, 1, 2, 37, 513):
        for k in sorted({0, 1, max(0, m - 1), m, m // 2}):
            TALLY_CASES.append((m, n, k))


@pytest.mark.parametrize("m,n,k", TALLY_CASES)
def test_tally_dense_and_sparse(m, n, k):
    seed = m * 1000 + n * 10 + k
    r = W.mallows(seed, n, m, k, 0.85, W.permutation(seed, m)) if k else np.zeros((n, 0), np.int32)
    want = oracle.tally(r, m)
    for flags in (S.F_TALLY_DENSE, S.F_TALLY_SPARSE, S.F_TALLY_SPARSE | S.F_TALLY_GROUPED, 0):
        eq(host(S.schulze_tally(cu(r), m, flags=flags)), want, f"tally flags={flags}")


@pytest.mark.parametrize("m,n,k,phi", [(4096, 3000, 50, 0.9), (1000, 777, 20, 0.97), (1000, 3000, 100, 0.9),
                                       (600, 2000, 256, 0.995),
                                       (256, 4000, 5, 1.0), (257, 4000, 5, 1.0), (5003, 1500, 3, 0.5)])
def test_tally_compact_and_grouped_agree(m, n, k, phi):
    """Top-k ballots over few listed candidates (the compact pair count:
    a lane per ballot up to 64 entries, a warp per ballot beyond) and over
    many (the grouped one), both forms forced, against the oracle; 256
    listed candidates is the largest compact case, 257 the smallest grouped
    one."""
    r = W.mallows(m + n + k, n, m, k, phi, W.permutation(m + k, m))
    want = oracle.tally(r, m)
    for flags in (S.F_TALLY_SPARSE, S.F_TALLY_SPARSE | S.F_TALLY_GROUPED):
        eq(host(S.schulze_tally(cu(r), m, flags=flags)), want, f"tally flags={flags}")


@pytest.mark.parametrize("k", [1, 2, 16, 31, 32, 33, 47, 63, 64, 65])
def test_tally_compact_ballot_lengths(k):
    """The compact pair count packs the rows of each ballot's triangles two
    to an atomic (p < q < 32 and 32 <= p < q): every ballot length around
    those edges, against the oracle."""
    m, n = 220, 1500
    r = W.mallows(900 + k, n, m, k, 0.9, W.permutation(901 + k, m))
    assert len(np.unique(r)) <= 256
    eq(host(S.schulze_tally(cu(r), m, flags=S.F_TALLY_SPARSE)), oracle.tally(r, m), f"k={k}")


def test_tally_compact_many_ballots_per_warp():
    """Each warp of the compact pair count takes many ballots in turn from
    its slice (ids and slots fetched ahead): the whole tally against the
    oracle."""
    m, n, k = 300, 60000, 8
    r = W.mallows(911, n, m, k, 0.9, W.permutation(912, m))
    assert len(np.unique(r)) <= 256
    eq(host(S.schulze_tally(cu(r), m, flags=S.F_TALLY_SPARSE)), oracle.tally(r, m), "many ballots")


def test_tally_compact_wide_counters():
    """More ballots per slice than 16-bit counters hold: the compact pair
    count switches to 32-bit counters. Sampled entries against the
    definition, all row and column sums against their closed forms."""
    m, n, k = 180, 10_500_000, 3
    r = W.mallows(77, n, m, k, 0.7, W.permutation(78, m))
    d = host(S.schulze_tally(cu(r), m, flags=S.F_TALLY_SPARSE))
    listed = np.unique(r)
    rs = np.random.Generator(np.random.PCG64(3))
    for _ in range(12):
        i, j = (int(x) for x in rs.choice(listed, 2, replace=False))
        assert d[i, j] == oracle.tally_entry(r, m, i, j)
    _check_row_col_sums(r, m, d)


def test_tally_many_ballots_chunked():
    """More than 65536 ballots: dense path accumulates chunks, sparse path
    switches to 32-bit counters."""
    m, n = 40, 70001
    r = W.impartial(5, n, m, m)
    want = oracle.tally(r, m)
    eq(host(S.schulze_tally(cu(r), m, flags=S.F_TALLY_DENSE)), want, "dense chunks")
    r2 = W.mallows(6, n, 300, 9, 0.9, W.permutation(6, 300))
    eq(host(S.schulze_tally(cu(r2), 300, flags=S.F_TALLY_SPARSE)), oracle.tally(r2, 300), "sparse int32")


def test_tally_column_split():
    """Rows of d wider than the shared-memory budget: column chunks."""
    m, n, k = 26000, 70000, 4
    r = W.impartial(8, n, m, k)
    d = host(S.schulze_tally(cu(r), m, flags=S.F_TALLY_SPARSE))
    rs = np.random.Generator(np.random.PCG64(1))
    for _ in range(40):
        i, j = (int(x) for x in rs.integers(0, m, 2))
        assert d[i, j] == oracle.tally_entry(r, m, i, j)
    # pairs that actually co-occur in ballots
    for v in range(0, n, 7001):
        for a in range(k):
            for b in range(k):
                i, j = int(r[v, a]), int(r[v, b])
                assert d[i, j] == oracle.tally_entry(r, m, i, j)
    _check_row_col_sums(r, m, d)


def test_tally_heavy_rows_beyond_the_accumulators():
    """About 1100 candidates, each on more ballots than one unit of the
    grouped rows kernel counts (S = 822 entries here), at m = 65535, where
    only the first 1024 heavy rows get split-row accumulators: the other
    heavy rows are counted in chunks into the written row. Only the 1100
    are ever listed, so d restricted to them is the tally of the same
    ballots relabelled 0..1099 (checked whole against the oracle), an
    unlisted column holds each row's ballot count, an unlisted row is zero,
    and every row and column sum (taken on the device) meets its closed
    form."""
    m, n, k, core = 65535, 100000, 10, 1100
    ids = W.permutation(41, m)[:core].astype(np.int64)
    small = W.impartial(42, n, core, k)
    r = ids[small].astype(np.int32)
    d = S.schulze_tally(cu(r), m, flags=S.F_TALLY_SPARSE | S.F_TALLY_GROUPED)
    idx = torch.from_numpy(ids).cuda()
    eq(host(d[idx][:, idx]), oracle.tally(small, core), "listed square")
    listed_n = np.bincount(small.reshape(-1), minlength=core)
    unl = np.setdiff1d(np.arange(m), ids)
    rs = np.random.Generator(np.random.PCG64(43))
    for j in rs.choice(unl, 4, replace=False):
        eq(host(d[idx, int(j)]), listed_n, f"unlisted column {j}")
        assert int(host(d[int(j)].abs().sum())) == 0
    rows = np.zeros(m, np.int64)
    cols = np.full(m, n * k, np.int64)
    np.add.at(rows, r.reshape(-1), (m - 1 - np.tile(np.arange(k), n)))
    np.add.at(cols, r.reshape(-1), np.tile(np.arange(k), n) - k)
    eq(host(d.sum(dim=1, dtype=torch.int64)), rows, "row sums")
    eq(host(d.sum(dim=0, dtype=torch.int64)), cols, "column sums")
    del d
    torch.cuda.empty_cache()


def _check_row_col_sums(r, m, d):
    n, k = r.shape
    rows = np.zeros(m, np.int64)
    cols = np.full(m, n * k, np.int64)  # unlisted j has k candidates above it
    np.add.at(rows, r.reshape(-1), (m - 1 - np.tile(np.arange(k), n)))
    np.add.at(cols, r.reshape(-1), np.tile(np.arange(k), n) - k)
    eq(d.sum(axis=1, dtype=np.int64), rows, "row sums")
    eq(d.sum(axis=0, dtype=np.int64), cols, "column sums")


def test_tally_rejects_bad_ids():
    ctx = S.context()
    assert ctx.status() == S.OK
    bad = np.array([[0, 1, 2], [1, 1, 0]], np.int32)
    for flags in (S.F_TALLY_DENSE, S.F_TALLY_SPARSE, S.F_TALLY_SPARSE | S.F_TALLY_GROUPED):
        S.schulze_tally(cu(bad), 4, flags=flags)
        assert ctx.status() == S.EDATA
    out_of_range = np.array([[0, 7, 2]], np.int32)
    for flags in (S.F_TALLY_DENSE, S.F_TALLY_SPARSE, S.F_TALLY_SPARSE | S.F_TALLY_GROUPED):
        S.schulze_tally(cu(out_of_range), 4, flags=flags)
        assert ctx.status() == S.EDATA
    S.schulze_tally(cu(np.array([[3, 1, 2]], np.int32)), 4)
    assert ctx.status() == S.OK


# ----------------------------------------------------------- closure

CLOSURE_M = [1, 2, 3, 5, 63, 64, 65, 127, 128, 129, 200, 257, 511]


@pytest.mark.parametrize("m", CLOSURE_M)
def test_closure_and_extraction(m):
    n = 301
    r = W.mallows(m, n, m, min(m, 17), 0.93, W.permutation(m + 1, m))
    d = oracle.tally(r, m)
    p_want = oracle.strongest_paths(d)
    win_want = oracle.winners(p_want)
    order_want, bb_want = oracle.ranking(p_want)
    dd = cu(d)
    for flags in (S.F_FORCE_S16, S.F_FORCE_S32):
        p = S.schulze_strongest_paths(dd, bound=n, flags=flags)
        eq(host(p), p_want, f"closure m={m} flags={flags}")
    eq(host(S.schulze_winners(p)), win_want, "winners")
    order, bb = S.schulze_ranking(p)
    eq(host(order), order_want, "ranking")
    eq(host(bb), bb_want, "beaten_by")


def test_closure_random_weight_matrices():
    """Arbitrary nonnegative count matrices, including ties and zeros."""
    rs = np.random.Generator(np.random.PCG64(3))
    for m in (7, 70, 190):
        for density in (0.05, 0.5, 1.0):
            d = rs.integers(0, 30000, size=(m, m)).astype(np.int32)
            d[rs.random((m, m)) > density] = 0
            np.fill_diagonal(d, 0)
            want = oracle.strongest_paths(d)
            for flags in (S.F_FORCE_S16, S.F_FORCE_S32):
                eq(host(S.schulze_strongest_paths(cu(d), 30000, flags=flags)), want, f"random m={m}")


@pytest.mark.parametrize("m,cold_frac", [(700, 0.0), (700, 0.6), (1500, 0.9), (1029, 0.3)])
def test_closure_many_rounds_with_edgeless_candidates(m, cold_frac):
    """Candidates without outgoing edges interleaved with the others: the
    relabeling moves them last and their tiles are skipped."""
    rs = np.random.Generator(np.random.PCG64(m))
    d = rs.integers(0, 20000, size=(m, m)).astype(np.int32)
    d[rs.random((m, m)) < 0.5] = 0
    cold = rs.random(m) < cold_frac
    d[cold, :] = 0
    np.fill_diagonal(d, 0)
    want = oracle.strongest_paths(d, nthreads=16)
    for flags in (S.F_FORCE_S16, S.F_FORCE_S32):
        eq(host(S.schulze_strongest_paths(cu(d), 20000, flags=flags)), want, f"m={m} cold={cold_frac}")


@pytest.mark.parametrize("nw", [2, 3, 17, 64, 151, 192, 256])
def test_closure_long_widest_paths(nw):
    """Warm squares whose widest paths are long: a heavy Hamiltonian chain
    through the warm candidates in a shuffled order under light random
    edges, so that p(a, b) for distant a, b needs every edge of the chain.
    The small-square closure then needs about log2(nw) + 1 sweeps."""
    m = 400
    rs = np.random.Generator(np.random.PCG64(5000 + nw))
    warm = rs.permutation(m)[:nw]
    d = np.zeros((m, m), np.int32)
    d[np.ix_(warm, warm)] = rs.integers(0, 100, size=(nw, nw)) * (rs.random((nw, nw)) < 0.3)
    heavy = rs.integers(20000, 30000, size=nw)
    for a in range(nw):  # chain warm[0] -> warm[1] -> ... -> warm[nw - 1] -> warm[0]
        d[warm[a], warm[(a + 1) % nw]] = heavy[a]
    np.fill_diagonal(d, 0)
    want = oracle.strongest_paths(d, nthreads=16)
    for flags in (S.F_FORCE_S16, S.F_FORCE_S32):
        eq(host(S.schulze_strongest_paths(cu(d), 30000, flags=flags)), want, f"nw={nw} flags={flags}")


@pytest.mark.parametrize("nw", [1, 31, 32, 33, 64, 65, 151, 192, 193, 255, 256, 257, 300])
def test_closure_warm_set_sizes(nw):
    """nw candidates with outgoing edges spread over m = 600 ids, the rest
    edgeless: the cluster closure takes warm sets up to 256 (16-bit) or 192
    (int32) candidates, the persistent kernel the larger ones; cold columns
    come from the product with the closed warm square."""
    m = 600
    rs = np.random.Generator(np.random.PCG64(1000 + nw))
    warm = rs.choice(m, nw, replace=False)
    d = np.zeros((m, m), np.int32)
    d[np.ix_(warm, np.arange(m))] = rs.integers(1, 30000, size=(nw, m)) * (rs.random((nw, m)) < 0.3)
    cold = np.setdiff1d(np.arange(m), warm)
    d[warm, cold[rs.integers(0, cold.size, nw)]] = rs.integers(1, 30000, nw)  # every warm one has an edge
    np.fill_diagonal(d, 0)
    want = oracle.strongest_paths(d, nthreads=16)
    for flags in (S.F_FORCE_S16, S.F_FORCE_S32):
        eq(host(S.schulze_strongest_paths(cu(d), 30000, flags=flags)), want, f"nw={nw} flags={flags}")


def test_closure_large_counts_int32():
    rs = np.random.Generator(np.random.PCG64(4))
    m = 150
    d = rs.integers(0, 2_000_000_000, size=(m, m)).astype(np.int32)
    np.fill_diagonal(d, 0)
    eq(host(S.schulze_strongest_paths(cu(d), 2_000_000_000)), oracle.strongest_paths(d), "int32 counts")


def test_closure_bound_violation_flagged():
    ctx = S.context()
    d = np.array([[0, 40000], [0, 0]], np.int32)
    S.schulze_strongest_paths(cu(d), 30000)
    assert ctx.status() == S.EDATA
    with pytest.raises(S.SchulzeError):
        S.schulze_strongest_paths(cu(d), 40000, flags=S.F_FORCE_S16)
    S.schulze_strongest_paths(cu(d), 40000)
    assert ctx.status() == S.OK


# ------------------------------------------------------- end to end

def test_unaligned_caller_buffers():
    """Caller matrices need only the 4-byte alignment of int32: d and p one
    element past a 16-byte boundary (m a multiple of 4, so aligned buffers
    would take 16-byte row accesses) give the oracle's results through the
    tally's streaming fill, the closure's reads of d and its writes of p."""
    def unaligned(m):
        buf = torch.full((m * m + 1,), -9, dtype=torch.int32, device="cuda")
        t = buf[1:].view(m, m)
        assert t.data_ptr() % 16 != 0 and t.is_contiguous()
        return t
    m, n, k = 300, 2000, 20
    r = W.mallows(77, n, m, k, 0.9, W.permutation(77, m))
    d_o, p_o, win_o, order_o, bb_o = oracle.schulze(r, m)
    d, p = unaligned(m), unaligned(m)
    eq(host(S.schulze_tally(cu(r), m, d=d, flags=S.F_TALLY_SPARSE)), d_o, "compact tally, unaligned d")
    eq(host(S.schulze_tally(cu(r), m, d=d, flags=S.F_TALLY_SPARSE | S.F_TALLY_GROUPED)), d_o, "grouped, unaligned d")
    eq(host(S.schulze_strongest_paths(d, n, p=p)), p_o, "closure, unaligned d and p")
    out = S.schulze_run(cu(r), m, out={"d": unaligned(m), "p": unaligned(m)})
    eq(host(out["d"]), d_o)
    eq(host(out["p"]), p_o)
    eq(host(out["winners"]), win_o)
    eq(host(out["order"]), order_o)
    # a dense square above the cluster kernel's size (persistent closure)
    rs = np.random.Generator(np.random.PCG64(78))
    m = 516
    dd = rs.integers(0, 30000, size=(m, m)).astype(np.int32)
    np.fill_diagonal(dd, 0)
    d = unaligned(m)
    d.copy_(cu(dd))
    want = oracle.strongest_paths(dd, nthreads=NT)
    for flags in (0, S.F_FORCE_S32):
        eq(host(S.schulze_strongest_paths(d, 30000, p=unaligned(m), flags=flags)), want, f"persistent flags={flags}")


@pytest.mark.parametrize("flags", [0, 1])
def test_closure_wait_limit_runs_out_and_recovers(flags):
    """The persistent closure's bounded waits, made to run out (a limit of
    one clock cycle on a square of 11 x 11 tiles, where items wait for the
    tiles of the round before): the call returns, the status word reports
    SCHULZE_ETIMEOUT, and the next call at the normal limit is exact."""
    ctx = S.context()
    assert ctx.status() == S.OK
    rs = np.random.Generator(np.random.PCG64(91 + flags))
    m = 700
    d = rs.integers(0, 30000, size=(m, m)).astype(np.int32)
    np.fill_diagonal(d, 0)
    want = oracle.strongest_paths(d, nthreads=NT)
    dd = cu(d)
    try:
        ctx.set_wait_limit(1)
        S.schulze_strongest_paths(dd, 30000, flags=flags, ctx=ctx)
        assert ctx.status() == S.ETIMEOUT
    finally:
        ctx.set_wait_limit(4_000_000_000)
    eq(host(S.schulze_strongest_paths(dd, 30000, flags=flags, ctx=ctx)), want, "after a timed-out call")
    assert ctx.status() == S.OK


CANARY = -0x5A5A5A5B  # 0xA5A5A5A5
PAD = 64  # canary words before and after each buffer (256 bytes: the buffer itself stays 16-byte aligned)


def guarded(shape, dtype=torch.int32):
    """An output buffer with canary words on both sides; returns (view, check)
    where check() asserts that no canary word changed."""
    n = int(np.prod(shape))
    fill = CANARY if dtype == torch.int32 else float("nan")
    buf = torch.full((n + 2 * PAD,), fill, dtype=dtype, device="cuda")

    def check(what=""):
        torch.cuda.synchronize()
        edge = torch.cat([buf[:PAD], buf[PAD + n:]]).cpu()
        ok = (edge == CANARY).all() if dtype == torch.int32 else torch.isnan(edge).all()
        assert bool(ok), f"canary overwritten around {what} {tuple(shape)}"
    return buf[PAD:PAD + n].view(*shape), check


@pytest.mark.parametrize("m,n,k", [(1, 5, 1), (63, 300, 63), (65, 500, 20), (200, 1000, 12), (300, 900, 300),
                                   (517, 800, 40), (1029, 400, 30)])
def test_outputs_stay_within_their_buffers(m, n, k):
    """A stand-in for a device memory checker: canary words before and after
    every output buffer must survive every call that writes it (the whole
    path, each tally form, both closures and margin weights, winners,
    ranking, weak-order tally, the allocation-free closure, the learned
    calls), and the outputs still equal the oracle's."""
    r = W.mallows(m * 3 + k, n, m, k, 0.9, W.permutation(m, m))
    d_o, p_o, win_o, order_o, bb_o = oracle.schulze(r, m)
    rr = cu(r)
    outs = {key: guarded(shape) for key, shape in (("d", (m, m)), ("p", (m, m)), ("winners", (m,)),
                                                   ("order", (m,)), ("beaten_by", (m,)))}
    S.schulze_run(rr, m, out={key: v for key, (v, _) in outs.items()})
    for key, want in (("d", d_o), ("p", p_o), ("winners", win_o), ("order", order_o), ("beaten_by", bb_o)):
        outs[key][1](f"schulze_run {key}")
        eq(host(outs[key][0]), want, key)
    for flags in (S.F_TALLY_DENSE, S.F_TALLY_SPARSE, S.F_TALLY_SPARSE | S.F_TALLY_GROUPED):
        d, chk = guarded((m, m))
        S.schulze_tally(rr, m, d=d, flags=flags)
        chk(f"tally {flags}")
        eq(host(d), d_o, f"tally {flags}")
    dd = cu(d_o)
    for flags in (0, S.F_FORCE_S32, S.F_MARGIN):
        p, chk = guarded((m, m))
        S.schulze_strongest_paths(dd, n, p=p, flags=flags)
        chk(f"strongest_paths {flags}")
        if not flags & S.F_MARGIN:
            eq(host(p), p_o, f"closure {flags}")
    pp = cu(p_o)
    w, chk = guarded((m,))
    S.schulze_winners(pp, winners=w)
    chk("winners")
    o, chk_o = guarded((m,))
    b, chk_b = guarded((m,))
    S.schulze_ranking(pp, order=o, beaten_by=b)
    chk_o("order"), chk_b("beaten_by")
    eq(host(o), order_o, "order")
    pos = np.full((n, m), k, np.int32)
    for v in range(n):
        pos[v, r[v]] = np.arange(k)
    d, chk = guarded((m, m))
    S.schulze_tally_positions(cu(pos), d=d)
    chk("tally_positions")
    eq(host(d), d_o, "positions")
    if m <= 1024:
        p, chk = guarded((m, m))
        S.schulze_strongest_paths_static(dd, n, p=p)
        chk("strongest_paths_static")
        eq(host(p), p_o, "static")
    f, chk = guarded((m, 16), torch.float32)
    S.schulze_features(dd, n, feat=f)
    chk("features")
    w, chk = guarded((m,))
    S.schulze_winners_fast(dd, n, None, top=4, winners=w)
    chk("winners_fast")
    eq(host(w), win_o, "winners_fast")


def test_degenerate_elections():
    for m in (1, 2, 9):
        for r in (np.zeros((0, m), np.int32), np.zeros((5, 0), np.int32)):
            out = S.schulze_run(cu(r) if r.size else torch.zeros(r.shape, dtype=torch.int32, device="cuda"), m)
            assert not host(out["d"]).any() and not host(out["p"]).any()
            assert host(out["winners"]).tolist() == [1] * m
            assert host(out["order"]).tolist() == list(range(m))
    r = np.tile(np.array([4, 1, 6], np.int32), (9, 1))
    out = S.schulze_run(cu(r), 8)
    assert np.flatnonzero(host(out["winners"])).tolist() == [4]
    assert host(out["order"]).tolist() == [4, 1, 6, 0, 2, 3, 5, 7]


def test_small_mallows_workload_end_to_end():
    e = W.small_mallows()
    out = S.schulze_run(cu(e.ranks), e.m)
    d, p, win, order, bb = oracle.schulze(e.ranks, e.m)
    eq(host(out["d"]), d)
    eq(host(out["p"]), p)
    eq(host(out["winners"]), win)
    eq(host(out["order"]), order)
    eq(host(out["beaten_by"]), bb)


def test_host_buffers_path_matches_device_path():
    e = W.large_topk(seed=9, n=2000, m=700, k=30)
    win, order = S.schulze_run_host(e.ranks, e.m)
    _, p, win_o, order_o, _ = oracle.schulze(e.ranks, e.m, nthreads=8)
    eq(win, win_o)
    eq(order, order_o)
    with pytest.raises(S.SchulzeError):
        S.schulze_run_host(np.array([[0, 0]], np.int32), 3)


NT = os.cpu_count() or 1


def _sampled_closure_checks(w, p_gpu, rows, wT=None):
    """Rows and columns of p by max-min Dijkstra (columns on the transposed
    graph, whose rows are the columns of p)."""
    wT = np.ascontiguousarray(w.T) if wT is None else wT
    eq(p_gpu[rows], oracle.widest_many(w, rows, nthreads=NT), f"rows {rows}")
    eq(p_gpu[:, rows].T, oracle.widest_many(wT, rows, nthreads=NT), f"columns {rows}")


def _exact_winners_and_beaten_by(w, win_gpu, bb_gpu, seed, extra=64, wT=None):
    """Completeness of the winner set on a profile too large for the oracle's
    whole closure (Sect. 2.1). One reported winner c gets its row and column
    of p by max-min Dijkstra: it must beat or tie everyone. Any other winner y
    would need p(y, c) >= p(c, y) and, c being a winner, p(c, y) >= p(y, c):
    a tie. So the exact winner set is c plus the candidates tied with c that
    no one beats, each checked by its own row and column; it must equal the
    reported set. beaten_by is then checked exactly on every candidate
    reported with beaten_by <= 1 and on `extra` seeded others."""
    m = w.shape[0]
    wT = np.ascontiguousarray(w.T) if wT is None else wT
    reported = np.flatnonzero(win_gpu)
    assert reported.size >= 1, "empty winner set"
    c = int(reported[0])
    fc = oracle.widest_many(w, [c], nthreads=1)[0]
    bc = oracle.widest_many(wT, [c], nthreads=1)[0]
    assert np.all(fc >= bc), f"reported winner {c} is beaten"
    tied = np.flatnonzero(fc == bc)
    tied = tied[tied != c]
    assert tied.size <= 512, f"{tied.size} candidates tied with the winner: too many to check one by one"
    exact = {c}
    if tied.size:
        F = oracle.widest_many(w, tied, nthreads=NT)
        B = oracle.widest_many(wT, tied, nthreads=NT)
        exact |= {int(x) for x, f, b in zip(tied, F, B) if np.all(f >= b)}
    assert sorted(exact) == reported.tolist(), f"winner set: reported {reported.tolist()}, exact {sorted(exact)}"
    rs = np.random.Generator(np.random.PCG64(seed))
    check = np.unique(np.concatenate([np.flatnonzero(bb_gpu <= 1), rs.integers(0, m, extra)])).astype(np.int32)
    F = oracle.widest_many(w, check, nthreads=NT)
    B = oracle.widest_many(wT, check, nthreads=NT)
    for x, f, b in zip(check, F, B):
        assert bb_gpu[x] == int(np.sum(b > f)), f"beaten_by[{x}]"
    return len(exact), check.size


def test_large_topk_workload_full_size():
    """m=4096, n=20000, top-50 Mallows(0.9): whole d against the oracle, the
    closure on sampled rows and columns (max-min Dijkstra), every winner
    certified and sampled beaten_by counts recomputed."""
    e = W.large_topk()
    out = S.schulze_run(cu(e.ranks), e.m)
    d = host(out["d"])
    eq(d, oracle.tally(e.ranks, e.m), "tally")
    w = oracle.weights(d)
    p = host(out["p"])
    rs = np.random.Generator(np.random.PCG64(2))
    # the listed candidates: paths between them never leave them (the others
    # have no outgoing edge), so p on A x A is the oracle closure of d[A, A]
    A = np.unique(e.ranks)
    dA = np.ascontiguousarray(d[np.ix_(A, A)])
    eq(p[np.ix_(A, A)], oracle.strongest_paths(dA, nthreads=NT), "closure on the listed candidates")
    # the rest of p, whole: an unlisted candidate is preferred to nobody, so
    # its row is zero, and every unlisted column equals p[., c] of the
    # closure of the listed candidates plus that column (paths into c run
    # through listed candidates only); the oracle's closure over A and eight
    # unlisted columns gives those values, the same in every unlisted column
    cold = np.setdiff1d(np.arange(e.m), A)
    assert cold.size > 0
    eq(p[cold], np.zeros((cold.size, e.m), np.int32), "rows of unlisted candidates")
    C8 = cold[rs.choice(cold.size, min(8, cold.size), replace=False)]
    AC = np.concatenate([A, C8])
    pAC = oracle.strongest_paths(np.ascontiguousarray(d[np.ix_(AC, AC)]), nthreads=NT)
    ucol = pAC[:A.size, A.size]
    for t in range(1, C8.size):
        eq(pAC[:A.size, A.size + t], ucol, "uniform unlisted columns in the oracle closure")
    eq(p[np.ix_(A, cold)], np.repeat(ucol[:, None], cold.size, axis=1), "unlisted columns, listed rows")
    # p is now checked entry by entry: winners, order and beaten_by follow
    # from it by the oracle's own definitions
    eq(host(out["winners"]), oracle.winners(p), "winners")
    order_o, bb_o = oracle.ranking(p)
    eq(host(out["order"]), order_o, "order")
    eq(host(out["beaten_by"]), bb_o, "beaten_by")
    _sampled_closure_checks(w, p, [0, e.m - 1] + rs.integers(0, e.m, 4).tolist() + rs.choice(A, 4).tolist())


def test_huge_pl_workload_full_size():
    """m=16384, n=200000, top-20 Plackett-Luce Zipf(1.1): int32 closure.
    Tally by row/column sums and sampled entries; closure on the
    2048-candidate popular subsample against the oracle closure, and on full-m
    sampled rows by Dijkstra; winners certified."""
    e = W.huge_pl()
    m = e.m
    out = S.schulze_run(cu(e.ranks), m)
    d = host(out["d"])
    _check_row_col_sums(e.ranks, m, d)
    sub = W.popular_subsample(m, 2048)
    for a in range(0, 2048, 97):
        for b in range(3, 2048, 331):
            i, j = int(sub[a]), int(sub[b])
            assert d[i, j] == oracle.tally_entry(e.ranks, m, i, j)
    dS = np.ascontiguousarray(d[np.ix_(sub, sub)])
    pS = S.schulze_strongest_paths(cu(dS), bound=e.n)
    pS_want = oracle.strongest_paths(dS, nthreads=NT)
    eq(host(pS), pS_want, "subsample closure")
    eq(host(S.schulze_winners(pS)), oracle.winners(pS_want), "subsample winners")
    eq(host(S.schulze_ranking(pS)[0]), oracle.ranking(pS_want)[0], "subsample ranking")
    w = oracle.weights(d)
    wT = np.ascontiguousarray(w.T)
    p = host(out["p"])
    _sampled_closure_checks(w, p, [int(sub[0]), int(sub[1]), 5], wT)
    bb = host(out["beaten_by"])
    _exact_winners_and_beaten_by(w, host(out["winners"]), bb, seed=16384, wT=wT)
    order = host(out["order"])
    assert sorted(order.tolist()) == list(range(m))
    assert np.all(np.diff(bb[order]) >= 0)


# ------------------------------------------ margins and weak-order ballots

def test_fig1_margin_closure_on_gpu():
    """Fig. 1 realised by 42 ballots (McGarvey): with margin weights the GPU
    closure of the tally reproduces the printed width table itself."""
    _, mu, p_paper, win = fig1()
    ballots = mcgarvey_ballots(mu)
    d = S.schulze_tally(cu(ballots), 4)
    for flags in (S.F_MARGIN | S.F_FORCE_S16, S.F_MARGIN | S.F_FORCE_S32):
        p = S.schulze_strongest_paths(d, bound=42, flags=flags)
        eq(host(p), p_paper, "fig1 margin widths")
        assert np.flatnonzero(host(S.schulze_winners(p))).tolist() == win


@pytest.mark.parametrize("m", [7, 70, 190, 300])
def test_margin_closure_random(m):
    rs = np.random.Generator(np.random.PCG64(50 + m))
    d = rs.integers(0, 30000, size=(m, m)).astype(np.int32)
    d[rs.random((m, m)) > 0.6] = 0
    np.fill_diagonal(d, 0)
    want = oracle.closure(oracle.weights_margin(d), nthreads=8)
    for flags in (S.F_MARGIN | S.F_FORCE_S16, S.F_MARGIN | S.F_FORCE_S32):
        eq(host(S.schulze_strongest_paths(cu(d), 30000, flags=flags)), want, f"margin m={m}")


@pytest.mark.parametrize("m,n,k", [(700, 2000, 30), (150, 500, 150)])
def test_margin_run_end_to_end(m, n, k):
    """schulze_run with margin weights: top-k ballots with unlisted candidates
    (one uniform cold column) and full rankings, against the oracle."""
    r = W.mallows(m + k, n, m, k, 0.9, W.permutation(m, m))
    out = S.schulze_run(cu(r), m, flags=S.F_MARGIN)
    d = oracle.tally(r, m)
    p = oracle.closure(oracle.weights_margin(d), nthreads=8)
    eq(host(out["p"]), p, "margin p")
    eq(host(out["winners"]), oracle.winners(p), "margin winners")
    order, bb = oracle.ranking(p)
    eq(host(out["order"]), order, "margin order")
    eq(host(out["beaten_by"]), bb, "margin beaten_by")


@pytest.mark.parametrize("m,n,levels", [(1, 5, 1), (5, 40, 2), (65, 300, 4), (150, 700, 20), (300, 100, 300)])
def test_tally_positions_weak_orders(m, n, levels):
    """Weak orders (positions drawn from `levels` values, so ties abound)
    against the oracle's position-form tally."""
    rs = np.random.Generator(np.random.PCG64(m * 7 + n))
    pos = rs.integers(0, levels, size=(n, m)).astype(np.int32)
    eq(host(S.schulze_tally_positions(cu(pos))), oracle.tally_positions(pos), f"weak m={m}")


def test_tally_positions_wide_positions():
    """Positions above 32767 take the 16-bit compare instead of the guard-bit
    count; both against the oracle, with ties."""
    rs = np.random.Generator(np.random.PCG64(11))
    pos = rs.integers(0, 65535, size=(300, 130)).astype(np.int32)
    pos[:, 7] = pos[:, 3]  # ties
    pos[5, :] = 65534
    eq(host(S.schulze_tally_positions(cu(pos))), oracle.tally_positions(pos), "wide positions")
    small = (pos // 2).astype(np.int32)  # below 2^15
    eq(host(S.schulze_tally_positions(cu(small))), oracle.tally_positions(small), "narrow positions")


def test_tally_positions_many_ballots_and_order_form():
    """More ballots than one chunk of position rows; and order-form ballots
    written as positions give the order-form tally."""
    rs = np.random.Generator(np.random.PCG64(9))
    pos = rs.integers(0, 6, size=(70001, 40)).astype(np.int32)
    eq(host(S.schulze_tally_positions(cu(pos))), oracle.tally_positions(pos), "weak chunked")
    m, n, k = 200, 900, 12
    r = W.mallows(4, n, m, k, 0.9, W.permutation(4, m))
    pos = np.full((n, m), k, np.int32)
    for v in range(n):
        pos[v, r[v]] = np.arange(k)
    eq(host(S.schulze_tally_positions(cu(pos))), host(S.schulze_tally(cu(r), m)), "positions vs order form")


def test_tally_rejects_bad_ids_in_long_ballots():
    """Repeated or out-of-range ids anywhere in ballots of 33 to 64
    positions (each lane of the count pass holds two positions): a repeat
    inside the first 32 positions, across the two halves, inside the second
    half, and an out-of-range id in the second half are each reported; the
    clean ballots around them tally as the oracle says."""
    ctx = S.context()
    assert ctx.status() == S.OK
    m, n = 300, 3000
    for k in (33, 50, 64):
        good = W.mallows(600 + k, n, m, k, 0.9)
        S.schulze_tally(cu(good), m, flags=S.F_TALLY_SPARSE)
        assert ctx.status() == S.OK, k
        eq(host(S.schulze_tally(cu(good), m, flags=S.F_TALLY_SPARSE)), oracle.tally(good, m), f"clean k={k}")
        for a, b in ((3, 17), (5, 40), (35, k - 1), (0, 32)):
            if max(a, b) >= k:
                continue
            bad = good.copy()
            bad[n // 2, b] = bad[n // 2, a]
            S.schulze_tally(cu(bad), m, flags=S.F_TALLY_SPARSE)
            assert ctx.status() == S.EDATA, (k, a, b)
        bad = good.copy()
        bad[n - 1, k - 1] = m + 1
        S.schulze_tally(cu(bad), m, flags=S.F_TALLY_SPARSE)
        assert ctx.status() == S.EDATA, k
        S.schulze_tally(cu(good), m, flags=S.F_TALLY_SPARSE)
        assert ctx.status() == S.OK, k


def test_tally_positions_rejects_out_of_range():
    ctx = S.context()
    assert ctx.status() == S.OK
    S.schulze_tally_positions(cu(np.array([[0, 65535, 2]], np.int32)))
    assert ctx.status() == S.EDATA
    S.schulze_tally_positions(cu(np.array([[0, -3, 2]], np.int32)))
    assert ctx.status() == S.EDATA
    S.schulze_tally_positions(cu(np.array([[0, 65534, 2]], np.int32)))
    assert ctx.status() == S.OK


def test_spotify_like_workload_full_size():
    """m=18407, n=15553, top-200 Plackett-Luce Zipf(1.1) (the shape of the
    paper's largest Spotify profile). Tally by row/column sums and sampled
    entries; the closure on the 2048 most popular candidates against the
    oracle closure, and on full-m sampled rows and columns by Dijkstra;
    winners certified."""
    e = W.spotify_like()
    m = e.m
    out = S.schulze_run(cu(e.ranks), m)
    d = host(out["d"])
    _check_row_col_sums(e.ranks, m, d)
    sub = W.spotify_popular(m, 2048)
    for a in range(0, 2048, 211):
        for b in range(5, 2048, 397):
            i, j = int(sub[a]), int(sub[b])
            assert d[i, j] == oracle.tally_entry(e.ranks, m, i, j)
    dS = np.ascontiguousarray(d[np.ix_(sub, sub)])
    pS = S.schulze_strongest_paths(cu(dS), bound=e.n)
    eq(host(pS), oracle.strongest_paths(dS, nthreads=NT), "subsample closure")
    w = oracle.weights(d)
    wT = np.ascontiguousarray(w.T)
    p = host(out["p"])
    _sampled_closure_checks(w, p, [int(sub[0]), int(sub[1000]), m - 1], wT)
    bb = host(out["beaten_by"])
    _exact_winners_and_beaten_by(w, host(out["winners"]), bb, seed=18407, wT=wT)
    order = host(out["order"])
    assert sorted(order.tolist()) == list(range(m))
    assert np.all(np.diff(bb[order]) >= 0)


# ------------------------------------- top-k ranking by iterated removal

@pytest.mark.parametrize("m,n,k,phi,k_top", [(9, 30, 9, 0.9, 9), (70, 400, 70, 0.95, 70), (130, 300, 20, 0.9, 130),
                                             (700, 2000, 30, 0.9, 12), (300, 40, 300, 1.0, 25)])
def test_ranking_iterated(m, n, k, phi, k_top):
    r = W.mallows(m * 3 + n, n, m, k, phi, W.permutation(m + 5, m))
    d = oracle.tally(r, m)
    for margin in (False, True):
        level, nl = S.schulze_ranking_iterated(cu(d), n, k_top, flags=S.F_MARGIN if margin else 0)
        want, want_nl = oracle.ranking_iterated(d, k_top, margin)
        eq(host(level), want, f"levels m={m} margin={margin}")
        assert nl == want_nl


def test_ranking_iterated_degenerate():
    """No ballots: every candidate wins the first level. One candidate."""
    level, nl = S.schulze_ranking_iterated(torch.zeros((5, 5), dtype=torch.int32, device="cuda"), 0, 3)
    assert host(level).tolist() == [1] * 5 and nl == 1
    level, nl = S.schulze_ranking_iterated(torch.zeros((1, 1), dtype=torch.int32, device="cuda"), 0)
    assert host(level).tolist() == [1] and nl == 1


# ---------------------- the paper's vertex-centric algorithm (Alg. 1-4)

@pytest.mark.parametrize("m,n,k,phi", [(1, 3, 1, 1.0), (2, 5, 2, 0.5), (33, 200, 10, 0.9), (130, 400, 130, 0.97),
                                       (700, 2000, 30, 0.9), (300, 50, 300, 1.0)])
def test_winners_propagation_elections(m, n, k, phi):
    """Same winners as the closure, and the same while-loop iterations and
    propagation rounds as the oracle's synchronous simulation."""
    r = W.mallows(m + 2 * n, n, m, k, phi, W.permutation(m + 9, m))
    d = oracle.tally(r, m)
    for margin in (False, True):
        w = oracle.weights_margin(d) if margin else oracle.weights(d)
        win, stats = S.schulze_winners_propagation(cu(d), flags=S.F_MARGIN if margin else 0)
        eq(host(win), oracle.winners(oracle.closure(w, nthreads=8)), f"winners m={m} margin={margin}")
        _, it, rounds = oracle.winners_pregel(w)
        assert stats == [it, rounds]


@pytest.mark.parametrize("seed", range(6))
def test_winners_propagation_random_weights(seed):
    """Arbitrary count matrices with many ties and 2-cycles."""
    rs = np.random.Generator(np.random.PCG64(4000 + seed))
    m = int(rs.integers(20, 200))
    d = rs.integers(0, 6, size=(m, m)).astype(np.int32) * (rs.random((m, m)) < rs.random())
    np.fill_diagonal(d, 0)
    win, stats = S.schulze_winners_propagation(cu(d.astype(np.int32)))
    w = oracle.weights(d)
    eq(host(win), oracle.winners(oracle.closure(w, nthreads=8)), "winners")
    _, it, rounds = oracle.winners_pregel(w)
    assert stats == [it, rounds]
