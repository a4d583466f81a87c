"""Batched elections (one persistent launch) against the oracle, election by
election, bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

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


def _mixed_elections(seed=3):
    """Uneven elections: tiny to m = 330, n from 0 to 4000, full and top-k,
    Mallows and impartial culture, plus degenerate ones."""
    rs = np.random.Generator(np.random.PCG64(seed))
    out = []
    sizes = [1, 2, 3, 8, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 257, 300, 330]
    for t, m in enumerate(sizes):
        n = int(rs.integers(1, 4000)) if t % 5 else int(rs.integers(1, 60))
        k = [m, max(0, m - 1), max(1, m // 3), 1][t % 4]
        if t % 2:
            r = W.impartial(100 + t, n, m, k)
        else:
            r = W.mallows(100 + t, n, m, k, float(rs.uniform(0.5, 1.0)), W.permutation(t, m))
        out.append((r, m))
    out.append((np.zeros((0, 5), np.int32), 5))  # no ballots
    out.append((np.zeros((7, 0), np.int32), 4))  # empty ballots
    out.append((np.tile(np.array([4, 1, 6], np.int32), (9, 1)), 8))  # all voters identical
    return out


def _pack(elections):
    n = np.array([r.shape[0] for r, _ in elections], np.int32)
    k = np.array([r.shape[1] for r, _ in elections], np.int32)
    m = np.array([mm for _, mm in elections], np.int32)
    flat = np.concatenate([r.reshape(-1) for r, _ in elections]).astype(np.int32) if len(elections) else \
        np.zeros(0, np.int32)
    return n, m, k, flat


def _check(b, elections, outs):
    d, p, win, order, bb = (t.cpu().numpy() if t is not None else None for t in outs)
    for e, (r, m) in enumerate(elections):
        mo, vo = int(b.mat_off[e]), int(b.vec_off[e])
        dw, pw, ww, ow, bw = oracle.schulze(r, m)
        if d is not None:
            np.testing.assert_array_equal(d[mo:mo + m * m].reshape(m, m), dw, err_msg=f"d of election {e}")
        if p is not None:
            np.testing.assert_array_equal(p[mo:mo + m * m].reshape(m, m), pw, err_msg=f"p of election {e}")
        np.testing.assert_array_equal(win[vo:vo + m], ww, err_msg=f"winners of election {e}")
        np.testing.assert_array_equal(order[vo:vo + m], ow, err_msg=f"order of election {e}")
        np.testing.assert_array_equal(bb[vo:vo + m], bw, err_msg=f"beaten_by of election {e}")


def _outputs(b, with_matrices=True):
    z = lambda size: torch.full((max(1, size),), -3, dtype=torch.int32, device="cuda")
    return (z(b.mat_elems) if with_matrices else None, z(b.mat_elems) if with_matrices else None,
            z(b.vec_elems), z(b.vec_elems), z(b.vec_elems))


@pytest.mark.parametrize("tally_policy,order_policy", [(0, 0), (1, 0), (0, 1)])
def test_batch_matches_oracle(tally_policy, order_policy):
    els = _mixed_elections()
    n, m, k, flat = _pack(els)
    b = S.SchulzeBatch(n, m, k)
    b.set_schedule(tally_policy, order_policy)
    ranks = torch.from_numpy(flat).cuda() if flat.size else torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = _outputs(b)
    b.run(ranks, *outs)
    torch.cuda.synchronize()
    _check(b, els, outs)


def test_batch_without_matrices_and_int32_counts():
    """More than 32767 ballots in one election selects the int32 closure; d
    and p are not requested."""
    els = [(W.impartial(5, 40000, 20, 20), 20), (W.mallows(6, 300, 90, 30, 0.8, W.permutation(6, 90)), 90)]
    n, m, k, flat = _pack(els)
    b = S.SchulzeBatch(n, m, k)
    outs = _outputs(b, with_matrices=False)
    b.run(torch.from_numpy(flat).cuda(), *outs)
    torch.cuda.synchronize()
    _check(b, els, outs)


def test_batch_workload_sample_and_graph_replay():
    """A sample of the mixed workload (m ~ U[8,512], n ~ U[50,5000]); the run is
    captured in a CUDA graph and replayed on new ballots of the same shape."""
    bw = W.batch_mixed(E=24, seed=77)
    els = [(bw.election(e).ranks, int(bw.m[e])) for e in range(bw.E)]
    b = S.SchulzeBatch(bw.n, bw.m, bw.k)
    ranks = torch.from_numpy(bw.ranks).cuda()
    outs = _outputs(b)
    b.run(ranks, *outs)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run(ranks, *outs)
    for t in outs:
        t.fill_(-5)
    g.replay()
    torch.cuda.synchronize()
    _check(b, els, outs)
    # new ballots of the same shapes, copied into the captured buffer: replay again
    for e in range(bw.E):
        r = bw.election(e).ranks
        r[:] = W.impartial(900 + e, r.shape[0], int(bw.m[e]), r.shape[1])
    ranks.copy_(torch.from_numpy(bw.ranks))
    g.replay()
    torch.cuda.synchronize()
    _check(b, [(bw.election(e).ranks, int(bw.m[e])) for e in range(bw.E)], outs)


def test_batch_autotune_keeps_results_exact(tmp_path):
    """The autotuner picks ballots per tally step for every m-bucket of the
    batch and the election order; the cached choices are reused by a second
    call, and the tuned plan stays exact."""
    bw = W.batch_mixed(E=40, seed=5, m_range=(8, 700), n_range=(50, 800))
    b = S.SchulzeBatch(bw.n, bw.m, bw.k)
    ranks = torch.from_numpy(bw.ranks).cuda()
    cache = str(tmp_path / "autotune.txt")
    t1, o1 = b.autotune(ranks, cache)
    sched1 = b.bucket_schedule()
    assert t1 == 0 and 0 <= o1 <= 1
    used = [q for q, (_, _, e) in enumerate(sched1) if e > 0]
    assert len(used) >= 4
    lines = open(cache).read().splitlines()
    assert sum("bucket<=" in ln for ln in lines) == len(used) and sum("|order|" in ln for ln in lines) == 1
    for q in used:  # every choice is a staging size that fits the bucket
        mx, ch, _ = sched1[q]
        assert ch in (8, 16, 32, 64) and ch * (-(-mx // 64) * 64) * 6 <= 131584 and ch * mx <= 8192
    tiles1 = b.bucket_tiles()
    assert all(g in (1, 2, 4) for g in tiles1)
    b2 = S.SchulzeBatch(bw.n, bw.m, bw.k)
    t2, o2 = b2.autotune(ranks, cache)  # a new plan of the same batch reads the cache
    assert (t1, o1) == (t2, o2) and b2.bucket_schedule() == sched1 and b2.bucket_tiles() == tiles1
    assert open(cache).read().splitlines() == lines  # nothing re-timed
    outs = _outputs(b)
    b.run(ranks, *outs)
    torch.cuda.synchronize()
    _check(b, [(bw.election(e).ranks, int(bw.m[e])) for e in range(bw.E)], outs)


def test_batch_every_bucket_schedule_is_exact():
    """Every ballots-per-step size each m-bucket accepts (8 to 64 where the
    position rows fit) and every number of tile groups per tally tile (1, 2,
    4) gives the oracle's results; sizes that do not fit, and other group
    counts, are refused."""
    els = _mixed_elections(seed=8) + [(W.mallows(41, 900, 700, 700, 0.9, W.permutation(41, 700)), 700),
                                      (W.impartial(42, 300, 1000, 60), 1000)]
    n, m, k, flat = _pack(els)
    b = S.SchulzeBatch(n, m, k)
    ranks = torch.from_numpy(flat).cuda()
    bucket_max = [mx for mx, _, _ in b.bucket_schedule()]
    for chunk in (8, 16, 32, 64):
        fits = [c * (-(-mx // 64) * 64) * 6 <= 131584 and c * mx <= 8192 for mx in bucket_max for c in [chunk]]
        for q, ok in enumerate(fits):
            if ok:
                b.set_bucket_chunk(q, chunk)
            else:
                with pytest.raises(S.SchulzeError):
                    b.set_bucket_chunk(q, chunk)
        outs = _outputs(b)
        b.run(ranks, *outs)
        torch.cuda.synchronize()
        _check(b, els, outs)
    for q in range(5):
        b.set_bucket_chunk(q, 8)
        with pytest.raises(S.SchulzeError):
            b.set_bucket_tiles(q, 3)
    for gpt in (2, 4):
        for q in range(5):
            b.set_bucket_tiles(q, gpt)
        assert b.bucket_tiles() == [gpt] * 5
        outs = _outputs(b)
        b.run(ranks, *outs)
        torch.cuda.synchronize()
        _check(b, els, outs)


def test_batch_from_host_buffers_matches_oracle():
    """schulze_batch_run_host: ballots from host memory (page-locked, and a
    plain numpy array), copied segment by segment beside the computation;
    winners and order on the host equal the oracle's, for every election,
    on two calls in a row and after the schedule changed in between."""
    els = _mixed_elections(seed=11) + [(W.mallows(51, 700, 300, 300, 0.9, W.permutation(51, 300)), 300)]
    n, m, k, flat = _pack(els)
    b = S.SchulzeBatch(n, m, k)
    pinned = torch.from_numpy(flat).pin_memory() if flat.size else torch.zeros(1, dtype=torch.int32)
    win1, ord1 = b.run_host(pinned)
    b.set_schedule(1, 1)  # eight ballots per step, the caller's order
    win2, ord2 = b.run_host(flat if flat.size else np.zeros(1, np.int32))
    for e, (r, mm) in enumerate(els):
        vo = int(b.vec_off[e])
        _, _, ww, ow, _ = oracle.schulze(r, mm)
        for win, order, what in ((win1, ord1, "pinned"), (win2, ord2, "pageable")):
            np.testing.assert_array_equal(win[vo:vo + mm], ww, err_msg=f"{what} winners of election {e}")
            np.testing.assert_array_equal(order[vo:vo + mm], ow, err_msg=f"{what} order of election {e}")


def test_batch_host_wait_limit_returns_and_recovers():
    """schulze_batch_run_host's bounded wait for a segment's arrival mark:
    with the context's wait limit at one clock cycle (and about 8 MB of
    ballots per segment, so the first marks come long after the first CTAs
    look) the call still returns, the status word holds OK or
    SCHULZE_ETIMEOUT, and the next call at the normal limit is exact."""
    ctx = S.context()
    assert ctx.status() == S.OK
    els = [(W.impartial(300 + e, 4000, 64, 64), 64) for e in range(64)]  # 64 x 1 MB of ballots
    n, m, k, flat = _pack(els)
    b = S.SchulzeBatch(n, m, k, ctx=ctx)
    pinned = torch.from_numpy(flat).pin_memory()
    try:
        ctx.set_wait_limit(1)
        b.run_host(pinned)
        assert ctx.status() in (S.OK, S.ETIMEOUT)
    finally:
        ctx.set_wait_limit(4_000_000_000)
    win, order = b.run_host(pinned)
    assert ctx.status() == S.OK
    for e, (r, mm) in enumerate(els[:8]):
        vo = int(b.vec_off[e])
        _, _, ww, ow, _ = oracle.schulze(r, mm)
        np.testing.assert_array_equal(win[vo:vo + mm], ww, err_msg=f"winners of election {e}")
        np.testing.assert_array_equal(order[vo:vo + mm], ow, err_msg=f"order of election {e}")


def test_batch_reports_bad_ballots():
    ctx = S.context()
    assert ctx.status() == S.OK
    els = [(np.array([[0, 1, 2], [2, 2, 0]], np.int32), 3)]
    n, m, k, flat = _pack(els)
    b = S.SchulzeBatch(n, m, k)
    b.run(torch.from_numpy(flat).cuda(), *_outputs(b))
    assert ctx.status() == S.EDATA
