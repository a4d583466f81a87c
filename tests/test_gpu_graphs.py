"""schulze_run captured as a CUDA graph, and schulze_run_host (which caches
its own graph). Several stages choose on the device among kernel sequences
(compact or grouped tally, the closure's own warm-row pass, cluster or
persistent closure, uniform or general cold columns): the graph holds every
alternative and the kernels whose case it is not return at once. A replay
must give the oracle's results whichever way the device decides, including
when the data of a replay decides differently from the data the graph was
captured on."""
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


def _outs(m, dev):
    return {key: torch.full(shape, -7, dtype=torch.int32, device=dev)
            for key, shape in (("d", (m, m)), ("p", (m, m)), ("winners", (m,)), ("order", (m,)),
                               ("beaten_by", (m,)))}


def _capture(fn):
    """fn() run once on a side stream, then captured; returns the graph."""
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        fn()
    return g


def _check_oracle(ranks, m, out, what):
    d, p, win, order, bb = oracle.schulze(ranks, m, nthreads=8)
    torch.cuda.synchronize()
    for key, want in (("d", d), ("p", p), ("winners", win), ("order", order), ("beaten_by", bb)):
        got = out[key].cpu().numpy()
        bad = np.argwhere(got != want)
        assert bad.size == 0, f"{what} {key}: {len(bad)} mismatches, first {bad[:3].tolist()}"


# (label, ballots, m): each takes a different set of device decisions
def _cases():
    return [
        # few listed candidates: compact tally, tally's warm flags, cluster
        # closure, uniform cold columns
        ("compact", W.mallows(101, 3000, 700, 30, phi=0.9), 700),
        # every candidate listed: grouped tally, the closure's own warm rows,
        # persistent closure (more than 256 warm)
        ("grouped_all_listed", W.impartial(102, 3000, 400, 40), 400),
        # grouped tally with unlisted candidates: persistent closure, uniform
        # cold columns
        ("grouped_some_unlisted", W.plackett_luce_zipf(103, 1500, 2000, 15, s=1.1), 2000),
        # full rankings: dense tally (no branch there), closure's own rows
        ("full_rankings", W.mallows(104, 600, 200, None, phi=0.8), 200),
    ]


@pytest.mark.parametrize("case", range(4))
def test_graph_replay_matches_oracle_and_eager(case):
    label, ranks, m = _cases()[case]
    dev = torch.device("cuda", 0)
    ctx = S.context(0)
    r = torch.from_numpy(np.ascontiguousarray(ranks)).to(dev)
    out = _outs(m, dev)

    def step():
        S.schulze_run(r, m, out=out, ctx=ctx)

    step()
    torch.cuda.synchronize()
    _check_oracle(ranks, m, out, label + " eager")
    eager = {key: t.clone() for key, t in out.items()}
    g = _capture(step)
    for t in out.values():
        t.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    for key in out:
        assert torch.equal(out[key], eager[key]), f"{label}: graph {key} differs from eager"
    assert ctx.status() == S.OK


def test_graph_follows_the_data():
    """One graph, captured on ballots that take the compact tally and the
    cluster closure, replayed on ballots of the same shape that take the
    grouped tally, the closure's own warm-row pass and the persistent
    closure, and back: each replay equals the oracle."""
    m, n, k = 600, 3000, 30
    A = W.mallows(201, n, m, k, phi=0.9)
    B = W.impartial(202, n, m, k)
    assert len(np.unique(A)) <= 256 < len(np.unique(B)) == m
    dev = torch.device("cuda", 0)
    ctx = S.context(0)
    r = torch.from_numpy(A).to(dev)
    out = _outs(m, dev)

    def step():
        S.schulze_run(r, m, out=out, ctx=ctx)

    g = _capture(step)
    for label, ballots in (("A", A), ("B", B), ("A again", A)):
        r.copy_(torch.from_numpy(ballots))
        for t in out.values():
            t.fill_(-7)
        g.replay()
        _check_oracle(ballots, m, out, "replay on " + label)
    assert ctx.status() == S.OK


def test_closure_graph_without_tally_flags():
    """schulze_strongest_paths alone (no tally flags) in a graph: a warm set
    for the cluster closure and one for the persistent closure."""
    dev = torch.device("cuda", 0)
    ctx = S.context(0)
    for seed, m, nw in ((301, 900, 120), (302, 900, 700)):
        rs = np.random.Generator(np.random.PCG64(seed))
        d = np.zeros((m, m), np.int32)
        warm = rs.choice(m, nw, replace=False)
        d[np.ix_(warm, np.arange(m))] = rs.integers(0, 50, (nw, m))
        np.fill_diagonal(d, 0)
        dd = torch.from_numpy(d).to(dev)
        p = torch.empty((m, m), dtype=torch.int32, device=dev)

        def step():
            S.schulze_strongest_paths(dd, 100, p=p, ctx=ctx)

        g = _capture(step)
        p.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        want = oracle.strongest_paths(d, nthreads=8)
        assert np.array_equal(p.cpu().numpy(), want), (seed, m, nw)
    assert ctx.status() == S.OK


def test_host_call_graph_replays():
    """schulze_run_host with page-locked buffers runs as a cached graph: new
    ballots in the same buffer, a second buffer (captured anew), pageable
    buffers (eager), and invalid ballots (status reported, then cleared),
    each against the oracle."""
    m, n, k = 500, 2000, 20
    dev = torch.device("cuda", 0)
    ctx = S.context(0)
    ballots = [W.mallows(401 + i, n, m, k, 0.9, W.permutation(402 + i, m)) for i in range(3)]
    r_pin = torch.empty((n, k), dtype=torch.int32).pin_memory()
    win = torch.empty(m, dtype=torch.int32).pin_memory()
    order = torch.empty(m, dtype=torch.int32).pin_memory()

    def check(ranks, got_win, got_order, what):
        _, _, w_want, o_want, _ = oracle.schulze(ranks, m, nthreads=8)
        assert np.array_equal(np.asarray(got_win), w_want), what
        assert np.array_equal(np.asarray(got_order), o_want), what

    for i in (0, 1, 0, 2):  # same buffers, new contents each call
        r_pin.copy_(torch.from_numpy(ballots[i]))
        S.schulze_run_host(r_pin, m, winners=win, order=order, device=0)
        check(ballots[i], win.numpy(), order.numpy(), f"pinned call on ballots {i}")
    r_pin2 = torch.from_numpy(ballots[1]).pin_memory()  # another buffer: a new capture
    S.schulze_run_host(r_pin2, m, winners=win, order=order, device=0)
    check(ballots[1], win.numpy(), order.numpy(), "second pinned buffer")
    w_np, o_np = S.schulze_run_host(ballots[2], m, device=0)  # pageable: eager
    check(ballots[2], w_np, o_np, "pageable buffers")
    bad = ballots[0].copy()
    bad[7, 3] = m + 5
    r_pin.copy_(torch.from_numpy(bad))
    with pytest.raises(S.SchulzeError):
        S.schulze_run_host(r_pin, m, winners=win, order=order, device=0)
    r_pin.copy_(torch.from_numpy(ballots[0]))
    S.schulze_run_host(r_pin, m, winners=win, order=order, device=0)
    check(ballots[0], win.numpy(), order.numpy(), "after invalid ballots")
    assert ctx.status() == S.OK


def test_run_outputs_are_ordered_on_the_callers_stream():
    """schulze_run writes p on a side stream of its context and joins it back
    to the caller's stream: work queued on that stream after the call sees all
    of p, with no device-wide synchronisation in between. p is filled with -1
    first; a reduction queued right after the call must find no -1 left, the
    diagonal zero, and the same p as a call that synchronises the device."""
    e = W.large_topk()  # 151 listed of 4096: p is mostly the zero rows of unlisted candidates
    m = e.m
    dev = torch.device("cuda")
    r = torch.from_numpy(e.ranks).to(dev)
    ref = S.schulze_run(r, m)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        out = _outs(m, dev)
        out["p"].fill_(-1)
        S.schulze_run(r, m, out=out)
        low = out["p"].min()
        diag = out["p"].diagonal().abs().sum()
        same = torch.equal(out["p"], ref["p"])  # a host read: synchronises s only
    torch.cuda.synchronize()
    assert int(low) >= 0 and int(diag) == 0 and same
