#!/usr/bin/env python3
"""Benchmark of the Schulze hot path on GB300.

One step = one election through the whole path (pairwise tally, widest-path
closure, winners, ranking) via the C ABI (`schulze_run`). Default workload:
m=16384 candidates, n=200000 top-20 Plackett-Luce Zipf(1.1) ballots, whose
closure runs on 32-bit lanes over (almost) every candidate, so that its
cand^3/s counts cubic work the step really does. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores

Under torchrun every rank runs its own election (different seed, no
collective on the data path) and rank 0 prints the whole-job rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))


def profiled_traffic() -> dict:
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    the kernels captured with ncu, from the table in profiles/dram_traffic.md:
    {(kernel class, workload): bytes}, kept only for kernels whose source file
    still has the digest recorded at capture time (a changed kernel has no
    traffic figure until it is captured again)."""
    out = {}
    try:
        lines = open(os.path.join(ROOT, "profiles", "dram_traffic.md")).read().splitlines()
    except OSError:
        return out
    for line in lines:
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) != 6:
            continue
        cls, _kernel, workload, nbytes, src, digest = cells
        try:
            value = float(nbytes.replace(",", ""))
            with open(os.path.join(ROOT, src), "rb") as f:
                current = hashlib.sha256(f.read()).hexdigest()[:16]
        except (ValueError, OSError):
            continue
        if current == digest:
            out[(cls, workload)] = value
    return out


def hbm_peak_gbs():
    """HBM copy bandwidth measured on this GPU pool (MEASURED_PEAKS.json,
    written beside the repository), else the recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        if v > 0:
            return v, "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return 6800.0, "6.8 TB/s earlier GB300 copy measurement (of fallback)"


sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "candidates^3/sec strongest-path closure + elections/sec winners, exact vs oracle"
UNIT = "cand^3/s"

WORKLOADS = {
    "large_topk": dict(desc="m=4096, n=20000, top-50 Mallows phi=0.9, random reference order"),
    "small_mallows": dict(desc="m=64, n=1000, full Mallows phi=0.8, identity reference order"),
    "huge_pl": dict(desc="m=16384, n=200000, top-20 Plackett-Luce Zipf(1.1), int32 closure"),
    "batch_mixed": dict(desc="4096 elections, m~U[8,512], n~U[50,5000], full rankings, half Mallows "
                             "(phi~U[0.5,1]) half impartial culture, one persistent launch"),
    "learned": dict(desc="proposal network trained on GPU-solved top-k Mallows elections (20000 by "
                         "default); evaluation elections m=8192, n=20000, top-50, phi=0.9 (256 by default)"),
    "spotify_like": dict(desc="m=18407, n=15553, top-200 Plackett-Luce Zipf(1.1): the shape of the paper's "
                              "largest Spotify profile, synthetic"),
    "iterated_topk": dict(desc="top-10 ranking by iterated winner removal on the m=4096, n=20000, top-50 "
                               "Mallows(0.9) election (tally first, outside the timed region)"),
    "propagation": dict(desc="winners from the tally by the paper's Alg. 1-4 restated on the GPU, against "
                             "the closure + winners, on the default election and the Spotify-shaped one"),
    "weak_orders": dict(desc="m=1024, n=20000 weak orders in position form: Mallows(0.97) rankings cut into "
                             "tiers of 16 tied places; position-compare tally, closure, winners, ranking"),
}


def make_election(name: str, rank: int, m=None, n=None):
    """The workload's election; m / n override its size (profiling runs)."""
    import workloads as W
    size = {k: v for k, v in (("m", m), ("n", n)) if v}
    if name == "large_topk":
        return W.large_topk(seed=W.SEED_BASE + 1 + 1000 * rank, **size)
    if name == "small_mallows":
        if size:
            raise SystemExit("small_mallows has a fixed size")
        return W.small_mallows(seed=W.SEED_BASE + 1000 * rank)
    if name == "huge_pl":
        return W.huge_pl(seed=W.SEED_BASE + 2 + 1000 * rank, **size)
    if name == "spotify_like":
        return W.spotify_like(seed=W.SEED_BASE + 8 + 1000 * rank, **size)
    raise SystemExit(f"unknown workload {name}")


def cpu_sample_election(name: str):
    """A bounded sample of the workload for the oracle: a smaller election
    from the same generator (same ballot model, fewer candidates)."""
    import workloads as W
    if name == "large_topk":
        return W.large_topk(seed=W.SEED_BASE + 77, m=1536), "one m=1536, n=20000 top-50 Mallows(0.9) election"
    if name == "small_mallows":
        return W.small_mallows(), "the full m=64, n=1000 election"
    if name == "huge_pl":
        return (W.huge_pl(seed=W.SEED_BASE + 78, n=60000, m=2048),
                "one m=2048, n=60000 top-20 Plackett-Luce Zipf(1.1) election")
    if name == "spotify_like":
        return (W.spotify_like(seed=W.SEED_BASE + 81, m=1536),
                "one m=1536, n=15553 top-200 Plackett-Luce Zipf(1.1) election")
    if name == "batch_mixed":
        return W.batch_mixed(E=48, seed=W.SEED_BASE + 79), "48 elections drawn like the 4096-election batch"
    raise SystemExit(name)


def time_oracle_batch(b, nthreads: int):
    """Wall time of the oracle's whole path over every election of a batch."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for e in range(b.E):
        oracle.schulze(b.election(e).ranks, int(b.m[e]), nthreads=nthreads)
    return time.perf_counter() - t0


def run_learned(args, world, rank, local):
    """Learned winner proposals: train the proposal network on GPU-solved
    elections (m~U[256,2048], n~U[1000,20000], top-k k~U[10,100], Mallows
    phi~U[0.6,1]), then on evaluation elections (m=8192, n=20000, top-50,
    phi=0.9) time exact winner determination from the tally by (a) the full
    closure + winners, (b) certified MLP proposals, (c) certified Copeland
    proposals, each bracketed by CUDA events on the current stream. Winner
    sets of (b) and (c) must equal (a) on every election. The same three are
    timed on the Spotify-shaped dense profile, where the certification
    hands over to the paper's propagation (warm set above 2048)."""
    import torch
    import paper_2505_12976_gb300 as S
    from paper_2505_12976_gb300 import learned as L
    import workloads as W

    dev = torch.device("cuda", local)
    ctx = S.context(local)
    t_start = time.perf_counter()
    data = L.Dataset(dev)
    chunk = 256
    for c0 in range(0, args.train_elections, chunk):
        tb = W.learned_train(E=min(chunk, args.train_elections - c0), seed=W.SEED_BASE + 4 + 7919 * c0)
        for e in range(tb.E):
            data.add(torch.from_numpy(tb.election(e).ranks).to(dev), int(tb.m[e]))
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t_start
    trainer = L.Trainer(W.mlp_init(), seed=W.SEED_BASE + 6)
    t0 = time.perf_counter()
    hist = trainer.train(data, epochs=args.epochs, elections_per_step=64, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        b.synchronize()
        return out, a.elapsed_time(b)

    def compare(d, n):
        p = torch.empty_like(d)
        wc, t_c = timed(lambda: S.schulze_winners(S.schulze_strongest_paths(d, n, p=p, ctx=ctx), ctx=ctx))
        (wm, sm), t_m = timed(lambda: S.schulze_winners_fast(d, n, trainer.params, top=4, ctx=ctx))
        (wk, sk), t_k = timed(lambda: S.schulze_winners_fast(d, n, None, top=4, ctx=ctx))
        return {"agree_mlp": bool(torch.equal(wc, wm)), "agree_copeland": bool(torch.equal(wc, wk)),
                "closure_ms": t_c, "mlp_ms": t_m, "copeland_ms": t_k, "mlp_hit": sm[0], "mlp_fallback": sm[1],
                "copeland_hit": sk[0], "copeland_fallback": sk[1]}

    ev = W.learned_eval(E=args.eval_elections, m=args.m or 8192, n=args.n or 20000)
    rows = []
    clocks = ClockSampler(local)
    clocks.start()
    for e in range(ev.E):
        d = S.schulze_tally(torch.from_numpy(ev.election(e).ranks).to(dev), int(ev.m[e]), ctx=ctx)
        if e == 0:  # warm-up of every path
            compare(d, int(ev.n[e]))
        rows.append(compare(d, int(ev.n[e])))
    clock_info = clocks.stop()
    dense = W.spotify_like(seed=W.SEED_BASE + 8 + 1000 * rank)
    dd = S.schulze_tally(torch.from_numpy(dense.ranks).to(dev), dense.m, ctx=ctx)
    compare(dd, dense.n)
    dense_row = compare(dd, dense.n)
    E = len(rows)
    avg = lambda key: sum(x[key] for x in rows) / E
    closure_ms, mlp_ms, cop_ms = avg("closure_ms"), avg("mlp_ms"), avg("copeland_ms")
    # per-kernel durations of the MLP path on the library's stream, from a
    # second, profiled pass over 16 of the evaluation elections: the features
    # pass dominates (algorithmic bytes: one read of d, m^2 4 B); the
    # certification's work is its widest-path rounds over the warm square
    # (two int32 copies of it, read once per round)
    sample = []
    for e in range(min(16, ev.E)):
        sample.append((S.schulze_tally(torch.from_numpy(ev.election(e).ranks).to(dev), int(ev.m[e]), ctx=ctx),
                       int(ev.n[e])))
    warm = [int(((d > d.t()).any(dim=1)).sum().item()) for d, _ in sample]
    torch.cuda.synchronize()
    ctx.profile(True)
    rounds = [S.schulze_winners_fast(d, nn, trainer.params, top=4, ctx=ctx)[1][3] for d, nn in sample]
    prof = ctx.profile_read()
    ctx.profile(False)
    del sample
    hbm_peak, hbm_src = hbm_peak_gbs()
    mm4 = float(ev.m[0]) * float(ev.m[0]) * 4
    fst = prof.get("learn_features")
    roof = None
    if fst:
        per = fst["ms"] / max(1, fst["launches"])
        roof = {"bound": "hbm", "kernel": "learn_features (features pass)", "achieved": mm4 / (per * 1e-3) / 1e9,
                "peak": hbm_peak, "unit": "GB/s", "frac": mm4 / (per * 1e-3) / 1e9 / hbm_peak,
                "traffic": profiled_traffic().get(("learn_features", "learned")) if not (args.m or args.n) else None,
                "bytes_per_launch": mm4, "work": "d read once (m^2 4 B; each entry is read twice, the second "
                "time mostly from L2)", "per_launch_ms": per, "launches": fst["launches"],
                "peak_source": hbm_src}
    cst = prof.get("certify_paths")
    certify = None
    if cst:
        cert_bytes = sum(r * 2.0 * 4.0 * w * w for r, w in zip(rounds, warm))
        certify = {"per_launch_ms": cst["ms"] / max(1, cst["launches"]), "launches": cst["launches"],
                   "rounds_mean": sum(rounds) / len(rounds), "warm_mean": sum(warm) / len(warm),
                   "bytes_per_round": "2 x 4 B x warm^2 (the warm square and its transpose)",
                   "achieved_GBps": cert_bytes / (cst["ms"] * 1e-3) / 1e9,
                   "note": "one 1024-thread CTA; the warm square stays in L1/L2, so the rounds are latency-bound"}
    breakdown = {kname: {"ms_per_election": st["ms"] / max(1, len(rounds)), "launches": st["launches"]}
                 for kname, st in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    line = {"metric": METRIC + " (learned-proposal workload: elections/sec of exact winner determination)",
            "value": 1e3 / mlp_ms, "unit": "elections/s", "n_gpus": 1, "steps": E, "warmup": 1,
            "ms_per_step": mlp_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32+fp32", "data": "synthetic",
            "config": {"workload": "learned", "train_elections": len(data), "epochs": args.epochs,
                       "eval": f"{E} elections, m={int(ev.m[0])}, n={int(ev.n[0])}, top-{int(ev.k[0])} Mallows "
                               "phi=0.9", "proposals": 4,
                       "dense": f"spotify_like m={dense.m}, n={dense.n}, top-{dense.k} Plackett-Luce Zipf(1.1)",
                       "timing": "CUDA events on the current stream around each call (from the tally)"},
            "agreement_mlp": sum(x["agree_mlp"] for x in rows) / E,
            "agreement_copeland": sum(x["agree_copeland"] for x in rows) / E,
            "closure_ms_per_election": closure_ms, "mlp_ms_per_election": mlp_ms,
            "copeland_ms_per_election": cop_ms, "speedup_mlp_vs_closure": closure_ms / mlp_ms,
            "speedup_copeland_vs_closure": closure_ms / cop_ms,
            "mlp_top1_hit_rate": sum(x["mlp_hit"] == 0 for x in rows) / E,
            "mlp_fallback_rate": sum(x["mlp_fallback"] > 0 for x in rows) / E,
            "copeland_top1_hit_rate": sum(x["copeland_hit"] == 0 for x in rows) / E,
            "copeland_fallback_rate": sum(x["copeland_fallback"] > 0 for x in rows) / E,
            "dense_profile": dense_row,
            "train": {"seconds": t_train, "data_seconds": t_data, "loss_first_epoch": hist[0],
                      "loss_last_epoch": hist[-1]},
            "roofline": roof, "certify": certify, "kernels": breakdown, "cpu_baseline": None,
            "e2e": None, "e2e_note": "timed from a device-resident tally; no host buffers on this path",
            "device_status": ctx.status(), "clocks": clock_info}
    print(json.dumps(line), flush=True)
    return 0


def run_weak(args, world, rank, local):
    """Weak-order ballots: one step = schulze_tally_positions, then
    schulze_strongest_paths (winning votes, or margins with --margin),
    schulze_winners and schulze_ranking, captured as one CUDA graph."""
    import torch
    import torch.distributed as dist
    import paper_2505_12976_gb300 as S
    import workloads as W

    dev = torch.device("cuda", local)
    m, n = args.m or 1024, args.n or 20000
    pos_h = W.weak_orders(seed=W.SEED_BASE + 7 + 1000 * rank, n=n, m=m)
    pos_d = torch.from_numpy(pos_h).to(dev)
    ctx = S.context(local)
    ctx.reserve(m, n, m)
    flags = S.F_MARGIN if args.margin else 0
    d = torch.empty((m, m), dtype=torch.int32, device=dev)
    p = torch.empty((m, m), dtype=torch.int32, device=dev)
    win = torch.empty(m, dtype=torch.int32, device=dev)
    order = torch.empty(m, dtype=torch.int32, device=dev)
    bb = torch.empty(m, dtype=torch.int32, device=dev)

    def step(src):
        S.schulze_tally_positions(src, d=d, ctx=ctx)
        S.schulze_strongest_paths(d, n, p=p, flags=flags, ctx=ctx)
        S.schulze_winners(p, winners=win, ctx=ctx)
        S.schulze_ranking(p, order=order, beaten_by=bb, ctx=ctx)

    for _ in range(args.warmup):
        step(pos_d)
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    step(pos_d)
    launches_per_step = ctx.launch_count() - l0
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        step(pos_d)
    torch.cuda.current_stream().wait_stream(cap)
    with torch.cuda.graph(graph):
        step(pos_d)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record()
        graph.replay()
        evs[i][1].record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clock_info = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    ref = (win.clone(), order.clone())
    step(pos_d)
    torch.cuda.synchronize()
    graph_matches = torch.equal(ref[0], win) and torch.equal(ref[1], order)
    ctx.profile(True)
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda._sleep(2_000_000)
        step(pos_d)
    prof = ctx.profile_read()
    ctx.profile(False)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # dense tally: n m (m - 1) position compares, ALU-bound; 16-bit packed
    # compare + subtract = one instruction per compare and lane pair
    top = max(prof.items(), key=lambda kv: kv[1]["ms"])
    tally = prof.get("tally_dense")
    roof = None
    if tally:
        per = tally["ms"] / max(1, tally["launches"])
        cmp_per_launch = float(n) * m * (m - 1) / max(1, tally["launches"] // args.steps)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * 64 * 2 * 2.07e9  # 64 lanes/clk/SM x 2 lanes per packed op; a compare takes vsub + vcmp
        roof = {"bound": "alu", "kernel": "tally_dense", "achieved": cmp_per_launch / (per * 1e-3) / 1e9,
                "peak": peak / 2 / 1e9, "unit": "Gcompares/s", "frac": cmp_per_launch / (per * 1e-3) / (peak / 2),
                "traffic": None, "per_launch_ms": per,
                "peak_source": "152 SMs x 64 int lanes/clk x 2 lanes per 16-bit op x 2.07 GHz / 2 ops per compare"}
    # end to end: host positions (pinned) in, winners and order out, through the same calls
    pos_pin = torch.from_numpy(pos_h).pin_memory()
    win_h = torch.empty(m, dtype=torch.int32).pin_memory()
    ord_h = torch.empty(m, dtype=torch.int32).pin_memory()
    stage = torch.empty_like(pos_d)
    tot = 0.0
    e2e_steps = args.e2e_steps or max(3, args.steps)
    for _ in range(e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stage.copy_(pos_pin, non_blocking=True)
        step(stage)
        win_h.copy_(win, non_blocking=True)
        ord_h.copy_(order, non_blocking=True)
        torch.cuda.synchronize()
        tot += time.perf_counter() - t0 if _ else 0.0
    e2e_sec = tot / e2e_steps
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sm_, sn_ = 256, 2000
        sample = W.weak_orders(seed=W.SEED_BASE + 80, n=sn_, m=sm_)
        sec = time_oracle_weak(sample, args.margin, os.cpu_count() or 1)
        cpu = {"value": float(sm_) ** 3 / sec, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"one m={sm_}, n={sn_} weak-order election of the same model "
                         f"(tally, closure, winners, ranking in {sec:.2f} s; cand^3/s = m^3 / time)"}
    if rank == 0:
        line = {"metric": METRIC, "value": world * float(m) ** 3 / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int16x2" if n <= 32767 else "int32",
                "data": "synthetic",
                "config": {"workload": "weak_orders", "detail": WORKLOADS["weak_orders"]["desc"], "m": m, "n": n,
                           "weights": "margin" if args.margin else "winning votes",
                           "l2": "flushed (512 MiB write) before every timed step"},
                "elections_per_sec": world / (ms * 1e-3), "roofline": roof,
                "kernels": {k: {"ms_per_step": v["ms"] / args.steps} for k, v in
                            sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
                "dominant_kernel": top[0], "cpu_baseline": cpu,
                "e2e": {"value": world * float(m) ** 3 / e2e_sec, "unit": UNIT,
                        "h2d_bytes_per_step": int(n) * int(m) * 4, "d2h_bytes_per_step": 2 * int(m) * 4},
                "gpu_launches": int(launches_per_step * args.steps),
                "timed_as": "CUDA graph of the four calls, replayed", "graph_matches_eager": graph_matches,
                "device_status": ctx.status(), "clocks": clock_info}
        print(json.dumps(line), flush=True)
    return 0


def run_iterated(args, world, rank, local):
    """Top-10 levels by iterated winner removal from the default election's
    tally: one step = one schulze_ranking_iterated call (host round trip per
    level, so timed on the host around a synchronized call)."""
    import torch
    import torch.distributed as dist
    import paper_2505_12976_gb300 as S
    import workloads as W

    dev = torch.device("cuda", local)
    e = W.large_topk(seed=W.SEED_BASE + 1 + 1000 * rank, **{k: v for k, v in (("m", args.m), ("n", args.n)) if v})
    ctx = S.context(local)
    d = S.schulze_tally(torch.from_numpy(e.ranks).to(dev), e.m, ctx=ctx)
    flags = S.F_MARGIN if args.margin else 0
    level = torch.empty(e.m, dtype=torch.int32, device=dev)
    k_top = 10
    for _ in range(args.warmup):
        S.schulze_ranking_iterated(d, e.n, k_top, flags=flags, level=level, ctx=ctx)
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    clocks.start()
    times, nl = [], 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, nl = S.schulze_ranking_iterated(d, e.n, k_top, flags=flags, level=level, ctx=ctx)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clock_info = clocks.stop()
    sec = sum(times) / len(times)
    if world > 1:
        t = torch.tensor([sec], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        sec = float(t.item())
    placed = int((level > 0).sum().item())
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ce = W.large_topk(seed=W.SEED_BASE + 77, m=1536)
        dc = oracle.tally(ce.ranks, ce.m)
        t0 = time.perf_counter()
        oracle.ranking_iterated(dc, k_top, args.margin)
        csec = time.perf_counter() - t0
        cpu = {"value": float(ce.m) ** 3 / csec, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"top-{k_top} iterated ranking of one m=1536 election of the same model in {csec:.2f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": world * float(e.m) ** 3 / sec, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int16x2", "data": "synthetic",
                "config": {"workload": "iterated_topk", "detail": WORKLOADS["iterated_topk"]["desc"], "m": e.m,
                           "n": e.n, "k": e.k, "k_top": k_top, "levels": nl, "placed": placed,
                           "weights": "margin" if args.margin else "winning votes",
                           "l2": "flushed (512 MiB write) before every timed step"},
                "ms_per_level": sec * 1e3 / max(nl, 1), "roofline": None, "cpu_baseline": cpu,
                "e2e": {"value": world * float(e.m) ** 3 / sec, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 4 * nl},
                "timed_as": "host wall time of one synchronized call (device-resident tally)",
                "device_status": ctx.status(), "clocks": clock_info}
        print(json.dumps(line), flush=True)
    return 0


def run_propagation(args, world, rank, local):
    """Winners only, from a device-resident tally: the paper's vertex-centric
    algorithm (schulze_winners_propagation) against the closure path
    (schulze_strongest_paths + schulze_winners), on the default top-k
    election and on the Spotify-shaped one; winner sets compared."""
    import torch
    import paper_2505_12976_gb300 as S
    import workloads as W

    dev = torch.device("cuda", local)
    ctx = S.context(local)
    flags = S.F_MARGIN if args.margin else 0
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    rows = {}
    for name, e in (("large_topk", W.large_topk(seed=W.SEED_BASE + 1 + 1000 * rank)),
                    ("spotify_like", W.spotify_like(seed=W.SEED_BASE + 8 + 1000 * rank))):
        d = S.schulze_tally(torch.from_numpy(e.ranks).to(dev), e.m, ctx=ctx)
        p = torch.empty_like(d)
        win_c = torch.empty(e.m, dtype=torch.int32, device=dev)
        win_p = torch.empty(e.m, dtype=torch.int32, device=dev)

        def closure():
            S.schulze_strongest_paths(d, e.n, p=p, flags=flags, ctx=ctx)
            S.schulze_winners(p, winners=win_c, ctx=ctx)

        def propagation():
            return S.schulze_winners_propagation(d, flags=flags, winners=win_p, ctx=ctx)[1]

        def timed(fn, steps):
            out, ts = None, []
            for _ in range(steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                out = fn()
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            return sum(ts) / len(ts), out

        steps = max(1, min(args.steps, 5 if e.m > 8192 else args.steps))
        closure(), propagation()
        tc, _ = timed(closure, steps)
        tp, stats = timed(propagation, steps)
        rows[name] = {"m": e.m, "n": e.n, "k": e.k, "closure_ms": tc * 1e3, "propagation_ms": tp * 1e3,
                      "iterations": stats[0], "rounds": stats[1], "same_winners": bool(torch.equal(win_c, win_p)),
                      "winners": int(win_c.sum().item())}
    if rank == 0:
        main_row = rows["large_topk"]
        line = {"metric": METRIC + " (winners only: the paper's Alg. 1-4 restated on the GPU)",
                "value": world * 1e3 / main_row["propagation_ms"], "unit": "elections/s", "n_gpus": world,
                "steps": args.steps, "warmup": 1, "ms_per_step": main_row["propagation_ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": "propagation", "detail": WORKLOADS["propagation"]["desc"],
                           "weights": "margin" if args.margin else "winning votes",
                           "l2": "flushed (512 MiB write) before every timed call"},
                "comparison": rows, "roofline": None, "cpu_baseline": None,
                "e2e": {"value": world * 1e3 / main_row["propagation_ms"], "unit": "elections/s",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "timed_as": "host wall time of synchronized calls on a device-resident tally",
                "device_status": ctx.status()}
        print(json.dumps(line), flush=True)
    return 0


def time_oracle_weak(pos, margin: bool, nthreads: int):
    """Wall time of the oracle's whole path on weak-order ballots."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    d = oracle.tally_positions(pos)
    w = oracle.weights_margin(d) if margin else oracle.weights(d)
    p = oracle.closure(w, nthreads=nthreads)
    oracle.winners(p)
    oracle.ranking(p)
    return time.perf_counter() - t0


def run_batch(args, world, rank, local):
    """Batched elections: one step = one persistent launch over the whole batch
    (inputs of 10.8 GB, far larger than L2). Also times one launch sequence
    per election (schulze_run) on a sample for comparison."""
    import torch
    import torch.distributed as dist
    import paper_2505_12976_gb300 as S
    import workloads as W

    dev = torch.device("cuda", local)
    E = args.batch_size
    bw = W.batch_mixed(E=E, seed=W.SEED_BASE + 3 + 1000 * rank)
    ctx = S.context(local)
    plan = S.SchulzeBatch(bw.n, bw.m, bw.k, ctx=ctx)
    ranks = torch.from_numpy(bw.ranks).to(dev)
    vec = lambda: torch.empty(plan.vec_elems, dtype=torch.int32, device=dev)
    winners, order, beaten = vec(), vec(), vec()
    tile, ordp = plan.autotune(ranks, os.path.join(tempfile.gettempdir(), "schulze_batch_autotune.txt"))
    step = lambda: plan.run(ranks, winners=winners, order=order, beaten_by=beaten)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    launches0 = ctx.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        evs[i][0].record()
        step()
        evs[i][1].record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clock_info = clocks.stop()
    launches = ctx.launch_count() - launches0
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    cubes = float(np.sum(bw.m.astype(np.float64) ** 3))
    value = world * cubes / (ms * 1e-3)
    eps = world * E / (ms * 1e-3)
    # roofline of the one batch kernel: its algorithmic work is the tally's
    # position compares (n m (m - 1) / 2 per full-ranking election, n m (m - 1)
    # otherwise) and the closure's m^3 (max, min) updates, each at the rate the
    # probes measure on this GPU (guard-bit compare; packed 16-bit min/max with
    # a three-input max, or int32 when an election has more than 32767 ballots)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sec_c, cmp_c = S.probe_minmax(12, sms * 8, 4096, local)
    s16_batch = bool(np.all(bw.n <= 32767))
    sec_u, upd_u = S.probe_minmax(2 if s16_batch else 3, sms * 8, 4096, local)
    cmp_peak, upd_peak = cmp_c / sec_c, upd_u / sec_u
    mf, nf, kf = (x.astype(np.float64) for x in (bw.m, bw.n, bw.k))
    compares = float(np.sum(np.where(kf >= mf - 1, 0.5, 1.0) * nf * mf * (mf - 1)))
    at_peak = compares / cmp_peak + cubes / upd_peak  # seconds of ALU work at the measured rates
    roof = {"bound": "alu", "kernel": "batch_elections (tally compares + closure updates)",
            "achieved": (compares + cubes * cmp_peak / upd_peak) / (ms * 1e-3) / 1e9, "peak": cmp_peak / 1e9,
            "unit": "Gcompares/s (closure updates counted at the measured compare/update rate ratio)",
            "frac": at_peak / (ms * 1e-3), "traffic": None,
            "work": {"tally_compares": compares, "closure_updates": cubes,
                     "tally_ms_at_peak": compares / cmp_peak * 1e3, "closure_ms_at_peak": cubes / upd_peak * 1e3},
            "peak_source": "schulze_probe_minmax kinds 12 (compare) and 2/3 (min/max) measured in this run"}
    sched = plan.bucket_schedule()
    # one launch sequence per election on a sample of the same batch
    sample = list(range(0, E, max(1, E // 256)))[:256]
    singles = [(torch.from_numpy(bw.election(e).ranks).to(dev), int(bw.m[e])) for e in sample]
    for r, m in singles[:8]:
        S.schulze_run(r, m, ctx=ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r, m in singles:
        S.schulze_run(r, m, ctx=ctx)
    torch.cuda.synchronize()
    single_eps = len(singles) / (time.perf_counter() - t0)
    # end to end: pinned host ballots in, winners and order out, every step,
    # through the library's host-buffer call (its copies overlap the work)
    ranks_h = torch.from_numpy(bw.ranks).pin_memory()
    win_h = torch.empty(plan.vec_elems, dtype=torch.int32).pin_memory()
    ord_h = torch.empty(plan.vec_elems, dtype=torch.int32).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    plan.run_host(ranks_h, win_h, ord_h)  # first call: the plan's device buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.run_host(ranks_h, win_h, ord_h)
    e2e_sec = (time.perf_counter() - t0) / e2e_steps
    e2e_exact = bool(torch.equal(win_h, winners.cpu()) and torch.equal(ord_h, order.cpu()))
    status = ctx.status()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, sample_desc = cpu_sample_election("batch_mixed")
        threads = os.cpu_count() or 1
        sec = time_oracle_batch(cb, threads)
        cpu = {"value": float(np.sum(cb.m.astype(np.float64) ** 3)) / sec, "unit": UNIT, "cores": threads,
               "kind": "oracle", "sample": sample_desc + f" ({cb.E / sec:.1f} elections/s on the host)"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int16x2", "data": "synthetic",
                "config": {"workload": "batch_mixed", "detail": WORKLOADS["batch_mixed"]["desc"], "elections": E,
                           "ballot_bytes": int(bw.ranks.nbytes),
                           "schedule": {"tally_policy": tile, "order_policy": ordp,
                                        "by_m_bucket": {f"m<={mx}": {"ballots_per_step": ch, "groups_per_tile": g,
                                                                     "elections": el}
                                                        for (mx, ch, el), g in zip(sched, plan.bucket_tiles())}},
                           "l2": "inputs (ballots) larger than L2"},
                "elections_per_sec": eps, "one_launch_per_election_elections_per_sec": single_eps,
                "batch_speedup_vs_one_launch_per_election": eps / world / single_eps,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": world * cubes / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": int(bw.ranks.nbytes),
                        "d2h_bytes_per_step": 2 * int(plan.vec_elems) * 4, "call": "schulze_batch_run_host",
                        "matches_device_run": e2e_exact},
                "gpu_launches": int(launches), "device_status": status, "clocks": clock_info}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def time_oracle(e, nthreads: int):
    """Wall time of the oracle's whole path on election e."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.schulze(e.ranks, e.m, nthreads=nthreads)
    return time.perf_counter() - t0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.strip().split(",") for ln in self.file.read().splitlines() if ln.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_sharded(args, world, rank, local):
    """One election split by voters over the ranks: each rank tallies its
    shard, one int32 sum all-reduce (NCCL) gives every rank the whole d, and
    every rank closes it and extracts winners and ranking (the closure is
    replicated). Total work is fixed: strong scaling. Rank 0 checks the
    result against one-GPU schulze_run on all ballots."""
    import torch
    import paper_2505_12976_gb300 as S
    from paper_2505_12976_gb300 import distributed as D

    dev = torch.device("cuda", local)
    e = make_election(args.workload, 0, args.m, args.n)  # the same election on every rank
    n, k, m = e.n, e.k, e.m
    a, b = D.voter_shard(n, rank, world)
    shard = torch.from_numpy(e.ranks[a:b].copy()).to(dev)
    ctx = S.context(local)
    ctx.reserve(m, max(b - a, 1), k)
    p = torch.empty((m, m), dtype=torch.int32, device=dev)

    def step():
        d = D.tally_voter_sharded(shard, m, ctx=ctx) if world > 1 else S.schulze_tally(shard, m, ctx=ctx)
        S.schulze_strongest_paths(d, n, p=p, ctx=ctx)
        win = S.schulze_winners(p, ctx=ctx)
        order, _ = S.schulze_ranking(p, ctx=ctx)
        return d, win, order

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record()
        d, win, order = step()
        evs[i][1].record()
    torch.cuda.synchronize()
    ms = sum(x.elapsed_time(y) for x, y in evs) / args.steps
    if world > 1:
        ms = D.max_over_ranks(ms, device=dev)
    same = None
    if rank == 0:
        full = S.schulze_run(torch.from_numpy(e.ranks).to(dev), m, ctx=ctx)
        same = bool(torch.equal(full["d"], d) and torch.equal(full["winners"], win) and
                    torch.equal(full["order"], order))
    if rank == 0:
        line = {"metric": METRIC, "value": float(m) ** 3 / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "int16x2" if n <= 32767 else "int32",
                "data": "synthetic",
                "config": {"workload": args.workload + " (voters sharded over the ranks)", "m": m, "n": n, "k": k,
                           "parallelism": f"voter-sharded tally + int32 all-reduce of d over {world}, "
                                          "closure replicated",
                           "l2": "flushed (512 MiB write) before every timed step"},
                "sharded_matches_single_gpu": same, "device_status": ctx.status()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_kernel_case(args, local):
    """Small single-kernel cases for profiling (one GPU): `closure_s32` /
    `closure_s16` close a seeded dense random count matrix (m = --m, default
    4096) twice as warm-up and once timed; `tally_grouped` tallies the
    default m = 16384, n = 200000 top-20 election (the grouped form) three
    times and once timed; `tally_compact` does the same for the m = 4096,
    n = 20000 top-50 election (151 listed candidates: the compact form);
    `batch_sample` runs a 256-election sample of the mixed batch twice and
    once timed; `features` computes the 16 per-candidate features of one
    m = 8192, n = 20000 top-50 election of the learned workload's evaluation
    set three times and once timed. Prints the timed call's milliseconds."""
    import torch
    import paper_2505_12976_gb300 as S
    import workloads as W

    dev = torch.device("cuda", local)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    if args.kernel_case in ("closure_s32", "closure_s16"):
        m = args.m or 4096
        hi = 1000000 if args.kernel_case == "closure_s32" else 30000
        flags = S.F_FORCE_S32 if args.kernel_case == "closure_s32" else S.F_FORCE_S16
        rs = np.random.Generator(np.random.PCG64(5))
        d = rs.integers(0, hi, size=(m, m), dtype=np.int32)
        np.fill_diagonal(d, 0)
        dd = torch.from_numpy(d).to(dev)
        p = torch.empty_like(dd)
        call = lambda: S.schulze_strongest_paths(dd, hi, p=p, flags=flags)
        reps = 2
    elif args.kernel_case in ("tally_grouped", "tally_compact"):
        e = W.huge_pl() if args.kernel_case == "tally_grouped" else W.large_topk()
        r = torch.from_numpy(e.ranks).to(dev)
        d = torch.empty((e.m, e.m), dtype=torch.int32, device=dev)
        call = lambda: S.schulze_tally(r, e.m, d=d)
        reps = 3
    elif args.kernel_case == "features":
        lb = W.learned_eval(E=1)
        e = lb.election(0)
        d = S.schulze_tally(torch.from_numpy(e.ranks).to(dev), e.m)
        feat = torch.empty((e.m, 16), dtype=torch.float32, device=dev)
        call = lambda: S.schulze_features(d, int(lb.n[0]), feat=feat)
        reps = 3
    else:
        bw = W.batch_mixed(E=256, seed=123)
        plan = S.SchulzeBatch(bw.n, bw.m, bw.k)
        r = torch.from_numpy(bw.ranks).to(dev)
        w = torch.empty(plan.vec_elems, dtype=torch.int32, device=dev)
        call = lambda: plan.run(r, winners=w)
        reps = 2
    for _ in range(reps):
        call()
    torch.cuda.synchronize()
    ev[0].record()
    call()
    ev[1].record()
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "ms": ev[0].elapsed_time(ev[1]),
                      "device_status": S.context().status()}), flush=True)
    return 0


def run_reference(args, world, rank):
    """The CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return 0
    e, sample = cpu_sample_election(args.workload)
    threads = os.cpu_count() or 1
    batch = hasattr(e, "election")
    times = []
    for i in range(args.warmup + args.steps):
        t = time_oracle_batch(e, threads) if batch else time_oracle(e, threads)
        if i >= args.warmup:
            times.append(t)
    sec = sum(times) / len(times)
    # the same unit as this workload's own line: cand^3/s where the closure
    # does cubic work, elections/s for the top-k election with few listed
    # candidates
    if args.workload == "large_topk":
        value, unit = 1.0 / sec, "elections/s"
    else:
        value, unit = (float(np.sum(e.m.astype(np.float64) ** 3)) if batch else float(e.m) ** 3) / sec, UNIT
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "detail": WORKLOADS[args.workload]["desc"],
                       "sample": sample},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": unit, "cores": threads, "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="huge_pl", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--m", type=int, default=None, help="override the workload's candidate count")
    ap.add_argument("--n", type=int, default=None, help="override the workload's ballot count")
    ap.add_argument("--batch-size", type=int, default=4096, help="elections of the batch_mixed workload")
    ap.add_argument("--train-elections", type=int, default=20000, help="training elections (learned workload)")
    ap.add_argument("--eval-elections", type=int, default=256, help="evaluation elections (learned workload)")
    ap.add_argument("--epochs", type=int, default=20, help="training epochs (learned workload)")
    ap.add_argument("--margin", action="store_true", help="margin edge weights instead of winning votes")
    ap.add_argument("--kernel-case", default=None,
                    choices=["closure_s32", "closure_s16", "tally_grouped", "tally_compact", "batch_sample",
                             "features"],
                    help="run one small single-kernel case for profiling instead of the benchmark")
    ap.add_argument("--shard-voters", action="store_true",
                    help="one election, voters split over the ranks (tally + all-reduce of d; strong scaling)")
    args = ap.parse_args()
    world, rank, local = dist_setup()

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_12976_gb300 as S

    if args.kernel_case:
        return run_kernel_case(args, local)
    if args.shard_voters:
        return run_sharded(args, world, rank, local)
    if args.workload == "batch_mixed":
        return run_batch(args, world, rank, local)
    if args.workload == "learned":
        return run_learned(args, world, rank, local)
    if args.workload == "weak_orders":
        return run_weak(args, world, rank, local)
    if args.workload == "iterated_topk":
        return run_iterated(args, world, rank, local)
    if args.workload == "propagation":
        return run_propagation(args, world, rank, local)
    e = make_election(args.workload, rank, args.m, args.n)
    n, k, m = e.n, e.k, e.m
    ranks_d = torch.from_numpy(e.ranks).to(dev)
    ctx = S.context(local)
    ctx.reserve(m, n, k)
    out = {key: torch.empty(shape, dtype=torch.int32, device=dev)
           for key, shape in (("d", (m, m)), ("p", (m, m)), ("winners", (m,)), ("order", (m,)),
                              ("beaten_by", (m,)))}
    s16 = n <= 32767

    run_flags = S.F_MARGIN if args.margin else 0

    def step():
        S.schulze_run(ranks_d, m, out=out, flags=run_flags, ctx=ctx)

    # integer min/max issue rate (same lane format as the closure)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    probe = {}
    for kind, name in ((0, "s32"), (1, "s16x2"), (2, "s16x2_max3"), (3, "s32_max3"), (4, "f32"),
                       (5, "f32_max3"), (6, "s32_f32_mixed_max3"), (7, "bits_fmin_imax3"), (8, "bits_imin_fmax3"),
                       (9, "bits_third_int"), (10, "bits_two_thirds_int"), (11, "bits_half_int"),
                       (12, "guard_bit_compare")):
        sec, upd = S.probe_minmax(kind, sms * 8, 4096, local)
        probe[name] = upd / sec

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    step()
    launches_per_step = ctx.launch_count() - l0
    # the step as a CUDA graph: the same library call, captured once (the
    # reserved workspace means nothing is allocated inside it)
    graph = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        step()
    torch.cuda.current_stream().wait_stream(cap)
    with torch.cuda.graph(graph):
        step()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > L2 (129 MB)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record()
        graph.replay()
        evs[i][1].record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clock_info = clocks.stop()
    launches = launches_per_step * args.steps
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    graph_out = {key: t.clone() for key, t in out.items()}
    step()  # eager, for the check that the graph computed the same
    torch.cuda.synchronize()
    graph_matches = all(torch.equal(graph_out[key], out[key]) for key in out)
    # a second pass of the same steps, eager, with per-kernel events on the
    # library's stream: the breakdown and the dominant kernel's durations. A
    # GPU sleep ahead of each step lets the host queue every launch first, so
    # the events time the kernels and not the launch gaps.
    ctx.profile(True)
    cc0 = ctx.closure_counters()
    for i in range(args.steps):
        flush.zero_()
        torch.cuda._sleep(2_000_000)
        step()
    prof = ctx.profile_read()
    cc1 = ctx.closure_counters()
    ctx.profile(False)
    executed = {key: (cc1[key] - cc0[key]) / args.steps for key in cc0}
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * float(m) ** 3 / (ms * 1e-3)

    # exactness of this very run: winners certified by the oracle on rank 0
    # happens in the tests; here the device status must be clean
    status = ctx.status()

    # roofline of the dominant kernel class, and of every class for context:
    # algorithmic bytes (HBM-bound passes) or (max, min) updates (ALU-bound
    # closures) per launch over the mean launch duration
    dd = out["d"]
    nw = int(((dd > dd.t()).any(dim=1)).sum().item())  # candidates with an outgoing edge
    esz = 2 if s16 else 4
    nwp = -(-nw // 64) * 64
    alu_peak = max(probe["s16x2"], probe["s16x2_max3"]) if s16 else max(probe["s32"], probe["s32_max3"])
    hbm_peak, hbm_src = hbm_peak_gbs()
    mm4 = float(m) * m * 4
    work = {  # kernel class -> (bound, algorithmic units per launch, what)
        "tally_compact_pairs": ("hbm", mm4 + float(n) * k * 4, "d written once, ballots read once"),
        "tally_rows": ("hbm", mm4 + float(n) * k * 4, "d written once, ballots read once"),
        "tally_dense": ("alu", float(n) * m * (m - 1) / 2, "pair compares"),
        "tally_count": ("hbm", float(n) * k * 4, "ballots read once"),
        "closure_rowflags": ("hbm", mm4, "d read once"),
        "closure_widen": ("hbm", mm4, "p written once"),
        "closure_pack": ("hbm", float(nwp) * m * (8 + esz), "warm rows of d and d^T read, W written"),
        "closure_cluster": ("alu", float(nw) ** 3, "(max, min) updates of the warm square"),
        "closure_cold": ("alu", float(nw) ** 2 * (m - nw), "(max, min) updates of the cold columns"),
        "closure_persistent": ("alu", float(nw) ** 3, "(max, min) updates of the warm square, nw^3 (Floyd-Warshall "
                               "count; executed: 64^3 per tile update, reported beside it)"),
        "closure_beaten_by": ("hbm", 2.0 * nw * nw * esz, "warm square of W read along rows and columns"),
        "extract_beaten_by": ("hbm", 2 * mm4, "p and p^T read"),
    }

    traffic = profiled_traffic()

    def roofline(name, st):
        per_launch_ms = st["ms"] / max(1, st["launches"])
        bound, units, what = work.get(name, ("hbm", st["work"], "library estimate"))
        achieved = units / (per_launch_ms * 1e-3)
        dram = traffic.get((name, args.workload)) if not (args.m or args.n or args.margin) else None
        if bound == "alu":
            return {"bound": "alu", "kernel": name, "achieved": achieved / 1e9, "peak": alu_peak / 1e9,
                    "unit": "Gupdates/s", "frac": achieved / alu_peak, "traffic": dram,
                    "lane_format": "s16x2" if s16 else "s32", "work_per_launch": units, "work": what,
                    "per_launch_ms": per_launch_ms, "launches": st["launches"],
                    "peak_source": "schulze_probe_minmax measured in this run (best same-format variant)"}
        return {"bound": "hbm", "kernel": name, "achieved": achieved / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / 1e9 / hbm_peak, "traffic": dram, "bytes_per_launch": units, "work": what,
                "per_launch_ms": per_launch_ms, "launches": st["launches"],
                "peak_source": hbm_src}

    ranked = sorted(prof.items(), key=lambda kv: -kv[1]["ms"])
    roof = roofline(*ranked[0]) if ranked else None
    if roof and roof["kernel"] == "closure_persistent":
        roof["executed_updates_per_launch"] = (executed["tile_updates"] + executed["diag_closures"]) * 64.0 ** 3
    # kernels whose case the device decided against return at once: no work,
    # no roofline
    roof_all = {name: {key: r[key] for key in ("bound", "frac", "achieved", "unit", "per_launch_ms")}
                for name, r in ((name, roofline(name, st)) for name, st in ranked[:12]
                                if work.get(name, (None, st["work"]))[1] > 0)}
    breakdown = {kname: {"ms_per_step": st["ms"] / args.steps, "launches_per_step": st["launches"] / args.steps}
                 for kname, st in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    tally_ms = sum(st["ms"] for kname, st in prof.items() if kname.startswith("tally")) / args.steps
    tally_bytes = float(n) * k * 4 + float(m) * m * 4
    # the tally stage as a whole (every tally_* kernel of a step) against HBM:
    # ballots read once and d written once
    tally_roof = None
    if tally_ms:
        tally_roof = {"bound": "hbm", "kernel": "tally stage (all tally_* kernels)",
                      "achieved": tally_bytes / (tally_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                      "frac": tally_bytes / (tally_ms * 1e-3) / 1e9 / hbm_peak, "traffic": None,
                      "bytes_per_step": tally_bytes, "ms_per_step": tally_ms,
                      "work": "ballots read once (n k 4 B) + d written once (m^2 4 B)",
                      "peak_source": hbm_src}

    # end to end through host buffers (pinned), copies inside the timed region
    ranks_h = torch.from_numpy(e.ranks).pin_memory()
    win_h = torch.empty(m, dtype=torch.int32).pin_memory()
    ord_h = torch.empty(m, dtype=torch.int32).pin_memory()
    e2e_steps = args.e2e_steps or max(3, args.steps)
    S.schulze_run_host(ranks_h, m, flags=run_flags, winners=win_h, order=ord_h, device=local)
    tot = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.schulze_run_host(ranks_h, m, flags=run_flags, winners=win_h, order=ord_h, device=local)
        tot += time.perf_counter() - t0
    e2e_sec = tot / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_sec], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_sec = float(t.item())

    cpu = None
    # the closure does the cubic work when (almost) every candidate has an
    # outgoing edge; on a top-k profile with few listed candidates it closes
    # an nw-candidate square instead, and the line leads with elections/s,
    # the cubic rate reported beside the warm-square count
    cubic = nw >= 0.9 * m
    eps = world / (ms * 1e-3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ce, sample = cpu_sample_election(args.workload)
        threads = os.cpu_count() or 1
        reps = 3
        sec = sum(time_oracle(ce, threads) for _ in range(reps)) / reps
        cpu = {"value": float(ce.m) ** 3 / sec if cubic else 1.0 / sec, "unit": UNIT if cubic else "elections/s",
               "cores": threads, "kind": "oracle",
               "sample": sample + f" (tally, closure, winners, ranking in {sec:.2f} s, mean of {reps}; " +
               ("cand^3/s = m^3 / time)" if cubic else "elections/s = 1 / time)")}

    if rank == 0:
        head = {"value": value, "unit": UNIT} if cubic else {"value": eps, "unit": "elections/s"}
        e2e_value = world * float(m) ** 3 / e2e_sec if cubic else world / e2e_sec
        line = {"metric": METRIC, **head, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int16x2" if s16 else "int32", "data": "synthetic",
                "config": {"workload": args.workload + ("" if not (args.m or args.n) else f" (m={m}, n={n})"),
                           "detail": WORKLOADS[args.workload]["desc"], "m": m, "n": n, "k": k, "elections_per_step": world,
                           "closure": "16-bit packed" if s16 else "int32",
                           "weights": "margin" if args.margin else "winning votes",
                           "l2": "flushed (512 MiB write) before every timed step"},
                "elections_per_sec": eps,
                "closure_work": {"warm_candidates": nw, "warm_square_updates": float(nw) ** 3,
                                 "warm_square_updates_per_s": world * float(nw) ** 3 / (ms * 1e-3),
                                 "cand3_per_s": value},
                "tally": {"ms_per_step": tally_ms, "algorithmic_GBps": tally_bytes / (tally_ms * 1e-3) / 1e9
                          if tally_ms else None},
                "roofline": roof, "roofline_tally": tally_roof, "roofline_top_kernels": roof_all,
                "warm_candidates": nw,
                "probe_updates_per_s": probe, "kernels": breakdown,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": head["unit"],
                        "h2d_bytes_per_step": int(n) * int(k) * 4, "d2h_bytes_per_step": 2 * int(m) * 4 + 4},
                "gpu_launches": int(launches), "timed_as": "CUDA graph of one schulze_run call, replayed",
                "graph_matches_eager": graph_matches, "device_status": status, "clocks": clock_info}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
