"""Training and evaluation of the winner-proposal network on the GPU.

Host orchestration only: labels come from the library's exact path
(schulze_run: tally, closure, winners), features from schulze_features, and
every training step is one schulze_mlp_train_step (forward, listwise loss,
backward, Adam in the library's kernels). Winner sets never depend on the
model: schulze_winners_fast certifies proposals and falls back to the closure.

Checkpoints are a little-endian binary: magic b"SCHMLP01", int64 step,
int64 seed, int64 parameter count, then params, Adam first and second moments
as float32.
"""
from __future__ import annotations

import struct
import time

import numpy as np
import torch

from . import (NPARAM, context, schulze_features, schulze_mlp_train_step, schulze_run, schulze_winners_fast,
               schulze_strongest_paths, schulze_winners)

MAGIC = b"SCHMLP01"


class Dataset:
    """Per-candidate features and winner labels of many elections, on the GPU,
    packed back to back; seg_off[e] is election e's first candidate."""

    def __init__(self, device="cuda"):
        self.feats, self.labels, self.sizes = [], [], []
        self.device = torch.device(device)

    def add(self, ranks: torch.Tensor, m: int):
        """Tally, solve and featurise one election (ranks: int32 [n, k] on the GPU)."""
        out = schulze_run(ranks, m)
        self.feats.append(schulze_features(out["d"], int(ranks.shape[0])))
        self.labels.append(out["winners"])
        self.sizes.append(m)

    def pack(self):
        X = torch.cat(self.feats)
        y = torch.cat(self.labels)
        seg = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int32)
        return X, y, torch.from_numpy(seg).to(self.device)

    def __len__(self):
        return len(self.sizes)


class Trainer:
    """Adam training state on the GPU (params, moments, step)."""

    def __init__(self, params: np.ndarray, seed: int = 0, device="cuda"):
        assert params.shape == (NPARAM,)
        self.params = torch.from_numpy(np.ascontiguousarray(params, np.float32)).to(device)
        self.m1 = torch.zeros(NPARAM, dtype=torch.float32, device=device)
        self.m2 = torch.zeros(NPARAM, dtype=torch.float32, device=device)
        self.step = 0
        self.seed = seed

    def train(self, data: Dataset, epochs: int, elections_per_step: int = 64, lr: float = 3e-3, log=None):
        """Mini-batches of whole elections in a seeded shuffled order; returns
        the mean loss of each epoch."""
        X, y, seg = data.pack()
        seg_h = seg.cpu().numpy()
        E = len(data)
        rs = np.random.Generator(np.random.PCG64(self.seed))
        history = []
        for ep in range(epochs):
            order = rs.permutation(E)
            tot, cnt = torch.zeros((), device=X.device), 0
            for b0 in range(0, E, elections_per_step):
                idx = np.sort(order[b0:b0 + elections_per_step])
                rows = np.concatenate([np.arange(seg_h[e], seg_h[e + 1]) for e in idx])
                sizes = seg_h[idx + 1] - seg_h[idx]
                sub_seg = torch.from_numpy(np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)).to(X.device)
                rt = torch.from_numpy(rows).to(X.device)
                self.step += 1
                loss, _ = schulze_mlp_train_step(self.params, self.m1, self.m2, self.step,
                                                 X.index_select(0, rt).contiguous(),
                                                 y.index_select(0, rt).contiguous(), sub_seg, lr)
                tot += loss[0]
                cnt += 1
            history.append(float(tot.item()) / max(cnt, 1))
            if log:
                log(f"epoch {ep}: loss {history[-1]:.4f}")
        return history

    def save(self, path: str):
        with open(path, "wb") as f:
            f.write(MAGIC)
            f.write(struct.pack("<qqq", self.step, self.seed, NPARAM))
            for t in (self.params, self.m1, self.m2):
                f.write(t.cpu().numpy().astype("<f4").tobytes())

    @classmethod
    def load(cls, path: str, device="cuda") -> "Trainer":
        with open(path, "rb") as f:
            if f.read(8) != MAGIC:
                raise ValueError("not a proposal-network checkpoint")
            step, seed, npar = struct.unpack("<qqq", f.read(24))
            if npar != NPARAM:
                raise ValueError("parameter count mismatch")
            arrs = [np.frombuffer(f.read(4 * NPARAM), dtype="<f4").astype(np.float32) for _ in range(3)]
        t = cls(arrs[0], seed=seed, device=device)
        t.m1.copy_(torch.from_numpy(arrs[1]))
        t.m2.copy_(torch.from_numpy(arrs[2]))
        t.step = step
        return t


def compare_on(d: torch.Tensor, n: int, params: torch.Tensor | None, top: int = 4, ctx=None):
    """Winners of one election by the full closure and by certified proposals
    (params None: Copeland proposals). Returns a dict with both winner sets,
    the device times in ms and the proposal statistics."""
    ctx = ctx or context(d.device)
    m = d.shape[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p = schulze_strongest_paths(d, n, ctx=ctx)
    w_closure = schulze_winners(p, ctx=ctx)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    w_fast, stats = schulze_winners_fast(d, n, params, top=top, ctx=ctx)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return {"closure_winners": w_closure, "fast_winners": w_fast, "closure_ms": (t1 - t0) * 1e3,
            "fast_ms": (t2 - t1) * 1e3, "stats": stats, "m": m}
