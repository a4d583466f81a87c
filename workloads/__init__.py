"""Seeded synthetic preference profiles (the only code the CUDA path and the
CPU oracle both use).

Nothing here computes any part of the Schulze method: the functions only draw
ballots. A ballot array is int32 [n, k], row-major; row v lists candidate ids
best first (distinct, 0 <= id < m). k == m is a full ranking; with k < m the
unlisted candidates are tied below all listed ones.

The named workloads follow the five evaluation settings of the build:

* ``small_mallows``   m=64, n=1000, full rankings, Mallows phi=0.8, identity reference
* ``large_topk``      m=4096, n=20000, top-50, Mallows phi=0.9, random reference
* ``huge_pl``         m=16384, n=200000, top-20, Plackett-Luce with Zipf(1.1) weights
* ``batch_mixed``     E elections, m~U[8,512], n~U[50,5000], half Mallows / half IC
* ``learned_train`` / ``learned_eval``  top-k Mallows elections for the proposal model

The paper evaluates on Spotify chart data (Sect. 5.1, Table 1), which is not
available; these synthetic profiles stand in for it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgen.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 20260


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so next to it (plain gcc, no -march)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gen_permutation.argtypes = [ctypes.c_uint64, ctypes.c_int32, i32p]
            lib.gen_permutation.restype = None
            lib.gen_impartial.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                          i32p, ctypes.c_int]
            lib.gen_mallows.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_double, i32p, i32p, ctypes.c_int]
            lib.gen_plackett_luce_zipf.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_double, i32p, i32p, ctypes.c_int]
            lib.gen_batch.argtypes = [ctypes.c_uint64, ctypes.c_int32, i32p, i32p, i32p, i32p,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32p, ctypes.c_int]
            for f in (lib.gen_impartial, lib.gen_mallows, lib.gen_plackett_luce_zipf, lib.gen_batch):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None else None


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def permutation(seed: int, m: int) -> np.ndarray:
    out = np.empty(m, dtype=np.int32)
    _load().gen_permutation(seed, m, _ptr(out))
    return out


def impartial(seed: int, n: int, m: int, k: int | None = None, out=None, nthreads=None) -> np.ndarray:
    k = m if k is None else k
    out = np.empty((n, k), dtype=np.int32) if out is None else out
    rc = _load().gen_impartial(seed, n, m, k, _ptr(out), _threads(nthreads))
    if rc:
        raise ValueError("gen_impartial: bad arguments")
    return out


def mallows(seed: int, n: int, m: int, k: int | None = None, phi: float = 1.0, sigma0=None, out=None,
            nthreads=None) -> np.ndarray:
    """Mallows(phi) ballots around reference order sigma0 (None = identity)."""
    k = m if k is None else k
    out = np.empty((n, k), dtype=np.int32) if out is None else out
    s0 = None if sigma0 is None else np.ascontiguousarray(sigma0, dtype=np.int32)
    rc = _load().gen_mallows(seed, n, m, k, float(phi), _ptr(s0), _ptr(out), _threads(nthreads))
    if rc:
        raise ValueError("gen_mallows: bad arguments")
    return out


def plackett_luce_zipf(seed: int, n: int, m: int, k: int, s: float = 1.1, perm=None, out=None,
                       nthreads=None) -> np.ndarray:
    out = np.empty((n, k), dtype=np.int32) if out is None else out
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    rc = _load().gen_plackett_luce_zipf(seed, n, m, k, float(s), _ptr(pm), _ptr(out), _threads(nthreads))
    if rc:
        raise ValueError("gen_plackett_luce_zipf: bad arguments")
    return out


# ------------------------------------------------------------ named workloads

@dataclass
class Election:
    ranks: np.ndarray  # int32 [n, k]
    m: int
    label: str = ""

    @property
    def n(self) -> int:
        return int(self.ranks.shape[0])

    @property
    def k(self) -> int:
        return int(self.ranks.shape[1])


def small_mallows(seed: int = SEED_BASE + 0) -> Election:
    """m=64, n=1000, full rankings, Mallows phi=0.8 around the identity."""
    return Election(mallows(seed, 1000, 64, 64, 0.8), 64, "mallows-full m=64 n=1000 phi=0.8")


def large_topk(seed: int = SEED_BASE + 1, n: int = 20000, m: int = 4096, k: int = 50) -> Election:
    """m=4096, n=20000, top-50 Mallows phi=0.9 around a seeded random reference."""
    sigma0 = permutation(seed ^ 0x5151, m)
    return Election(mallows(seed, n, m, k, 0.9, sigma0), m, f"mallows-top{k} m={m} n={n} phi=0.9")


def huge_pl(seed: int = SEED_BASE + 2, n: int = 200000, m: int = 16384, k: int = 20) -> Election:
    """m=16384, n=200000, top-20 Plackett-Luce, Zipf(1.1) weights on a seeded id permutation."""
    perm = permutation(seed ^ 0x7A7A, m)
    return Election(plackett_luce_zipf(seed, n, m, k, 1.1, perm), m, f"pl-zipf1.1-top{k} m={m} n={n}")


def popular_subsample(m: int, size: int, seed: int = SEED_BASE + 2) -> np.ndarray:
    """The `size` highest-weight candidate ids of ``huge_pl`` (its Zipf order)."""
    perm = permutation(seed ^ 0x7A7A, m)
    return np.sort(perm[:size]).astype(np.int64)


def spotify_like(seed: int = SEED_BASE + 8, n: int = 15553, m: int = 18407, k: int = 200) -> Election:
    """Shaped like the paper's largest Spotify profile (Sect. 5.1: about 18.4k
    candidates, 15.5k voters, top-200 lists): top-200 Plackett-Luce with
    Zipf(1.1) weights on a seeded id permutation. Synthetic; no item of any
    data set is reproduced."""
    perm = permutation(seed ^ 0x5B5B, m)
    return Election(plackett_luce_zipf(seed, n, m, k, 1.1, perm), m, f"pl-zipf1.1-top{k} m={m} n={n}")


def spotify_popular(m: int, size: int, seed: int = SEED_BASE + 8) -> np.ndarray:
    """The `size` highest-weight candidate ids of ``spotify_like``."""
    perm = permutation(seed ^ 0x5B5B, m)
    return np.sort(perm[:size]).astype(np.int64)


@dataclass
class Batch:
    """E independent elections packed back to back."""
    ranks: np.ndarray      # int32, all ballots concatenated
    n: np.ndarray          # int32 [E]
    m: np.ndarray          # int32 [E]
    k: np.ndarray          # int32 [E]
    ranks_off: np.ndarray  # int64 [E] element offset of each election's ballots
    kind: list

    @property
    def E(self) -> int:
        return int(self.n.shape[0])

    def election(self, e: int) -> Election:
        n, m, k = int(self.n[e]), int(self.m[e]), int(self.k[e])
        off = int(self.ranks_off[e])
        return Election(self.ranks[off:off + n * k].reshape(n, k), m, self.kind[e])


def batch_mixed(E: int = 4096, seed: int = SEED_BASE + 3, m_range=(8, 512), n_range=(50, 5000),
                nthreads=None) -> Batch:
    """E elections, m ~ U[8,512], n ~ U[50,5000], full rankings; even e: Mallows
    (phi ~ U[0.5, 1.0], random reference), odd e: impartial culture."""
    rs = np.random.Generator(np.random.PCG64(seed))
    m = rs.integers(m_range[0], m_range[1] + 1, size=E).astype(np.int32)
    n = rs.integers(n_range[0], n_range[1] + 1, size=E).astype(np.int32)
    phi = rs.uniform(0.5, 1.0, size=E)
    k = m.copy()
    kind = (np.arange(E) % 2).astype(np.int32)  # 0 Mallows, 1 impartial culture
    sizes = n.astype(np.int64) * k.astype(np.int64)
    off = np.zeros(E, dtype=np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    ranks = np.empty(int(sizes.sum()), dtype=np.int32)
    rc = _load().gen_batch(seed, E, _ptr(kind), _ptr(n), _ptr(m), _ptr(k),
                           phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(ranks), _threads(nthreads))
    if rc:
        raise ValueError("gen_batch: bad arguments")
    labels = [f"mallows phi={phi[e]:.3f}" if kind[e] == 0 else "ic" for e in range(E)]
    return Batch(ranks, n, m, k, off, labels)


def learned_elections(E: int, seed: int, m_range, n_range, k_range, phi_range, nthreads=None) -> Batch:
    """Top-k Mallows elections with per-election m, n, k, phi drawn uniformly."""
    rs = np.random.Generator(np.random.PCG64(seed))
    m = rs.integers(m_range[0], m_range[1] + 1, size=E).astype(np.int32)
    n = rs.integers(n_range[0], n_range[1] + 1, size=E).astype(np.int32)
    k = np.minimum(rs.integers(k_range[0], k_range[1] + 1, size=E), m).astype(np.int32)
    phi = rs.uniform(phi_range[0], phi_range[1], size=E)
    sizes = n.astype(np.int64) * k.astype(np.int64)
    off = np.zeros(E, dtype=np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    ranks = np.empty(int(sizes.sum()), dtype=np.int32)
    kind = []
    for e in range(E):
        view = ranks[off[e]:off[e] + sizes[e]].reshape(int(n[e]), int(k[e]))
        es = seed * 1000003 + e
        sigma0 = permutation(es ^ 0x44, int(m[e]))
        mallows(es, int(n[e]), int(m[e]), int(k[e]), float(phi[e]), sigma0, out=view, nthreads=nthreads)
        kind.append(f"mallows-top{k[e]} phi={phi[e]:.3f}")
    return Batch(ranks, n, m, k, off, kind)


def learned_train(E: int = 20000, seed: int = SEED_BASE + 4, **kw) -> Batch:
    """Training set: m~U[256,2048], n~U[1000,20000], k~U[10,100], phi~U[0.6,1.0]."""
    return learned_elections(E, seed, (256, 2048), (1000, 20000), (10, 100), (0.6, 1.0), **kw)


def learned_eval(E: int = 256, seed: int = SEED_BASE + 5, m: int = 8192, n: int = 20000, k: int = 50,
                 phi: float = 0.9, **kw) -> Batch:
    """Evaluation set: E elections of m=8192, n=20000, top-50 Mallows phi=0.9."""
    return learned_elections(E, seed, (m, m), (n, n), (k, k), (phi, phi), **kw)


def weak_orders(seed: int = SEED_BASE + 7, n: int = 20000, m: int = 1024, tier: int = 16,
                phi: float = 0.97) -> np.ndarray:
    """Weak-order ballots in position form, int32 [n, m]: a full Mallows(phi)
    ranking around a seeded random reference order, cut into tiers of `tier`
    consecutive places (tied inside a tier): pos[v][c] = place of c // tier."""
    r = mallows(seed, n, m, m, phi, permutation(seed ^ 0x5A, m))
    pos = np.empty((n, m), dtype=np.int32)
    rows = np.arange(n)[:, None]
    pos[rows, r] = (np.arange(m, dtype=np.int32) // tier)[None, :]
    return pos


def mlp_init(seed: int = SEED_BASE + 6) -> np.ndarray:
    """Initial weights of the 16-64-64-1 proposal network (5313 float32):
    He-normal weights, zero biases; a seeded draw, fed to both the GPU
    training and its float64 reference."""
    rs = np.random.Generator(np.random.PCG64(seed))
    theta = np.zeros(5313)
    theta[0:1024] = rs.normal(0, np.sqrt(2.0 / 16), 1024)
    theta[1088:5184] = rs.normal(0, np.sqrt(2.0 / 64), 4096)
    theta[5248:5312] = rs.normal(0, np.sqrt(1.0 / 64), 64)
    return theta.astype(np.float32)
