"""CPU oracle for the Schulze hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check of ``__graft_entry__`` and the CPU-baseline leg
of ``bench.py`` may import this package. The product path (the CUDA library
and its Python binding) never calls it and shares no code with it.

The arithmetic lives in ``schulze_oracle.c`` (plain loops, integer only),
compiled here with gcc; ``mlp.py`` holds the float64 reference of the
proposal network. Each function states the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "schulze_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, EDATA = 0, -1, -2, -4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP if the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # SCHULZE_ORACLE_LIB points the tests at a deliberately broken build
            # of this file (mutation checks of the pins); unset in normal use.
            lib = ctypes.CDLL(os.environ.get("SCHULZE_ORACLE_LIB") or build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            lib.oracle_validate.argtypes = [i32p, i64, i32, i32]
            lib.oracle_validate.restype = ctypes.c_int
            lib.oracle_tally.argtypes = [i32p, i64, i32, i32, i32p]
            lib.oracle_tally.restype = ctypes.c_int
            lib.oracle_winners_pregel.argtypes = [i32p, i32, i32p, i32p, i32p]
            lib.oracle_winners_pregel.restype = ctypes.c_int
            lib.oracle_ranking_iterated.argtypes = [i32p, i32, i32, ctypes.c_int, i32p, i32p]
            lib.oracle_ranking_iterated.restype = ctypes.c_int
            lib.oracle_tally_positions.argtypes = [i32p, i64, i32, i32p]
            lib.oracle_tally_positions.restype = ctypes.c_int
            lib.oracle_tally_entry.argtypes = [i32p, i64, i32, i32, i32, i32]
            lib.oracle_tally_entry.restype = i64
            lib.oracle_weights.argtypes = [i32p, i32, i32p]
            lib.oracle_weights_margin.argtypes = [i32p, i32, i32p]
            lib.oracle_closure.argtypes = [i32p, i32, i32p, ctypes.c_int]
            lib.oracle_winners.argtypes = [i32p, i32, i32p]
            lib.oracle_beaten_by.argtypes = [i32p, i32, i32p]
            lib.oracle_ranking.argtypes = [i32p, i32, i32p, i32p]
            lib.oracle_widest_one.argtypes = [i32p, i32, i32, ctypes.c_int, i32p]
            lib.oracle_widest_many.argtypes = [i32p, i32, i32p, i32, ctypes.c_int, i32p, ctypes.c_int]
            for f in (lib.oracle_weights, lib.oracle_weights_margin, lib.oracle_closure, lib.oracle_winners,
                      lib.oracle_beaten_by, lib.oracle_ranking, lib.oracle_widest_one, lib.oracle_widest_many):
                f.restype = None
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _i32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.int32)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


class OracleError(ValueError):
    def __init__(self, code):
        super().__init__({EINVAL: "invalid arguments", ENOMEM: "out of memory",
                          EDATA: "bad ballot (id out of range or repeated)"}.get(code, str(code)))
        self.code = code


def validate(ranks, m: int) -> int:
    r = _i32(ranks)
    n, k = (r.shape if r.ndim == 2 else (0, 0))
    return int(_load().oracle_validate(_p(r), n, m, k))


def tally(ranks, m: int) -> np.ndarray:
    """d[i][j] = number of voters preferring i to j (Sect. 2.1)."""
    r = _i32(ranks)
    if r.ndim != 2:
        raise OracleError(EINVAL)
    n, k = r.shape
    d = np.zeros((m, m), dtype=np.int32)
    rc = _load().oracle_tally(_p(r), n, m, k, _p(d))
    if rc:
        raise OracleError(rc)
    return d


def tally_positions(pos) -> np.ndarray:
    """Weak-order ballots in position form (Sect. 2.1): pos [n, m], smaller
    is better, equal positions tied; d[i][j] = #{v : pos[v][i] < pos[v][j]}."""
    p = _i32(pos)
    if p.ndim != 2:
        raise OracleError(EINVAL)
    n, m = p.shape
    d = np.zeros((m, m), dtype=np.int32)
    rc = _load().oracle_tally_positions(_p(p), n, m, _p(d))
    if rc:
        raise OracleError(rc)
    return d


def tally_entry(ranks, m: int, i: int, j: int) -> int:
    r = _i32(ranks)
    n, k = r.shape
    v = int(_load().oracle_tally_entry(_p(r), n, m, k, int(i), int(j)))
    if v < 0:
        raise OracleError(EINVAL)
    return v


def weights(d) -> np.ndarray:
    """Winning-votes edge weights: w = d where d > d^T, else 0."""
    d = _i32(d)
    m = d.shape[0]
    w = np.empty_like(d)
    _load().oracle_weights(_p(d), m, _p(w))
    return w


def weights_margin(d) -> np.ndarray:
    """The paper's weighted tournament graph: positive margins d - d^T (Sect. 2.1)."""
    d = _i32(d)
    m = d.shape[0]
    w = np.empty_like(d)
    _load().oracle_weights_margin(_p(d), m, _p(w))
    return w


def closure(w, nthreads: int = 1) -> np.ndarray:
    """All-pairs widest-path widths by textbook (max, min) Floyd-Warshall."""
    w = _i32(w)
    m = w.shape[0]
    p = np.empty_like(w)
    _load().oracle_closure(_p(w), m, _p(p), int(nthreads))
    return p


def strongest_paths(d, nthreads: int = 1) -> np.ndarray:
    """p = closure(weights(d)): the widths the Schulze method compares."""
    return closure(weights(d), nthreads)


def winners(p) -> np.ndarray:
    p = _i32(p)
    m = p.shape[0]
    out = np.empty(m, dtype=np.int32)
    _load().oracle_winners(_p(p), m, _p(out))
    return out


def beaten_by(p) -> np.ndarray:
    p = _i32(p)
    m = p.shape[0]
    out = np.empty(m, dtype=np.int32)
    _load().oracle_beaten_by(_p(p), m, _p(out))
    return out


def ranking(p):
    """(order, beaten_by): ids sorted by (beaten_by, id)."""
    p = _i32(p)
    m = p.shape[0]
    order = np.empty(m, dtype=np.int32)
    bb = np.empty(m, dtype=np.int32)
    _load().oracle_ranking(_p(p), m, _p(order), _p(bb))
    return order, bb


def widest_from(w, s: int) -> np.ndarray:
    """Row s of the closure by max-min Dijkstra: out[v] = p(s, v)."""
    w = _i32(w)
    m = w.shape[0]
    out = np.empty(m, dtype=np.int32)
    _load().oracle_widest_one(_p(w), m, int(s), 0, _p(out))
    return out


def widest_to(w, t: int) -> np.ndarray:
    """Column t of the closure by max-min Dijkstra on reversed edges: out[v] = p(v, t)."""
    w = _i32(w)
    m = w.shape[0]
    out = np.empty(m, dtype=np.int32)
    _load().oracle_widest_one(_p(w), m, int(t), 1, _p(out))
    return out


def widest_many(w, sources, transpose: bool = False, nthreads: int = 1) -> np.ndarray:
    """Rows p(s, .) for every s in sources (columns p(., s) with transpose),
    by max-min Dijkstra, sources spread over nthreads: [len(sources), m]."""
    w = _i32(w)
    m = w.shape[0]
    src = np.ascontiguousarray(sources, dtype=np.int32).reshape(-1)
    out = np.empty((src.size, m), dtype=np.int32)
    if src.size:
        _load().oracle_widest_many(_p(w), m, _p(src), int(src.size), int(bool(transpose)), _p(out), int(nthreads))
    return out


def schulze(ranks, m: int, nthreads: int = 1):
    """Whole path for one election: (d, p, winners, order, beaten_by)."""
    d = tally(ranks, m)
    p = strongest_paths(d, nthreads)
    win = winners(p)
    order, bb = ranking(p)
    return d, p, win, order, bb


def ranking_iterated(d, k_top: int | None = None, margin: bool = False):
    """Top-k ranking by iterated winner removal (Sect. 4, closing remark):
    (level [m], number of levels); level 0 = not placed."""
    d = _i32(d)
    m = d.shape[0]
    level = np.zeros(m, dtype=np.int32)
    nl = np.zeros(1, dtype=np.int32)
    rc = _load().oracle_ranking_iterated(_p(d), m, m if k_top is None else int(k_top), int(bool(margin)),
                                         _p(level), _p(nl))
    if rc:
        raise OracleError(rc)
    return level, int(nl[0])


def winners_pregel(w):
    """Winners by the paper's vertex-centric algorithm (Sect. 4, Alg. 1-4) on
    edge weights w: (win [m] 0/1, while-loop iterations, propagation rounds)."""
    w = _i32(w)
    m = w.shape[0]
    win = np.zeros(m, dtype=np.int32)
    it = np.zeros(1, dtype=np.int32)
    rd = np.zeros(1, dtype=np.int32)
    rc = _load().oracle_winners_pregel(_p(w), m, _p(win), _p(it), _p(rd))
    if rc:
        raise OracleError(rc)
    return win, int(it[0]), int(rd[0])
