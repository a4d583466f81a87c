"""Python binding of the GB300 Schulze library (libschulze.so).

Argument marshalling only: every step of the Schulze path runs in the CUDA
kernels behind the C ABI of ``include/schulze.h``. PyTorch supplies device
memory and the current CUDA stream. The functions carry the C names:

    schulze_tally(ranks, m)            -> d        int32 [m, m]
    schulze_strongest_paths(d, bound)  -> p        int32 [m, m]
    schulze_winners(p)                 -> winners  int32 [m] (0/1)
    schulze_ranking(p)                 -> (order, beaten_by)
    schulze_run(ranks, m)              -> dict with all of the above
    schulze_run_host(ranks_np, m)      -> (winners, order) as numpy, host buffers in and out

There is no CPU fallback: importing works without a GPU, but every call
needs the compiled library and a CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libschulze.so")

OK, EINVAL, ENOMEM, ECUDA, EDATA, ETIMEOUT, ERANGE, ETOOBIG = 0, -1, -2, -3, -4, -5, -6, -7
F_AUTO, F_FORCE_S32, F_FORCE_S16, F_TALLY_DENSE, F_TALLY_SPARSE, F_TALLY_GROUPED, F_MARGIN = 0, 1, 2, 4, 8, 16, 32

_lock = threading.Lock()
_lib = None
_ctx = {}

_c = ctypes
_i32, _i64, _u32, _vp = _c.c_int32, _c.c_int64, _c.c_uint32, _c.c_void_p

# (name, restype, argtypes) of every entry point declared in include/schulze.h
SIGNATURES = [
    ("schulze_strerror", _c.c_char_p, [_c.c_int]),
    ("schulze_ctx_create", _c.c_int, [_c.c_int, _c.POINTER(_vp)]),
    ("schulze_ctx_destroy", _c.c_int, [_vp]),
    ("schulze_reserve", _c.c_int, [_vp, _i32, _i64, _i32]),
    ("schulze_workspace_bytes", _c.c_size_t, [_vp]),
    ("schulze_get_status", _c.c_int, [_vp, _c.POINTER(_i32), _vp]),
    ("schulze_set_wait_limit", _c.c_int, [_vp, _i64]),
    ("schulze_tally", _c.c_int, [_vp, _vp, _i64, _i32, _i32, _vp, _u32, _vp]),
    ("schulze_tally_positions", _c.c_int, [_vp, _vp, _i64, _i32, _vp, _vp]),
    ("schulze_ranking_iterated", _c.c_int, [_vp, _vp, _i32, _i64, _i32, _vp, _vp, _u32, _vp]),
    ("schulze_winners_propagation", _c.c_int, [_vp, _vp, _i32, _u32, _vp, _vp, _vp]),
    ("schulze_strongest_paths", _c.c_int, [_vp, _vp, _i32, _i64, _vp, _u32, _vp]),
    ("schulze_winners", _c.c_int, [_vp, _vp, _i32, _vp, _vp]),
    ("schulze_ranking", _c.c_int, [_vp, _vp, _i32, _vp, _vp, _vp]),
    ("schulze_run", _c.c_int, [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _u32, _vp]),
    ("schulze_run_host", _c.c_int, [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _u32, _vp]),
    ("schulze_strongest_paths_static", _c.c_int, [_vp, _i32, _i64, _vp, _u32, _vp, _vp]),
    ("schulze_batch_create", _c.c_int, [_vp, _i32, _vp, _vp, _vp, _c.POINTER(_vp)]),
    ("schulze_batch_destroy", _c.c_int, [_vp]),
    ("schulze_batch_layout", _c.c_int, [_vp, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_i64), _vp, _vp, _vp]),
    ("schulze_batch_run", _c.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("schulze_batch_set_schedule", _c.c_int, [_vp, _i32, _i32]),
    ("schulze_batch_set_bucket_chunk", _c.c_int, [_vp, _i32, _i32]),
    ("schulze_batch_bucket_schedule", _c.c_int, [_vp, _vp, _vp, _vp]),
    ("schulze_batch_set_bucket_tiles", _c.c_int, [_vp, _i32, _i32]),
    ("schulze_batch_run_host", _c.c_int, [_vp, _vp, _vp, _vp, _vp]),
    ("schulze_batch_bucket_tiles", _c.c_int, [_vp, _vp]),
    ("schulze_batch_autotune", _c.c_int, [_vp, _vp, _c.c_char_p, _c.POINTER(_i32), _c.POINTER(_i32), _vp]),
    ("schulze_features", _c.c_int, [_vp, _vp, _i32, _i64, _vp, _vp]),
    ("schulze_mlp_forward", _c.c_int, [_vp, _vp, _vp, _i32, _vp, _vp]),
    ("schulze_mlp_train_step", _c.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i32, _i32, _c.c_float, _vp, _vp,
                                          _vp]),
    ("schulze_certify", _c.c_int, [_vp, _vp, _i32, _i64, _vp, _i32, _vp, _vp, _vp]),
    ("schulze_winners_fast", _c.c_int, [_vp, _vp, _i32, _i64, _vp, _i32, _vp, _vp, _vp]),
    # include/schulze_profile.h
    ("schulze_profile_enable", _c.c_int, [_vp, _c.c_int]),
    ("schulze_profile_read", _c.c_int, [_vp, _vp, _c.c_int, _c.POINTER(_c.c_int)]),
    ("schulze_launch_count", _i64, [_vp]),
    ("schulze_closure_counters", _c.c_int, [_vp, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_i64)]),
    ("schulze_probe_minmax", _c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.POINTER(_c.c_double),
                                        _c.POINTER(_c.c_double)]),
]


class _KernelStats(ctypes.Structure):
    _fields_ = [("name", _c.c_char * 32), ("launches", _i64), ("ms", _c.c_double), ("work", _c.c_double)]


class SchulzeError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = load().schulze_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


def load():
    """Load libschulze.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                                   "(there is no CPU fallback)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(lib, name)
                f.restype, f.argtypes = res, args
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        raise SchulzeError(rc, what)


class Context:
    """One library context (workspace + device status word) per device."""

    def __init__(self, device: int):
        lib = load()
        h = _vp()
        _check(lib.schulze_ctx_create(int(device), ctypes.byref(h)), "schulze_ctx_create")
        self.handle, self.device, self._lib = h, int(device), lib

    def reserve(self, m_max: int, n_max: int, k_max: int):
        _check(self._lib.schulze_reserve(self.handle, m_max, n_max, k_max), "schulze_reserve")

    def workspace_bytes(self) -> int:
        return int(self._lib.schulze_workspace_bytes(self.handle))

    def status(self, stream=None) -> int:
        st = _i32(0)
        _check(self._lib.schulze_get_status(self.handle, ctypes.byref(st), _stream(stream, self.device)),
               "schulze_get_status")
        return int(st.value)

    def set_wait_limit(self, cycles: int):
        """Clock-cycle bound on each device-side wait of the persistent closure."""
        _check(self._lib.schulze_set_wait_limit(self.handle, int(cycles)), "schulze_set_wait_limit")

    def profile(self, enable: bool = True):
        """Start (clearing) or stop per-kernel event timing of this context."""
        _check(self._lib.schulze_profile_enable(self.handle, 1 if enable else 0), "schulze_profile_enable")

    def profile_read(self) -> dict:
        """{kernel class: {"launches", "ms", "work"}} accumulated since profile()."""
        buf = (_KernelStats * 64)()
        cnt = _c.c_int(0)
        _check(self._lib.schulze_profile_read(self.handle, buf, 64, ctypes.byref(cnt)), "schulze_profile_read")
        return {buf[i].name.decode(): {"launches": int(buf[i].launches), "ms": float(buf[i].ms),
                                       "work": float(buf[i].work)} for i in range(min(cnt.value, 64))}

    def launch_count(self) -> int:
        return int(self._lib.schulze_launch_count(self.handle))

    def closure_counters(self) -> dict:
        """Cumulative closure work: tile updates, diagonal closures, queue items."""
        t, dg, it = _i64(0), _i64(0), _i64(0)
        _check(self._lib.schulze_closure_counters(self.handle, ctypes.byref(t), ctypes.byref(dg), ctypes.byref(it)),
               "schulze_closure_counters")
        return {"tile_updates": t.value, "diag_closures": dg.value, "items": it.value}

    def __del__(self):
        try:
            if self.handle:
                self._lib.schulze_ctx_destroy(self.handle)
        except Exception:
            pass


def context(device=None) -> Context:
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    if dev not in _ctx:
        _ctx[dev] = Context(dev)
    return _ctx[dev]


# the current stream's raw handle without building a torch Stream object
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


def _stream(stream, device):
    if stream is None:
        if _raw_stream is not None and isinstance(device, int):
            return _vp(_raw_stream(device))
        stream = torch.cuda.current_stream(device)
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_i32(t: torch.Tensor, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.int32:
        raise ValueError(f"{name} must be int32")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _out(t, shape, device, name):
    if t is None:
        return torch.empty(shape, dtype=torch.int32, device=device)
    return _dev_i32(t, name, shape)


def _ptr(t):
    return _vp(t.data_ptr()) if t is not None else None


def schulze_tally(ranks: torch.Tensor, m: int, d: torch.Tensor | None = None, flags: int = 0,
                  ctx: Context | None = None, stream=None) -> torch.Tensor:
    """d[i][j] = #ballots preferring i to j; ranks int32 [n, k] on the GPU."""
    ranks = _dev_i32(ranks, "ranks")
    if ranks.dim() != 2:
        raise ValueError("ranks must be [n, k]")
    ctx = ctx or context(ranks.device)
    n, k = ranks.shape
    d = _out(d, (m, m), ranks.device, "d")
    _check(load().schulze_tally(ctx.handle, _ptr(ranks), n, m, k, _ptr(d), flags, _stream(stream, ctx.device)),
           "schulze_tally")
    return d


def schulze_tally_positions(pos: torch.Tensor, d: torch.Tensor | None = None, ctx: Context | None = None,
                            stream=None) -> torch.Tensor:
    """Weak-order ballots: pos int32 [n, m] on the GPU (smaller is better,
    equal is tied); d[i][j] = #{v : pos[v][i] < pos[v][j]}."""
    pos = _dev_i32(pos, "pos")
    if pos.dim() != 2:
        raise ValueError("pos must be [n, m]")
    ctx = ctx or context(pos.device)
    n, m = pos.shape
    d = _out(d, (m, m), pos.device, "d")
    _check(load().schulze_tally_positions(ctx.handle, _ptr(pos), n, m, _ptr(d), _stream(stream, ctx.device)),
           "schulze_tally_positions")
    return d


def schulze_strongest_paths(d: torch.Tensor, bound: int, p: torch.Tensor | None = None, flags: int = 0,
                            ctx: Context | None = None, stream=None) -> torch.Tensor:
    """Widest-path widths with winning-votes edge weights; bound >= max(d)."""
    d = _dev_i32(d, "d")
    m = d.shape[0]
    _dev_i32(d, "d", (m, m))
    ctx = ctx or context(d.device)
    p = _out(p, (m, m), d.device, "p")
    _check(load().schulze_strongest_paths(ctx.handle, _ptr(d), m, int(bound), _ptr(p), flags,
                                          _stream(stream, ctx.device)), "schulze_strongest_paths")
    return p


def schulze_winners(p: torch.Tensor, winners: torch.Tensor | None = None, ctx: Context | None = None,
                    stream=None) -> torch.Tensor:
    p = _dev_i32(p, "p")
    m = p.shape[0]
    _dev_i32(p, "p", (m, m))
    ctx = ctx or context(p.device)
    winners = _out(winners, (m,), p.device, "winners")
    _check(load().schulze_winners(ctx.handle, _ptr(p), m, _ptr(winners), _stream(stream, ctx.device)),
           "schulze_winners")
    return winners


def schulze_ranking(p: torch.Tensor, order: torch.Tensor | None = None, beaten_by: torch.Tensor | None = None,
                    ctx: Context | None = None, stream=None):
    p = _dev_i32(p, "p")
    m = p.shape[0]
    _dev_i32(p, "p", (m, m))
    ctx = ctx or context(p.device)
    order = _out(order, (m,), p.device, "order")
    beaten_by = _out(beaten_by, (m,), p.device, "beaten_by")
    _check(load().schulze_ranking(ctx.handle, _ptr(p), m, _ptr(order), _ptr(beaten_by),
                                  _stream(stream, ctx.device)), "schulze_ranking")
    return order, beaten_by


def schulze_run(ranks: torch.Tensor, m: int, flags: int = 0, out: dict | None = None, ctx: Context | None = None,
                stream=None) -> dict:
    """Tally, widest paths, winners and ranking for one election."""
    ranks = _dev_i32(ranks, "ranks")
    n, k = ranks.shape
    ctx = ctx or context(ranks.device)
    out = out or {}
    dev = ranks.device
    d = _out(out.get("d"), (m, m), dev, "d")
    p = _out(out.get("p"), (m, m), dev, "p")
    w = _out(out.get("winners"), (m,), dev, "winners")
    o = _out(out.get("order"), (m,), dev, "order")
    b = _out(out.get("beaten_by"), (m,), dev, "beaten_by")
    _check(load().schulze_run(ctx.handle, _ptr(ranks), n, m, k, _ptr(d), _ptr(p), _ptr(w), _ptr(o), _ptr(b),
                              flags, _stream(stream, ctx.device)), "schulze_run")
    return {"d": d, "p": p, "winners": w, "order": o, "beaten_by": b}


def schulze_strongest_paths_static(d: torch.Tensor, bound: int, p: torch.Tensor | None = None, flags: int = 0,
                                   status: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Widest paths without any device allocation inside the library, for
    callers that cannot allocate device memory (m <= 1024; scratch is a fixed
    array in the library). Calls must not overlap on the GPU.

    `status`: a zeroed device int32 [1] that receives data errors (EDATA,
    ETIMEOUT) asynchronously; the caller reads it and treats p as unspecified
    when it is nonzero. Without one, this wrapper makes its own status word,
    waits for the stream and raises SchulzeError on an error, so that a bad
    count or a timed-out wait is never returned silently."""
    d = _dev_i32(d, "d")
    m = d.shape[0]
    _dev_i32(d, "d", (m, m))
    p = _out(p, (m, m), d.device, "p")
    own = status is None
    if own:
        status = torch.zeros(1, dtype=torch.int32, device=d.device)
    else:
        _dev_i32(status, "status", (1,))
    with torch.cuda.device(d.device):
        _check(load().schulze_strongest_paths_static(_ptr(d), m, int(bound), _ptr(p), flags, _ptr(status),
                                                     _stream(stream, d.device)), "schulze_strongest_paths_static")
    if own:
        code = int(status.item())  # waits for the current stream
        if code != OK:
            raise SchulzeError(code, "schulze_strongest_paths_static (device status)")
    return p


def schulze_ranking_iterated(d: torch.Tensor, bound: int, k_top: int | None = None, flags: int = 0,
                             level: torch.Tensor | None = None, ctx: Context | None = None, stream=None):
    """Top-k ranking by iterated winner removal: (level int32 [m] on the
    GPU, 0 = not placed; number of levels)."""
    d = _dev_i32(d, "d")
    m = d.shape[0]
    _dev_i32(d, "d", (m, m))
    ctx = ctx or context(d.device)
    level = _out(level, (m,), d.device, "level")
    nl = _c.c_int32(0)
    _check(load().schulze_ranking_iterated(ctx.handle, _ptr(d), m, int(bound), m if k_top is None else int(k_top),
                                           _ptr(level), _c.byref(nl), flags, _stream(stream, ctx.device)),
           "schulze_ranking_iterated")
    return level, int(nl.value)


def schulze_winners_propagation(d: torch.Tensor, flags: int = 0, winners: torch.Tensor | None = None,
                                ctx: Context | None = None, stream=None):
    """Winners by the paper's vertex-centric algorithm (Alg. 1-4) on the
    tally: (winners int32 [m] on the GPU, [iterations, rounds])."""
    d = _dev_i32(d, "d")
    m = d.shape[0]
    _dev_i32(d, "d", (m, m))
    ctx = ctx or context(d.device)
    winners = _out(winners, (m,), d.device, "winners")
    stats = (_i32 * 2)()
    _check(load().schulze_winners_propagation(ctx.handle, _ptr(d), m, flags, _ptr(winners), stats,
                                              _stream(stream, ctx.device)), "schulze_winners_propagation")
    return winners, list(stats)


NPARAM = 5313  # MLP parameters: W1 [64][16], b1 [64], W2 [64][64], b2 [64], W3 [64], b3


def _dev_f32(t: torch.Tensor, name: str, numel=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements")
    return t


def schulze_features(d: torch.Tensor, n: int, feat: torch.Tensor | None = None, ctx: Context | None = None,
                     stream=None) -> torch.Tensor:
    """16 float32 features per candidate from the tally d (see include/schulze.h)."""
    d = _dev_i32(d, "d")
    m = d.shape[0]
    ctx = ctx or context(d.device)
    feat = torch.empty((m, 16), dtype=torch.float32, device=d.device) if feat is None else _dev_f32(feat, "feat")
    _check(load().schulze_features(ctx.handle, _ptr(d), m, int(n), _ptr(feat), _stream(stream, ctx.device)),
           "schulze_features")
    return feat


def schulze_mlp_forward(params: torch.Tensor, feat: torch.Tensor, score: torch.Tensor | None = None,
                        ctx: Context | None = None, stream=None) -> torch.Tensor:
    params = _dev_f32(params, "params", NPARAM)
    feat = _dev_f32(feat, "feat")
    N = feat.shape[0]
    ctx = ctx or context(feat.device)
    score = torch.empty(N, dtype=torch.float32, device=feat.device) if score is None else _dev_f32(score, "score")
    _check(load().schulze_mlp_forward(ctx.handle, _ptr(params), _ptr(feat), N, _ptr(score),
                                      _stream(stream, ctx.device)), "schulze_mlp_forward")
    return score


def schulze_mlp_train_step(params, adam_m, adam_v, step: int, feat, label, seg_off, lr: float, loss=None, grad=None,
                           ctx: Context | None = None, stream=None):
    """One forward/backward/Adam step in place; returns (loss, grad) device tensors."""
    params = _dev_f32(params, "params", NPARAM)
    adam_m = _dev_f32(adam_m, "adam_m", NPARAM)
    adam_v = _dev_f32(adam_v, "adam_v", NPARAM)
    feat = _dev_f32(feat, "feat")
    label = _dev_i32(label, "label")
    seg_off = _dev_i32(seg_off, "seg_off")
    N, nseg = feat.shape[0], seg_off.numel() - 1
    ctx = ctx or context(feat.device)
    loss = torch.empty(1, dtype=torch.float32, device=feat.device) if loss is None else _dev_f32(loss, "loss", 1)
    grad = torch.empty(NPARAM, dtype=torch.float32, device=feat.device) if grad is None else \
        _dev_f32(grad, "grad", NPARAM)
    _check(load().schulze_mlp_train_step(ctx.handle, _ptr(params), _ptr(adam_m), _ptr(adam_v), int(step), _ptr(feat),
                                         _ptr(label), _ptr(seg_off), nseg, N, float(lr), _ptr(loss), _ptr(grad),
                                         _stream(stream, ctx.device)), "schulze_mlp_train_step")
    return loss, grad


def schulze_certify(d: torch.Tensor, n: int, cand: torch.Tensor, winners: torch.Tensor | None = None,
                    ctx: Context | None = None, stream=None):
    """(winners, result) for proposals cand (device int32); result[0] == 1 means exact."""
    d = _dev_i32(d, "d")
    m = d.shape[0]
    cand = _dev_i32(cand, "cand")
    ctx = ctx or context(d.device)
    winners = _out(winners, (m,), d.device, "winners")
    result = torch.empty(4, dtype=torch.int32, device=d.device)
    _check(load().schulze_certify(ctx.handle, _ptr(d), m, int(n), _ptr(cand), cand.numel(), _ptr(winners),
                                  _ptr(result), _stream(stream, ctx.device)), "schulze_certify")
    return winners, result


def schulze_winners_fast(d: torch.Tensor, n: int, params: torch.Tensor | None = None, top: int = 4,
                         winners: torch.Tensor | None = None, ctx: Context | None = None, stream=None):
    """Exact winners via certified proposals (MLP, or Copeland when params is
    None); returns (winners, stats) with stats = [certified proposal index or
    -1, fallback (0 none, 1 closure, 2 the paper's propagation for warm sets
    above 2048), ties checked, relaxation rounds]."""
    d = _dev_i32(d, "d")
    m = d.shape[0]
    if params is not None:
        params = _dev_f32(params, "params", NPARAM)
    ctx = ctx or context(d.device)
    winners = _out(winners, (m,), d.device, "winners")
    stats = (_i32 * 4)()
    _check(load().schulze_winners_fast(ctx.handle, _ptr(d), m, int(n), _ptr(params), int(top), _ptr(winners), stats,
                                       _stream(stream, ctx.device)), "schulze_winners_fast")
    return winners, list(stats)


class SchulzeBatch:
    """A planned batch of independent elections (schulze_batch_create).

    n, m, k: host int arrays of length E. Ballots and outputs are packed back
    to back in this order; `ranks_off`, `mat_off`, `vec_off` give each
    election's element offsets and `ranks_elems`, `mat_elems`, `vec_elems`
    the totals."""

    def __init__(self, n, m, k, ctx: Context | None = None):
        lib = load()
        self.ctx = ctx or context()
        n, m, k = (np.ascontiguousarray(x, dtype=np.int32) for x in (n, m, k))
        self.E = int(n.shape[0])
        h = _vp()
        _check(lib.schulze_batch_create(self.ctx.handle, self.E, _vp(n.ctypes.data), _vp(m.ctypes.data),
                                        _vp(k.ctypes.data), ctypes.byref(h)), "schulze_batch_create")
        self.handle, self._lib = h, lib
        self.n, self.m, self.k = n, m, k
        tr, tm, tv = _i64(0), _i64(0), _i64(0)
        self.ranks_off = np.zeros(self.E, np.int64)
        self.mat_off = np.zeros(self.E, np.int64)
        self.vec_off = np.zeros(self.E, np.int64)
        _check(lib.schulze_batch_layout(h, ctypes.byref(tr), ctypes.byref(tm), ctypes.byref(tv),
                                        _vp(self.ranks_off.ctypes.data), _vp(self.mat_off.ctypes.data),
                                        _vp(self.vec_off.ctypes.data)), "schulze_batch_layout")
        self.ranks_elems, self.mat_elems, self.vec_elems = tr.value, tm.value, tv.value

    def run(self, ranks: torch.Tensor, d=None, p=None, winners=None, order=None, beaten_by=None, stream=None):
        """Run every election; outputs are optional flat int32 device tensors."""
        ranks = _dev_i32(ranks, "ranks")
        if ranks.numel() < self.ranks_elems:
            raise ValueError("ranks is smaller than the plan's ballots")
        for t, size, name in ((d, self.mat_elems, "d"), (p, self.mat_elems, "p"), (winners, self.vec_elems, "winners"),
                              (order, self.vec_elems, "order"), (beaten_by, self.vec_elems, "beaten_by")):
            if t is not None and (_dev_i32(t, name).numel() < size):
                raise ValueError(f"{name} is smaller than the plan's layout")
        _check(self._lib.schulze_batch_run(self.handle, _ptr(ranks), _ptr(d), _ptr(p), _ptr(winners), _ptr(order),
                                           _ptr(beaten_by), _stream(stream, self.ctx.device)), "schulze_batch_run")

    def run_host(self, ranks, winners=None, order=None, stream=None):
        """Run every election from host buffers (schulze_batch_run_host): ranks a
        contiguous int32 CPU tensor or array in the plan's layout (pinned memory
        copies fastest); winners / order host int32 buffers of vec_elems (made
        when None). Returns (winners, order) once they are on the host."""
        def host_ptr(a, name, size):
            if isinstance(a, torch.Tensor):
                if a.is_cuda or a.dtype != torch.int32 or not a.is_contiguous() or a.numel() < size:
                    raise ValueError(f"{name} must be a contiguous int32 CPU tensor of at least {size} elements")
                return a.data_ptr()
            if a.dtype != np.int32 or not a.flags.c_contiguous or a.size < size:
                raise ValueError(f"{name} must be a contiguous int32 array of at least {size} elements")
            return a.ctypes.data
        rptr = host_ptr(ranks, "ranks", self.ranks_elems)
        winners = np.empty(self.vec_elems, np.int32) if winners is None else winners
        order = np.empty(self.vec_elems, np.int32) if order is None else order
        wptr, optr = host_ptr(winners, "winners", self.vec_elems), host_ptr(order, "order", self.vec_elems)
        _check(self._lib.schulze_batch_run_host(self.handle, _vp(rptr), _vp(wptr), _vp(optr),
                                                _stream(stream, self.ctx.device)), "schulze_batch_run_host")
        return winners, order

    def set_schedule(self, tally_policy: int, order_policy: int):
        _check(self._lib.schulze_batch_set_schedule(self.handle, tally_policy, order_policy),
               "schulze_batch_set_schedule")

    def set_bucket_chunk(self, bucket: int, chunk: int):
        """Ballots staged per tally step for the elections of one m-bucket."""
        _check(self._lib.schulze_batch_set_bucket_chunk(self.handle, int(bucket), int(chunk)),
               "schulze_batch_set_bucket_chunk")

    def bucket_schedule(self):
        """[(largest m of the bucket, ballots per step, elections in it)] for the five m-buckets."""
        mx, ch, el = (_i32 * 5)(), (_i32 * 5)(), (_i32 * 5)()
        _check(self._lib.schulze_batch_bucket_schedule(self.handle, mx, ch, el), "schulze_batch_bucket_schedule")
        return [(mx[q], ch[q], el[q]) for q in range(5)]

    def set_bucket_tiles(self, bucket: int, groups_per_tile: int):
        """Tile groups (1, 2 or 4) sharing one tally tile for the elections of one m-bucket."""
        _check(self._lib.schulze_batch_set_bucket_tiles(self.handle, int(bucket), int(groups_per_tile)),
               "schulze_batch_set_bucket_tiles")

    def bucket_tiles(self):
        """Groups per tally tile of the five m-buckets."""
        g = (_i32 * 5)()
        _check(self._lib.schulze_batch_bucket_tiles(self.handle, g), "schulze_batch_bucket_tiles")
        return [g[q] for q in range(5)]

    def autotune(self, ranks: torch.Tensor, cache_path: str | None = None, stream=None):
        """Pick the fastest schedule for this batch; returns (tally_policy, order_policy)."""
        ranks = _dev_i32(ranks, "ranks")
        bt, bo = _i32(-1), _i32(-1)
        _check(self._lib.schulze_batch_autotune(self.handle, _ptr(ranks),
                                                cache_path.encode() if cache_path else None, ctypes.byref(bt),
                                                ctypes.byref(bo), _stream(stream, self.ctx.device)),
               "schulze_batch_autotune")
        return bt.value, bo.value

    def __del__(self):
        try:
            if self.handle:
                self._lib.schulze_batch_destroy(self.handle)
        except Exception:
            pass


def probe_minmax(kind: int, blocks: int, iters: int, device: int = 0):
    """(seconds, updates) of the integer min/max issue-rate probe; kind 0 int32,
    1 packed int16x2, 2 packed int16x2 with a three-input max."""
    sec, upd = _c.c_double(0), _c.c_double(0)
    _check(load().schulze_probe_minmax(device, kind, blocks, iters, ctypes.byref(sec), ctypes.byref(upd)),
           "schulze_probe_minmax")
    return sec.value, upd.value


def schulze_run_host(ranks: np.ndarray, m: int, flags: int = 0, winners: np.ndarray | None = None,
                     order: np.ndarray | None = None, device=None, stream=None):
    """Host buffers in and out (pinned or pageable numpy/torch CPU memory)."""
    if isinstance(ranks, torch.Tensor):
        if ranks.is_cuda or ranks.dtype != torch.int32 or not ranks.is_contiguous():
            raise ValueError("ranks must be a contiguous int32 CPU tensor")
        rptr, (n, k) = ranks.data_ptr(), ranks.shape
    else:
        if ranks.dtype != np.int32 or not ranks.flags.c_contiguous:
            raise ValueError("ranks must be a contiguous int32 array")
        rptr, (n, k) = ranks.ctypes.data, ranks.shape
    ctx = context(device)
    winners = np.empty(m, np.int32) if winners is None else winners
    order = np.empty(m, np.int32) if order is None else order
    wptr = winners.data_ptr() if isinstance(winners, torch.Tensor) else winners.ctypes.data
    optr = order.data_ptr() if isinstance(order, torch.Tensor) else order.ctypes.data
    _check(ctx._lib.schulze_run_host(ctx.handle, _vp(rptr), n, m, k, _vp(wptr), _vp(optr), flags,
                                     _stream(stream, ctx.device)), "schulze_run_host")
    return winners, order
