"""schulze_strongest_paths_static: widest paths for callers that cannot
allocate device memory (their device memory belongs to another allocator, or
they may not allocate once set up). Its scratch is a fixed array inside the
library, so it must give exactly what schulze_strongest_paths gives, call
after call, although every call reuses the array the previous one left behind.

The file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_12976_gb300 as S
    clib = ctypes.CDLL(S.LIB_PATH)
    f = clib.schulze_strongest_paths_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint32,
                  ctypes.c_void_p, ctypes.c_void_p]
    return S, f


def _call(f, d, bound, flags=0, status=None):
    m = d.shape[0]
    p = torch.full((m, m), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(ctypes.c_void_p(d.data_ptr()), m, bound, ctypes.c_void_p(p.data_ptr()), flags,
           ctypes.c_void_p(status.data_ptr()) if status is not None else None, ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc, p


def _inputs():
    """Two different elections: a dense count matrix with edge-less rows, then
    a smaller top-k tally (so the second call runs on leftovers of the first)."""
    rs = np.random.Generator(np.random.PCG64(17))
    m1 = 900
    d1 = rs.integers(0, 30000, size=(m1, m1)).astype(np.int32)
    d1[rs.random((m1, m1)) < 0.5] = 0
    d1[rs.random(m1) < 0.3, :] = 0
    np.fill_diagonal(d1, 0)
    e = W.large_topk(seed=23, n=3000, m=333, k=25)
    d2 = oracle.tally(e.ranks, e.m)
    return (d1, 30000), (d2, e.n)


def test_static_matches_allocating_entry_point_twice(lib):
    S, f = lib
    for flags in (0, S.F_FORCE_S32, S.F_MARGIN, S.F_MARGIN | S.F_FORCE_S32):
        for d_np, bound in _inputs():
            d = torch.from_numpy(d_np).cuda()
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            rc, p_static = _call(f, d, bound, flags, status)
            assert rc == S.OK
            assert int(status.item()) == S.OK
            p_ref = S.schulze_strongest_paths(d, bound, flags=flags)
            torch.cuda.synchronize()
            assert torch.equal(p_static, p_ref), "static scratch result differs from the allocating entry point"
    # the binding of the same name gives the same
    d_np, bound = _inputs()[1]
    d = torch.from_numpy(d_np).cuda()
    assert torch.equal(S.schulze_strongest_paths_static(d, bound), S.schulze_strongest_paths(d, bound))


def test_static_rejects_sizes_beyond_its_array(lib):
    S, f = lib
    d = torch.zeros((1025, 1025), dtype=torch.int32, device="cuda")
    rc, _ = _call(f, d, 10)
    assert rc == S.ETOOBIG
    d = torch.zeros((8, 8), dtype=torch.int32, device="cuda")
    rc, _ = _call(f, d, 40000, S.F_FORCE_S16)
    assert rc == S.EINVAL


def test_static_reports_data_errors_in_caller_status(lib):
    S, f = lib
    d = torch.tensor([[0, 40000], [0, 0]], dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc, _ = _call(f, d, 30000, 0, status)
    assert rc == S.OK and int(status.item()) == S.EDATA


def test_static_matches_oracle(lib):
    """Not only the other entry point: both elections, both edge weights,
    against the oracle's Floyd-Warshall (Sect. 2.1 definitions), each input
    run twice in a row on the shared array."""
    S, f = lib
    for margin in (False, True):
        for d_np, bound in _inputs():
            w = oracle.weights_margin(d_np) if margin else oracle.weights(d_np)
            want = oracle.closure(w, nthreads=os.cpu_count() or 1)
            d = torch.from_numpy(d_np).cuda()
            for _ in range(2):
                status = torch.zeros(1, dtype=torch.int32, device="cuda")
                rc, p = _call(f, d, bound, S.F_MARGIN if margin else 0, status)
                assert rc == S.OK and int(status.item()) == S.OK
                np.testing.assert_array_equal(p.cpu().numpy(), want)


def test_static_binding_raises_on_device_error_without_status(lib):
    """With no status word of the caller's, the binding checks its own and
    raises instead of returning an unspecified p."""
    S, _ = lib
    d = torch.tensor([[0, 40000], [0, 0]], dtype=torch.int32, device="cuda")
    with pytest.raises(S.SchulzeError):
        S.schulze_strongest_paths_static(d, 30000)
    # and a valid call afterwards is exact again
    d2 = torch.tensor([[0, 5, 1], [2, 0, 7], [3, 1, 0]], dtype=torch.int32, device="cuda")
    want = oracle.strongest_paths(d2.cpu().numpy())
    np.testing.assert_array_equal(S.schulze_strongest_paths_static(d2, 10).cpu().numpy(), want)
