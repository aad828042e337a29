"""td_depth_noalloc: the allocation-free entry point, for callers that must
not allocate device memory (a framework's memory pool owns the GPU, a fixed
device-memory budget, or a latency-critical path where cudaMalloc would
synchronise the device).  It must give exactly what td_depth gives -- the
counts are integers, so the tolerance of every parity test here is zero --
on consecutive calls that reuse its one static scratch array, and refuse
sizes beyond that array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _case(seed, n, p, m, lim):
    rng = np.random.default_rng(seed)
    X = rng.integers(-lim, lim + 1, size=(n, p)).astype(np.int32)
    X[1] = X[0]
    Z = np.vstack([X[: m // 2], rng.integers(-lim, lim + 1, size=(m - m // 2, p))]).astype(np.int32)
    return X, Z


def _noalloc(td, Xd, Zd, outd, stream=None):
    n, p = Xd.shape
    m = Zd.shape[0]
    return td.td_depth_noalloc(Xd.data_ptr(), n, p, Zd.data_ptr(), m, outd.data_ptr(), stream)


def test_noalloc_matches_td_depth_on_consecutive_calls():
    import torch
    from paper_1409_3901_gb300 import tukey as td
    ctx = td.Context(0)
    rng = np.random.default_rng(8)
    B = rng.integers(-3, 4, size=(2, 4))
    Xp = (rng.integers(-9, 10, size=(150, 2)) @ B).astype(np.int32)        # rank 2 inside p = 4
    Zp = np.vstack([Xp[:10], (rng.integers(-9, 10, size=(10, 2)) @ B)]).astype(np.int32)
    cases = [_case(1, 300, 4, 24, 60), _case(2, 120, 5, 16, 40), _case(5, 400, 2, 30, 50),
             (Xp, Zp), _case(6, 500, 3, 20, 90), _case(7, 90, 6, 8, 12), _case(1, 300, 4, 24, 60)]
    free_after = []
    for X, Z in cases:
        want = ctx.depth(X, Z)                     # the existing entry point
        Xd = torch.from_numpy(X).cuda()
        Zd = torch.from_numpy(Z).cuda()
        for _ in range(2):                         # two calls in a row
            outd = torch.full((Z.shape[0],), -7, dtype=torch.int32, device="cuda")
            rc = _noalloc(td, Xd, Zd, outd)
            assert rc == td.TD_OK, td.td_strerror(rc)
            assert np.array_equal(outd.cpu().numpy(), want)
            torch.cuda.synchronize()
            free_after.append(torch.cuda.mem_get_info()[0])
    # no device memory is taken by the calls themselves (the array is reserved
    # when the module loads, before the first call returns)
    assert max(free_after[1:]) - min(free_after[1:]) <= 8 << 20


def test_noalloc_rejects_sizes_beyond_the_array():
    import torch
    from paper_1409_3901_gb300 import tukey as td
    X, Z = _case(3, td.TD_NOALLOC_MAX_N + 1, 3, 4, 50)
    Xd = torch.from_numpy(X).cuda()
    Zd = torch.from_numpy(Z).cuda()
    outd = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    assert _noalloc(td, Xd, Zd, outd) == td.TD_ERR_INVALID
    assert int(outd[0]) == -7
    X, Z = _case(4, 50, 3, 4, 50)
    Zbig = torch.zeros((td.TD_NOALLOC_MAX_M + 1, 3), dtype=torch.int32, device="cuda")
    outbig = torch.zeros(td.TD_NOALLOC_MAX_M + 1, dtype=torch.int32, device="cuda")
    assert td.td_depth_noalloc(torch.from_numpy(X).cuda().data_ptr(), 50, 3, Zbig.data_ptr(),
                               td.TD_NOALLOC_MAX_M + 1, outbig.data_ptr(), None) == td.TD_ERR_INVALID


def test_noalloc_refuses_out_of_range_coordinates_and_leaves_out_untouched():
    """Device inputs one past td_coord_limit(p), on a pivot coordinate and
    on a coordinate that depends on the others (rank-2 data in p = 3, the
    third column 400 times the first): TD_ERR_RANGE, and out keeps its
    sentinel.  A call in range right after still gives td_depth's counts."""
    import torch
    from paper_1409_3901_gb300 import tukey as td
    rng = np.random.default_rng(31)
    bad = []
    for p in (3, 5, 6):
        L = int(td.td_coord_limit(p))
        X = rng.integers(-20, 21, size=(40, p)).astype(np.int64)
        X[5, p - 1] = L + 1                       # |x - z| = L + 1 for z = 0
        bad.append((X, np.zeros((3, p), np.int64)))
    c0 = rng.integers(-20000, 20001, size=60)
    Xr = np.stack([c0, rng.integers(-50, 51, size=60), 400 * c0], axis=1)
    assert np.abs(Xr).max() > td.td_coord_limit(3)
    bad.append((Xr, np.zeros((2, 3), np.int64)))
    for X, Z in bad:
        Xd = torch.from_numpy(X.astype(np.int32)).cuda()
        Zd = torch.from_numpy(Z.astype(np.int32)).cuda()
        outd = torch.full((Z.shape[0],), -7, dtype=torch.int32, device="cuda")
        assert _noalloc(td, Xd, Zd, outd) == td.TD_ERR_RANGE
        assert (outd.cpu().numpy() == -7).all()
    X, Z = _case(9, 200, 4, 10, 40)
    want = td.Context(0).depth(X, Z)
    outd = torch.full((Z.shape[0],), -7, dtype=torch.int32, device="cuda")
    assert _noalloc(td, torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda(), outd) == td.TD_OK
    assert np.array_equal(outd.cpu().numpy(), want)
