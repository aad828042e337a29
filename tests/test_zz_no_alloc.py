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
             (Xp, Zp), _case(1, 300, 4, 24, 60)]
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
