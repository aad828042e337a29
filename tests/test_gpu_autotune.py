"""The autotuner (td_autotune, td_set_tuned): it measures every candidate
work-tile size, keeps the fastest in the context when it beats the size
rule by more than 1%, and a context with tuned
(or any explicitly set) tile sizes still gives the oracle's counts bit for
bit -- the tile size changes only how the subset loop is cut into work."""
import numpy as np
import pytest

import oracle
from gpu_common import load_golden, random_case

pytestmark = pytest.mark.gpu


def test_autotune_measures_and_keeps_parity():
    from paper_1409_3901_gb300 import tukey, workloads as W
    ctx = tukey.Context(0)
    for p, n in ((4, 300), (5, 150)):
        r = ctx.autotune(p, n)
        assert r["p"] == p and r["n"] == n and r["queries"] >= 1
        assert sorted(r["candidates"]) == [16, 32, 64, 128, 192, 256, 512, 1024]
        assert all(ms > 0 for ms in r["candidates"].values()) and r["ms_default"] > 0
        # a candidate is kept only when it beats the size rule by more than 1%
        if r["best_spw"] == 0:
            assert r["best_ms"] == r["ms_default"]
            assert all(ms >= 0.99 * r["ms_default"] for ms in r["candidates"].values())
        else:
            assert r["best_ms"] == r["candidates"][r["best_spw"]] < 0.99 * r["ms_default"]
            assert r["best_ms"] == min(r["candidates"].values())
    rng = np.random.default_rng(41)
    for p, n in ((4, 300), (4, 270), (5, 150), (5, 140)):
        X = random_case(rng, p, n, 60)
        Z = np.vstack([X[:2], rng.integers(-60, 61, size=(2, p))]).astype(np.int32)
        assert np.array_equal(ctx.depth(X, Z), oracle.depth_many(X, Z)), (p, n)
    g = load_golden("W1")
    d = W.w1()
    assert np.array_equal(ctx.depth(d.X, d.Zq), np.array(g["T"]))


@pytest.mark.parametrize("spw", [4, 8, 100, 256])
def test_explicit_tile_sizes_keep_parity(spw):
    """td_set_tuned with small, odd and large tile sizes for the octave of
    the p = 5, n = 200 workload with ties (W4): the same counts."""
    from paper_1409_3901_gb300 import tukey, workloads as W
    g = load_golden("W4")
    d = W.w4()
    idx = np.arange(0, 256, 16)
    ctx = tukey.Context(0)
    ctx.set_tuned(5, 8, spw)        # 128 < n' <= 256
    ctx.set_tuned(4, 8, spw)        # queries of lower effective dimension, if any
    assert np.array_equal(ctx.depth(d.X, d.Zq[idx]), np.array(g["T"])[idx])
    with pytest.raises(tukey.TdError):
        ctx.set_tuned(7, 8, spw)
