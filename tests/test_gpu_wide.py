"""Full-range int32 data: queries whose centred coordinates exceed the fast
kernels' limit (td_coord_limit) are answered by the wide kernel (256-bit
integers, Proposition 1 with r = p - 1 applied recursively).  Bit-exact
against the full-range oracle (oracle/tukey_wide.py, Python integers) on
random and tie-heavy data with coordinates up to the int32 extremes, p = 1
to 6, in every entry point and form: filtered, plain exact, critical,
batched with in-range datasets, shards, the request stream."""
import numpy as np
import pytest

from gpu_common import random_case

pytestmark = pytest.mark.gpu

INT32_MAX = 2 ** 31 - 1
INT32_MIN = -2 ** 31


def _full_range_case(rng, p, n, kind):
    if kind == "uniform":
        X = rng.integers(INT32_MIN, INT32_MAX, size=(n, p), dtype=np.int64, endpoint=True)
    elif kind == "ties":
        # a few large base points, repeated, mirrored through z and scaled
        B = rng.integers(-2 ** 28, 2 ** 28, size=(max(p + 1, n // 3), p), dtype=np.int64)
        idx = rng.integers(0, len(B), size=n)
        sgn = rng.choice([-1, 1, 2], size=n)
        X = B[idx] * sgn[:, None]
    else:  # extremes: the corners of the int32 box and zero
        X = rng.choice([INT32_MIN, INT32_MAX, 0, 1, -1], size=(n, p))
    X = np.clip(X, INT32_MIN, INT32_MAX).astype(np.int32)
    Z = np.vstack([X[:2], np.zeros((1, p), np.int32),
                   rng.integers(-2 ** 30, 2 ** 30, size=(1, p), dtype=np.int64).astype(np.int32)])
    return X, Z


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_wide_filtered_plain_and_critical(p):
    from oracle import tukey_wide
    from paper_1409_3901_gb300 import tukey as td
    rng = np.random.default_rng(800 + p)
    n = {1: 24, 2: 20, 3: 16, 4: 12, 5: 11, 6: 10}[p]
    ctxs = [td.Context(0), td.Context(0, mode=td.TD_MODE_PLAIN_EXACT),
            td.Context(0, algorithm=td.TD_ALG_CRITICAL)]
    for kind in ("uniform", "ties", "extremes"):
        X, Z = _full_range_case(rng, p, n, kind)
        want = np.array(tukey_wide.depth_many(X, Z))
        for c in ctxs:
            assert np.array_equal(c.depth(X, Z), want), (p, kind, c.opts.mode, c.opts.algorithm)


def test_wide_mixed_batch_shards_and_stream():
    """In-range and full-range datasets in one batched call; the same under
    three shards merged by a minimum; the same through the stream."""
    import oracle
    from oracle import tukey_wide
    from paper_1409_3901_gb300 import tukey as td
    rng = np.random.default_rng(900)
    sets, wants = [], []
    for p, n in ((3, 14), (4, 12), (5, 11)):
        X, Z = _full_range_case(rng, p, n, "ties")
        sets.append((X, Z))
        wants.append(np.array(tukey_wide.depth_many(X, Z)))
        Xs = random_case(rng, p, 3 * n, 40)
        Zs = np.vstack([Xs[:2], rng.integers(-40, 41, size=(2, p))]).astype(np.int32)
        sets.append((Xs, Zs))
        wants.append(oracle.depth_many(Xs, Zs))
    outs = td.Context(0).depth_batched(sets)
    for o, w in zip(outs, wants):
        assert np.array_equal(o, w)
    parts = [td.Context(0, shard_index=s, shard_count=3).depth_batched(sets) for s in range(3)]
    for k, w in enumerate(wants):
        assert np.array_equal(np.min(np.stack([pp[k].astype(np.int64) for pp in parts]), axis=0), w)
    st = td.Context(0).stream(mem_budget_bytes=1 << 30)
    tickets = [st.submit(X, Z) for X, Z in sets]
    for t, w in zip(tickets, wants):
        assert np.array_equal(st.wait(t, timeout_us=120_000_000), w)
