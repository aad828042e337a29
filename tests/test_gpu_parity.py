"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer results, so the bar is bit-exact.  Both execution forms are checked:
the FP32-filtered persistent form (TD_MODE_FILTERED, what bench.py times)
and the plain exact one-query-per-launch form (TD_MODE_PLAIN_EXACT).
"""
import numpy as np
import pytest

import oracle
from gpu_common import load_golden, random_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def td():
    from paper_1409_3901_gb300 import tukey
    return tukey


@pytest.fixture(scope="module")
def ctx(td):
    return td.Context(0)


@pytest.fixture(scope="module")
def plain(td):
    return td.Context(0, mode=td.TD_MODE_PLAIN_EXACT)


def _check_both(ctx, plain, X, Z):
    want = oracle.depth_many(X, Z)
    got = ctx.depth(X, Z)
    assert np.array_equal(got, want), (got.tolist(), want.tolist())
    got_p = plain.depth(X, Z)
    assert np.array_equal(got_p, want), (got_p.tolist(), want.tolist())


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_small_random_with_ties(ctx, plain, p):
    rng = np.random.default_rng(100 + p)
    for trial in range(6):
        n = int(rng.integers(p + 1, {1: 80, 2: 80, 3: 70, 4: 45, 5: 30, 6: 18}[p]))
        lim = int(rng.choice([2, 5, 40, 127]))
        X = random_case(rng, p, n, lim)
        rows = X[rng.integers(0, n, size=3)]
        unif = rng.integers(-lim, lim + 1, size=(3, p)).astype(np.int32)
        _check_both(ctx, plain, X, np.vstack([rows, unif]))


@pytest.mark.parametrize("nnz", [63, 64, 65])
def test_round_tails_p5(ctx, nnz):
    """p = 5 rows of 63, 64 and 65 nonzero points: the last round of the
    coarse pass runs at half width when its points fit in 64 (one short of,
    exactly at and one past that): the filtered form against the oracle, two
    deep queries near the centre (not data points, so every row counts)."""
    rng = np.random.default_rng(900 + nnz)
    X = random_case(rng, 5, nnz, 60, tie_rate=0.2)
    Z = np.array([[1, 2, -1, 0, 3], [-2, 1, 0, 2, -1]], np.int32)
    assert not (X[:, None, :] == Z[None, :, :]).all(axis=2).any()
    want = oracle.depth_many(X, Z)
    assert np.array_equal(ctx.depth(X, Z), want)


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_tie_heavy_small_grid(ctx, plain, p):
    """Coordinates in {-2..2}: many equal directions, tight sets and duplicates."""
    rng = np.random.default_rng(200 + p)
    n = {3: 60, 4: 35, 5: 20, 6: 14}[p]
    for trial in range(4):
        X = rng.integers(-2, 3, size=(n, p)).astype(np.int32)
        Z = np.vstack([X[:3], rng.integers(-1, 2, size=(3, p))]).astype(np.int32)
        _check_both(ctx, plain, X, Z)


@pytest.mark.parametrize("p,r", [(3, 1), (3, 2), (4, 2), (4, 3), (5, 3), (5, 4), (6, 4), (6, 5)])
def test_rank_deficient(ctx, plain, p, r):
    rng = np.random.default_rng(300 + 10 * p + r)
    for trial in range(3):
        B = rng.integers(-3, 4, size=(r, p))
        n = int(rng.integers(r + 2, 24))
        C = rng.integers(-4, 5, size=(n, r))
        z = rng.integers(-3, 4, size=p)
        X = (C @ B + z).astype(np.int32)
        Z = np.vstack([z, X[0], X[1] + 1]).astype(np.int32)
        _check_both(ctx, plain, X, Z)


def test_edge_cases(ctx, plain, td):
    X = np.array([[5, 5, 5]], np.int32)
    _check_both(ctx, plain, X, np.array([[5, 5, 5], [0, 0, 0]], np.int32))       # n = 1
    X = np.tile(np.array([[1, -2, 3, 4]], np.int32), (9, 1))
    _check_both(ctx, plain, X, np.array([[1, -2, 3, 4], [1, -2, 3, 5]], np.int32))  # all equal
    X = np.arange(12, dtype=np.int32).reshape(4, 3)                               # n <= p
    _check_both(ctx, plain, X, np.array([[0, 0, 0], [3, 4, 5], [1, 2, 3]], np.int32))
    out = ctx.depth(np.zeros((3, 2), np.int32), np.zeros((0, 2), np.int32))       # m = 0
    assert out.shape == (0,)


def test_golden_w1(ctx, plain):
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W1")
    d = W.w1()
    assert d.checksum() == g["checksum"]
    want = np.array(g["T"])
    assert np.array_equal(ctx.depth(d.X, d.Zq), want)
    assert np.array_equal(plain.depth(d.X, d.Zq), want)


@pytest.mark.parametrize("name", ["W2", "W4", "W6"])
def test_golden_full_size(ctx, name):
    """The full benchmark workloads, every query, in the launch form bench.py times."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden(name)
    d = W.WORKLOADS[name]()
    assert d.checksum() == g["checksum"]
    got = ctx.depth(d.X, d.Zq)
    assert np.array_equal(got, np.array(g["T"])), np.nonzero(got != np.array(g["T"]))
    st = ctx.last_stats
    assert st.sweeps > 0 and st.kernel_launches >= 4


def test_golden_w4_plain_sample(plain):
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W4")
    d = W.w4()
    idx = np.array([0, 5, 20, 41, 129, 200])
    got = plain.depth(d.X, d.Zq[idx])
    assert np.array_equal(got, np.array(g["T"])[idx])


def test_batched_matches_single(ctx, td):
    rng = np.random.default_rng(7)
    sets = []
    for p in (1, 2, 3, 4, 5, 3, 4):
        n = int(rng.integers(p + 2, 50 if p <= 4 else 25))
        X = random_case(rng, p, n, 30)
        Z = np.vstack([X[:2], rng.integers(-30, 31, size=(2, p))]).astype(np.int32)
        sets.append((X, Z))
    outs = ctx.depth_batched(sets)
    for (X, Z), o in zip(sets, outs):
        assert np.array_equal(o, oracle.depth_many(X, Z))


def test_golden_w3_sample_batched(ctx):
    """Every stored W3S dataset (the cheap ones: C(n,p-2) n <= 6e7) in one
    batched call, as the batched workload is served."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W3S")
    sets = W.w3()
    items = g["items"]
    batch = []
    for it in items:
        d = sets[it["index"]]
        assert d.checksum() == it["checksum"]
        batch.append((d.X, d.Zq))
    outs = ctx.depth_batched(batch)
    for it, o in zip(items, outs):
        assert np.array_equal(o, np.array(it["T"]))


def test_golden_w3_large_batched(ctx):
    """The large W3 datasets that W3S leaves out (largest n for p = 4 and 5,
    and a stratified sample of the rest), their stored queries in one batched
    call: the long subset loops of the batched workload."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W3L")
    sets = W.w3()
    batch = []
    for it in g["items"]:
        d = sets[it["index"]]
        assert d.checksum() == it["checksum"]
        batch.append((d.X, d.Zq[it["queries"]]))
    outs = ctx.depth_batched(batch)
    for it, o in zip(g["items"], outs):
        assert np.array_equal(o, np.array(it["T"])), (it["index"], o.tolist(), it["T"])
    assert ctx.last_stats.sweeps > 10 ** 8


def test_golden_p6_ties(ctx, plain):
    """p = 6 (K = 4, the deepest subset loop) with duplicates and collinear
    rows, n = 64 in [-4, 4] and n = 120 in [-127, 127]; filtered form, and
    the plain exact form on the smaller set."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("P6")
    for it in g["items"]:
        d = W.ties6(*it["args"])
        assert d.checksum() == it["checksum"]
        want = np.array(it["T"])
        assert np.array_equal(ctx.depth(d.X, d.Zq), want), it["args"]
        if d.n <= 64:
            assert np.array_equal(plain.depth(d.X, d.Zq), want)


def test_golden_sampled_shards(td):
    """Where a whole query is too costly for the oracle (p = 6 with ties at
    n = 300; the costliest p = 5 requests of the stream, n near 1000), sampled
    ranges of the subset loop: with `unseeded`, shard s of S returns exactly
    Z + min V(S) over its colex range, stored from the oracle over the same
    subsets (INT32_MAX for a range without an independent subset)."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("SHARDS")
    data = {}
    for label, fn in (("ties6 n=300", lambda: W.ties6(63, 300, 60)),):
        data[label] = fn()
    w5 = W.w5(count=400)
    checked = 0
    for it in g["items"]:
        label = it["dataset"]
        if label not in data:
            data[label] = w5[int(label[3:-1])]
        d = data[label]
        assert d.checksum() == it["checksum"]
        c = td.Context(0, shard_index=it["shard_index"], shard_count=it["shard_count"], unseeded=True)
        got = int(c.depth(d.X, d.Zq[it["query"]: it["query"] + 1])[0])
        want = 2 ** 31 - 1 if it["value"] is None else it["value"]
        assert got == want, (label, it["query"], it["shard_index"], got, want)
        checked += 1
    assert checked == len(g["items"]) > 0


def test_stream_w5s_all_requests(td):
    """All 38 stored W5S requests (p = 3 to 6) through td_stream_*, submitted
    back to back so that they are coalesced into batched launches."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W5S")
    ctx = td.Context(0)
    s = ctx.stream(mem_budget_bytes=8 << 30)
    tickets = []
    for it in g["items"]:
        d = W.w5_request(4, it["index"])
        assert d.checksum() == it["checksum"]
        t = s.submit(d.X, d.Zq)
        assert t is not None
        tickets.append((t, it))
    assert {it["p"] for _, it in tickets} >= {3, 4, 5, 6}
    for t, it in tickets:
        out = s.wait(t, timeout_us=120_000_000)
        assert np.array_equal(out, np.array(it["T"])), it["index"]


def test_stream_time_slices(td):
    """A request large enough to be cut into time slices (the largest-n
    p = 5 dataset of W3, its four stored queries repeated four times: about
    6e10 point evaluations, five slices) followed by small requests: every
    output equals the stored oracle counts, the slices' minima merged."""
    from math import comb
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W3L")
    it = next(x for x in g["items"] if x["p"] == 5 and len(x["queries"]) == 4)
    d = W.w3()[it["index"]]
    assert d.checksum() == it["checksum"]
    Z = np.vstack([d.Zq[it["queries"]]] * 4)
    assert comb(d.n, 3) * d.n * Z.shape[0] > 4 * 1.5e10
    ctx = td.Context(0)
    s = ctx.stream(mem_budget_bytes=8 << 30)
    heavy = s.submit(d.X, Z)
    rng = np.random.default_rng(15)
    small = []
    for i in range(5):
        X = random_case(rng, 4, 40, 30)
        Zs = np.vstack([X[:2], rng.integers(-30, 31, size=(2, 4))]).astype(np.int32)
        small.append((s.submit(X, Zs), X, Zs))
    for t, X, Zs in small:
        assert np.array_equal(s.wait(t, timeout_us=120_000_000), oracle.depth_many(X, Zs))
    out = s.wait(heavy, timeout_us=300_000_000)
    assert np.array_equal(out, np.tile(np.array(it["T"]), 4))


def test_shards_merge_to_depth(td):
    rng = np.random.default_rng(9)
    X = random_case(rng, 4, 40, 20)
    Z = np.vstack([X[:3], rng.integers(-20, 21, size=(3, 4))]).astype(np.int32)
    want = oracle.depth_many(X, Z)
    parts = []
    for s in range(3):
        c = td.Context(0, shard_index=s, shard_count=3)
        parts.append(c.depth(X, Z).astype(np.int64))
    assert np.array_equal(np.min(np.stack(parts), axis=0), want)


def test_stream_api(td):
    rng = np.random.default_rng(11)
    ctx = td.Context(0)
    s = ctx.stream(mem_budget_bytes=1 << 30)
    reqs = []
    for i in range(6):
        p = int(rng.integers(3, 6))
        n = int(rng.integers(20, 60 if p < 5 else 30))
        X = random_case(rng, p, n, 50)
        Z = np.vstack([X[:2], rng.integers(-50, 51, size=(2, p))]).astype(np.int32)
        t = s.submit(X, Z)
        assert t is not None
        reqs.append((t, X, Z))
    for t, X, Z in reqs:
        out = s.wait(t, timeout_us=60_000_000)
        assert np.array_equal(out, oracle.depth_many(X, Z))
    # admission by memory: a budget too small for any request refuses it
    tiny = ctx.stream(mem_budget_bytes=16)
    assert tiny.submit(reqs[0][1], reqs[0][2]) is None


def test_stream_polling_and_ticket_lifetime(td):
    """Requests submitted while a batch runs are coalesced into the next
    one; poll returns outputs once, after which the library forgets the
    ticket; a zero-query request completes at once."""
    import ctypes
    rng = np.random.default_rng(12)
    ctx = td.Context(0)
    s = ctx.stream(mem_budget_bytes=1 << 30)
    items = []
    for i in range(20):
        p = int(rng.integers(3, 5))
        X = random_case(rng, p, int(rng.integers(20, 50)), 40)
        Z = np.vstack([X[:1], rng.integers(-40, 41, size=(2, p))]).astype(np.int32)
        items.append((s.submit(X, Z), X, Z))
    got = {}
    for _ in range(200000):
        for t, X, Z in items:
            if t not in got:
                o = s.poll(t)
                if o is not None:
                    got[t] = o
        if len(got) == len(items):
            break
    assert len(got) == len(items)
    for t, X, Z in items:
        assert np.array_equal(got[t], oracle.depth_many(X, Z))
    done = ctypes.c_int(0)
    assert td.td_stream_poll(s.ptr, items[0][0], ctypes.byref(done)) == td.TD_ERR_NOTFOUND
    X = random_case(rng, 3, 10, 5)
    t0 = s.submit(X, np.zeros((0, 3), np.int32))
    assert s.wait(t0, timeout_us=1_000_000).shape == (0,)


def test_errors_leave_outputs_untouched(ctx, td):
    out = np.full(1, -12345, np.int32)
    with pytest.raises(td.TdError) as e:
        ctx.depth(np.zeros((3, 7), np.int32), np.zeros((1, 7), np.int32), out=out)
    assert e.value.code == td.TD_ERR_INVALID
    assert out[0] == -12345
    with pytest.raises(td.TdError) as e:
        ctx.depth(np.zeros((td.TD_MAX_N + 1, 3), np.int32), np.zeros((1, 3), np.int32), out=out)
    assert e.value.code == td.TD_ERR_INVALID
    assert out[0] == -12345


def test_beyond_the_fast_limit_every_coordinate(td):
    """A coordinate beyond td_coord_limit(p) -- also one that depends on the
    others and so is not a pivot coordinate of the set-up's elimination
    (rank-2 data in p = 3, the third column 400 times the first) -- sends
    the query to the wide kernel, with host and device pointers and in every
    algorithm: the full-range oracle's count."""
    import torch
    from oracle import tukey_wide
    rng = np.random.default_rng(14)
    c0 = rng.integers(-20000, 20001, size=40)
    X = np.stack([c0, rng.integers(-50, 51, size=40), 400 * c0], axis=1).astype(np.int32)
    assert np.abs(X.astype(np.int64)).max() > td.td_coord_limit(3)
    Z = np.vstack([np.zeros((1, 3), np.int32), X[:1]])
    want = np.array(tukey_wide.depth_many(X, Z))
    assert np.array_equal(td.Context(0).depth(X, Z), want)
    for alg in (td.TD_ALG_RCOM, td.TD_ALG_ADIA, td.TD_ALG_CRITICAL):
        c = td.Context(0, device_pointers=True, algorithm=alg)
        out = torch.full((2,), -5, dtype=torch.int32, device="cuda")
        c.depth(torch.from_numpy(X).cuda(), torch.from_numpy(Z).cuda(), out)
        assert np.array_equal(out.cpu().numpy(), want), alg


def test_device_pointers(td):
    import torch
    rng = np.random.default_rng(13)
    X = random_case(rng, 4, 50, 40)
    Z = np.vstack([X[:3], rng.integers(-40, 41, size=(3, 4))]).astype(np.int32)
    want = oracle.depth_many(X, Z)
    c = td.Context(0, device_pointers=True)
    Xd = torch.from_numpy(X).cuda()
    Zd = torch.from_numpy(Z).cuda()
    got = c.depth(Xd, Zd).cpu().numpy()
    assert np.array_equal(got, want)
    got2 = c.depth(Xd, Zd).cpu().numpy()     # graph replay
    assert np.array_equal(got2, want)


def test_early_exit_same_depths(td, plain):
    """Early-exit mode (running minimum seeded with the data-direction bound
    of Algorithm 3 Step 2, a query stopped once it reaches V = 0) returns the
    same depths, and skips subsets of queries whose depth is Z."""
    ee = td.Context(0, early_exit=True)
    rng = np.random.default_rng(21)
    for p in (3, 4, 5, 6):
        for trial in range(3):
            n = int(rng.integers(p + 2, {3: 60, 4: 40, 5: 26, 6: 16}[p]))
            lim = int(rng.choice([2, 5, 40]))
            X = random_case(rng, p, n, lim)
            # data rows, points far outside the data (depth Z = 0) and uniform points
            Z = np.vstack([X[:2], np.full((1, p), 3 * lim, np.int32),
                           rng.integers(-lim, lim + 1, size=(2, p))]).astype(np.int32)
            want = oracle.depth_many(X, Z)
            got = ee.depth(X, Z)
            assert np.array_equal(got, want), (p, got.tolist(), want.tolist())
    from paper_1409_3901_gb300 import workloads as W
    for name in ("W1", "W2"):
        g = load_golden(name)
        d = W.WORKLOADS[name]()
        got = ee.depth(d.X, d.Zq)
        assert np.array_equal(got, np.array(g["T"])), name
        st = ee.last_stats
        assert st.early_skipped > 0, name
    # shards with early exit still merge to the depth
    X = random_case(rng, 4, 40, 20)
    Z = np.vstack([X[:3], rng.integers(-20, 21, size=(3, 4)), np.full((1, 4), 90, np.int32)]).astype(np.int32)
    want = oracle.depth_many(X, Z)
    parts = [td.Context(0, shard_index=s, shard_count=3, early_exit=True).depth(X, Z).astype(np.int64)
             for s in range(3)]
    assert np.array_equal(np.min(np.stack(parts), axis=0), want)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_coordinate_limits(ctx, plain, td, p):
    """Centred coordinates up to td_coord_limit(p): corners of the allowed
    box, duplicates and large-magnitude ties, which push the exact int64 /
    int128 intermediates and the FP32 error bound to their extremes."""
    L = int(td.td_coord_limit(p))
    h = L // 2
    rng = np.random.default_rng(400 + p)
    n = {1: 80, 2: 80, 3: 50, 4: 30, 5: 18, 6: 12}[p]
    for trial in range(3):
        X = rng.integers(-h, h + 1, size=(n, p))
        X[: n // 4] = np.where(rng.random((n // 4, p)) < 0.5, -h, h)   # corners
        X[-3:] = X[:3]                                                 # duplicates
        v = rng.integers(-3, 4, size=p)
        X[n // 4: n // 4 + 3] = np.outer([1, -2, 3], v) * (h // 9)    # collinear through 0, within h
        Z = np.vstack([X[:2], np.zeros((1, p), np.int64),
                       rng.integers(-h, h + 1, size=(2, p))]).astype(np.int32)
        _check_both(ctx, plain, X.astype(np.int32), Z)


def test_maximum_n(ctx, td):
    """n = 2048, the largest data set one call accepts, in both dimensions
    whose subset loops stay cheap for the oracle; n = 2049 is refused."""
    rng = np.random.default_rng(500)
    for p in (2, 3):
        X = rng.integers(-127, 128, size=(2048, p)).astype(np.int32)
        X[100:140] = X[0]                                      # ties at the maximum size
        Z = np.vstack([X[:2], rng.integers(-127, 128, size=(1, p))]).astype(np.int32)
        assert np.array_equal(ctx.depth(X, Z), oracle.depth_many(X, Z))
    with pytest.raises(td.TdError) as e:
        ctx.depth(np.zeros((2049, 3), np.int32), np.zeros((1, 3), np.int32))
    assert e.value.code == td.TD_ERR_INVALID
