"""GPU parity of Algorithm 3 (ADIA, td_options.algorithm = TD_ALG_ADIA)
against the oracle's Algorithm 3 (oracle.adia), element by element.

Integer results: the bar is bit-exact.  Both sides follow the same readings of
Algorithm 3 (order of subsets, critical points, stack, Step 5(a) side), so the
search visits the same nodes and returns the same count; every count is also
checked to be at least the exact count of Algorithm 1 on the GPU.
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
def adia(td):
    return td.Context(0, algorithm=td.TD_ALG_ADIA)


@pytest.fixture(scope="module")
def rcom(td):
    return td.Context(0)


def _want(X, Z):
    return np.array([oracle.adia(X, z)[0] for z in Z], dtype=np.int64)


def _check(adia, rcom, X, Z):
    want = _want(X, Z)
    got = adia.depth(X, Z)
    st = adia.last_stats
    assert st.adia_fallbacks == 0
    assert np.array_equal(got, want), (got.tolist(), want.tolist())
    exact = rcom.depth(X, Z)
    assert (got >= exact).all()
    return got, exact, st


def _queries(rng, X, lim):
    n, p = X.shape
    rows = X[rng.integers(0, n, size=2)]
    inner = np.rint(X[rng.integers(0, n, size=(2, 3))].mean(axis=1))
    unif = rng.integers(-lim, lim + 1, size=(1, p))
    return np.vstack([rows, inner, unif]).astype(np.int32)


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_small_tie_heavy(adia, rcom, p):
    rng = np.random.default_rng(500 + p)
    searched = 0
    for trial in range(6):
        n = int(rng.integers(2 * p + 1, {3: 90, 4: 55, 5: 32, 6: 20}[p]))
        lim = int(rng.choice([2, 3, 10, 127]))
        X = random_case(rng, p, n, lim, tie_rate=0.5)
        _, _, st = _check(adia, rcom, X, _queries(rng, X, lim))
        searched += st.adia_pops > 0
    assert searched > 0


@pytest.mark.parametrize("p,n", [(3, 320), (4, 160), (5, 60), (6, 36)])
def test_gaussian_alpha_queries(adia, rcom, p, n):
    """The simulation of Section 5.2 at small n: N(0, I_p) x 40 and z = alpha x 40 x 1_p."""
    rng = np.random.default_rng(600 + p)
    X = np.clip(np.rint(40 * rng.standard_normal((n, p))), -127, 127).astype(np.int32)
    Z = np.array([[round(40 * a)] * p for a in (0.0, 0.4, 0.8, 1.2)], dtype=np.int32)
    got, exact, st = _check(adia, rcom, X, Z)
    assert st.adia_pops > 0 and st.adia_subsets >= st.adia_pops


def test_rank_deficient_and_duplicates(adia, rcom):
    """Data of rank 3 in p = 5 (the search runs in pivot coordinates, Step 2
    in the input coordinates) and data with many repeated rows."""
    rng = np.random.default_rng(17)
    B = rng.integers(-3, 4, size=(3, 5))
    X = (rng.integers(-6, 7, size=(40, 3)) @ B).astype(np.int32)
    Z = np.vstack([X[:3], np.rint(X[:9].reshape(3, 3, 5).mean(axis=1))]).astype(np.int32)
    _check(adia, rcom, X, Z)
    X = rng.integers(-4, 5, size=(12, 4))
    X = X[rng.integers(0, 12, size=48)].astype(np.int32)
    _check(adia, rcom, X, _queries(rng, X, 4))


def test_batched_mixed_dimensions(adia):
    rng = np.random.default_rng(23)
    sets = []
    for p in (2, 3, 4, 5, 6, 3, 4):
        n = int(rng.integers(2 * p + 1, {2: 60, 3: 70, 4: 45, 5: 28, 6: 18}[p]))
        X = random_case(rng, p, n, 30)
        sets.append((X, _queries(rng, X, 30)))
    outs = adia.depth_batched(sets)
    assert adia.last_stats.adia_fallbacks == 0
    for (X, Z), o in zip(sets, outs):
        assert np.array_equal(o, _want(X, Z))


def test_device_pointers_and_graph_replay(td):
    import torch
    rng = np.random.default_rng(29)
    X = random_case(rng, 4, 80, 40)
    Z = _queries(rng, X, 40)
    want = _want(X, Z)
    c = td.Context(0, device_pointers=True, algorithm=td.TD_ALG_ADIA)
    Xd = torch.from_numpy(X).cuda()
    Zd = torch.from_numpy(Z).cuda()
    assert np.array_equal(c.depth(Xd, Zd).cpu().numpy(), want)
    assert np.array_equal(c.depth(Xd, Zd).cpu().numpy(), want)  # graph replay


def test_stream_api(td):
    rng = np.random.default_rng(31)
    c = td.Context(0, algorithm=td.TD_ALG_ADIA)
    s = c.stream(1 << 28)
    reqs = []
    for p in (3, 4, 5):
        X = random_case(rng, p, 40, 20)
        Z = _queries(rng, X, 20)
        reqs.append((X, Z, s.submit(X, Z)))
    for X, Z, t in reqs:
        assert np.array_equal(s.wait(t), _want(X, Z))
    s.close()


@pytest.mark.parametrize("name", ["W1A", "W2A"])
def test_golden_full_size(adia, name):
    """Every query of W1 and W2 in one call, against the stored oracle counts."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden(name)
    d = W.WORKLOADS[name[:2]]()
    assert d.checksum() == g["checksum"]
    got = adia.depth(d.X, d.Zq)
    assert adia.last_stats.adia_fallbacks == 0
    assert np.array_equal(got, np.array(g["T"])), np.nonzero(got != np.array(g["T"]))


def test_golden_w7_batched(adia):
    """The Section 5.2 shapes (W7, 40 datasets, 160 queries) in one batched call."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W7A")
    sets = W.w7()
    assert len(sets) == len(g["items"])
    for d, it in zip(sets, g["items"]):
        assert d.checksum() == it["checksum"]
    outs = adia.depth_batched([(d.X, d.Zq) for d in sets])
    assert adia.last_stats.adia_fallbacks == 0
    for it, o in zip(g["items"], outs):
        assert np.array_equal(o, np.array(it["T"])), (it["index"], o.tolist(), it["T"])


def test_golden_w3_sample_batched(adia):
    """40 datasets of the batched workload W3 (p in {3, 4, 5}, n from 100 to
    2000) in one call: the search kernel of each dimension runs in the block
    form for every query of the batch."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W3SA")
    sets = W.w3()
    batch = []
    for it in g["items"]:
        d = sets[it["index"]]
        assert d.checksum() == it["checksum"]
        batch.append((d.X, d.Zq))
    outs = adia.depth_batched(batch)
    assert adia.last_stats.adia_fallbacks == 0
    for it, o in zip(g["items"], outs):
        assert np.array_equal(o, np.array(it["T"])), (it["index"], o.tolist(), it["T"])


def test_early_exit_leaves_the_counts(td, adia):
    """Algorithm 3 with td_options.early_exit: the sweep of Step 5(b) stops a
    query whose minimum reached 0, which cannot change its count."""
    from paper_1409_3901_gb300 import workloads as W
    d = W.w1()
    ee = td.Context(0, algorithm=td.TD_ALG_ADIA, early_exit=True)
    assert np.array_equal(ee.depth(d.X, d.Zq), adia.depth(d.X, d.Zq))


def test_golden_w5_sample_stream(td):
    """30 requests of the stream workload W5 (p from 3 to 6, uniform integer
    data) through td_stream_*, against the stored oracle counts.  One of these
    queries (request 20, query 27) is a case where Algorithm 3 returns 33 and
    the exact count is 32."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W5SA")
    c = td.Context(0, algorithm=td.TD_ALG_ADIA)
    s = c.stream(1 << 30)
    pend = []
    for it in g["items"]:
        d = W.w5_request(4, it["index"])
        assert d.checksum() == it["checksum"]
        t = s.submit(d.X, d.Zq)
        assert t is not None
        pend.append((it, t))
    for it, t in pend:
        assert np.array_equal(s.wait(t), np.array(it["T"])), it["index"]
    s.close()


@pytest.mark.parametrize("req,query,T", [(20, 27, 32), (376, 3, 51)])
def test_upper_bound_cases(adia, rcom, req, query, T):
    """The two queries of the request stream where the oracle's Algorithm 3
    returns T + 1: the device search takes the same path, and Algorithm 1
    gives T."""
    from paper_1409_3901_gb300 import workloads as W
    d = W.w5_request(4, req)
    Z = d.Zq[query:query + 1]
    assert np.array_equal(rcom.depth(d.X, Z), [T])
    assert np.array_equal(adia.depth(d.X, Z), [T + 1])
