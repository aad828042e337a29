"""GPU parity of the critical-direction form (Proposition 1 with r = p-1,
td_options.algorithm = TD_ALG_CRITICAL, p <= 6) against the oracle, and
against Algorithm 1 on the GPU at full benchmark sizes: two routes to the
exact count that share no arithmetic beyond the tight-set recursion.
Bit-exact."""
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
def crit(td):
    return td.Context(0, algorithm=td.TD_ALG_CRITICAL)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_small_tie_heavy(crit, p):
    rng = np.random.default_rng(700 + p)
    for trial in range(6):
        n = int(rng.integers(p + 1, {1: 60, 2: 70, 3: 60, 4: 40, 5: 25, 6: 16}[p]))
        lim = int(rng.choice([2, 3, 10, 127]))
        X = random_case(rng, p, n, lim, tie_rate=0.5)
        Z = np.vstack([X[rng.integers(0, n, size=3)], rng.integers(-lim, lim + 1, size=(3, p))]).astype(np.int32)
        got = crit.depth(X, Z)
        assert np.array_equal(got, oracle.depth_many(X, Z)), (p, X.tolist(), Z.tolist())


def test_hyperplanes_with_many_points(crit):
    """Small grids: many hyperplanes through z hold more than p-1 points, so
    the open depth m_F inside the hyperplane is needed."""
    rng = np.random.default_rng(41)
    for p in (3, 4, 5, 6):
        X = rng.integers(-2, 3, size=({3: 40, 4: 30, 5: 20, 6: 14}[p], p)).astype(np.int32)
        Z = np.vstack([X[:3], np.zeros((1, p), np.int32)]).astype(np.int32)
        got = crit.depth(X, Z)
        assert np.array_equal(got, oracle.depth_many(X, Z))
        assert crit.last_stats.tight_exceptions > 0


def test_rank_deficient(crit):
    rng = np.random.default_rng(43)
    B = rng.integers(-3, 4, size=(3, 5))
    X = (rng.integers(-5, 6, size=(30, 3)) @ B).astype(np.int32)
    Z = X[:4].copy()
    assert np.array_equal(crit.depth(X, Z), oracle.depth_many(X, Z))


def test_limits(td, crit):
    """Beyond the int64 bound of the critical-direction kernel (p! M^p >=
    2^62) the query goes to the 256-bit path: the full-range oracle's count."""
    from oracle import tukey_wide
    X = np.array([[30000, 1, 2, 3], [1, 2, 3, 4], [5, 6, 7, -8], [1, 0, 0, 0], [0, 1, 0, 0]], np.int32)
    Z = np.zeros((1, 4), np.int32)                 # 4! * 30000^4 > 2^62
    assert np.array_equal(crit.depth(X, Z), tukey_wide.depth_many(X, Z))
    X = np.vstack([np.eye(6, dtype=np.int32) * 500, -np.ones((1, 6), np.int32)])
    Z = np.zeros((1, 6), np.int32)                 # 6! * 500^6 > 2^62
    assert np.array_equal(crit.depth(X, Z), tukey_wide.depth_many(X, Z))


@pytest.mark.parametrize("name,count", [("W1", 16), ("W4", 64)])
def test_golden_full_size(crit, name, count):
    """W1 (p = 3), every query; W4 (p = 5, n = 200, C(200, 4) hyperplanes per
    query), its first 64 queries: every copied and hyperplane row."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden(name)
    d = W.WORKLOADS[name]()
    assert d.checksum() == g["checksum"]
    got = crit.depth(d.X, d.Zq[:count])
    want = np.array(g["T"])[:count]
    assert np.array_equal(got, want), np.nonzero(got != want)


def test_golden_w2_sample(crit):
    """W2 (p = 4, n = 1000): C(1000, 3) hyperplanes per query, a sample of queries."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W2")
    d = W.w2()
    idx = np.array([0, 17, 32, 33, 50, 63])
    got = crit.depth(d.X, d.Zq[idx])
    assert np.array_equal(got, np.array(g["T"])[idx])


def test_shards_merge_to_the_depth(td):
    """shard_index / shard_count split the hyperplane positions of every query;
    the minimum over the shards is the depth."""
    rng = np.random.default_rng(47)
    X = random_case(rng, 4, 60, 20, tie_rate=0.4)
    Z = np.vstack([X[:3], rng.integers(-20, 21, size=(3, 4))]).astype(np.int32)
    want = oracle.depth_many(X, Z)
    parts = []
    for k in range(3):
        c = td.Context(0, algorithm=td.TD_ALG_CRITICAL, shard_index=k, shard_count=3)
        parts.append(c.depth(X, Z).astype(np.int64))
    assert np.array_equal(np.minimum.reduce(parts), want)


def test_golden_w5_sample_p6(crit):
    """The p = 6 requests of the stored W5 sample (uniform integer data)."""
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W5S")
    items = [it for it in g["items"] if it["p"] == 6][:6]
    assert items
    for it in items:
        d = W.w5_request(4, it["index"])
        assert d.checksum() == it["checksum"]
        assert np.array_equal(crit.depth(d.X, d.Zq), np.array(it["T"])), it["index"]
