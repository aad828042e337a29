"""Seeded synthetic workloads for the exact Tukey depth (no depth arithmetic here).

The paper's own experiments (Section 5) use two real data sets that are not
available (the vocabulary data and the IBM returns, Section 5.1) and standard
normal samples with z = alpha * 1_p (Section 5.2, Table 2).  The generators
below stand in for both with int32 data of the shapes and tie structure of the
five benchmark workloads:

  W1  p=3, n=300, i.i.d. uniform integers in [-127, 127]; 16 queries:
      8 distinct data rows and 8 uniform integer points.
  W2  p=4, n=1000, round(40 * N(0,1)) clipped to [-127, 127]; 64 queries:
      32 distinct data rows, the lower coordinate-wise median and 31 uniform
      points of the data's bounding box.
  W3  256 datasets, p uniform in {3,4,5}, n = round(exp(U(ln 100, ln 2000)))
      decremented until C(n, p-2) * n <= 4e9, coordinates Gaussian (x40) or
      uniform with probability 1/2 each; 16 queries per dataset: 8 data rows
      and 8 uniform points of the bounding box.
  W4  p=5, n=200, round(20 * t_3) clipped; 20 rows overwritten by copies of
      other rows, 10 rows placed on one hyperplane a'x = c (integer a, a_5 = 1);
      256 queries: 128 data rows (all copied and hyperplane rows among them)
      and 128 uniform points of the bounding box.
  W5  a stream of requests, each p in {3,4,5,6}, n uniform in [50, 1000]
      (p = 6: n <= 120), 1-64 queries (half data rows, half uniform points of
      the bounding box), uniform integer coordinates.
  W6  the bivariate case alone (p = 2: S is empty, one sweep per query):
      n = 2000, round(40 * N(0,1)) clipped; 16384 queries: 8192 data rows
      drawn with replacement and 8192 uniform points of the bounding box.
  W7  the shapes of the paper's simulation (Section 5.2, Tables 2 and 3):
      round(40 * N(0, I_p)) clipped, for (p, n) = (3, 1280), (4, 640),
      (5, 160), (6, 80); 10 datasets each, with the four queries
      z = alpha * 40 * 1_p, alpha in {0, 0.4, 0.8, 1.2} (160 queries).

Random numbers come from a counter-based SplitMix64 stream (defined by its
published constants), uniform doubles from its top 53 bits, Gaussians by the
Box-Muller transform, and rounding is half-to-even before clipping.  Every
workload carries a checksum of its integer arrays so that a copy generated on
another machine can be verified against stored expected values.
"""
from dataclasses import dataclass, field
from math import comb
import hashlib

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = float(2 ** 53)
LIM = 127


class Stream:
    """Counter-based SplitMix64: value k is mix(seed_key + (k+1) * golden)."""

    def __init__(self, seed, sub=0):
        with np.errstate(over="ignore"):
            self.key = np.uint64(seed) * np.uint64(0xD1B54A32D192ED03) + np.uint64(sub) * _GOLDEN
        self.ctr = 0

    def u64(self, count):
        k = np.arange(self.ctr + 1, self.ctr + 1 + count, dtype=np.uint64)
        self.ctr += count
        with np.errstate(over="ignore"):
            z = self.key + k * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, count):
        """Doubles in [0, 1)."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) / _TWO53

    def integers(self, lo, hi, count):
        """Integers uniform in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        v = np.floor(self.uniform(count) * span).astype(np.int64)
        return (lo + np.minimum(v, span - 1)).astype(np.int64)

    def normal(self, count):
        u1 = ((self.u64(count) >> np.uint64(11)).astype(np.float64) + 1.0) / _TWO53  # (0, 1]
        u2 = self.uniform(count)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def choice(self, n, k):
        """k distinct indices of range(n), by a partial Fisher-Yates shuffle."""
        perm = np.arange(n, dtype=np.int64)
        r = self.uniform(k)
        for i in range(k):
            j = i + int(np.floor(r[i] * (n - i)))
            j = min(j, n - 1)
            perm[i], perm[j] = perm[j], perm[i]
        return perm[:k].copy()


def _round_clip(v, lim=LIM):
    return np.clip(np.rint(v), -lim, lim).astype(np.int32)


def _bbox_uniform(st, X, m):
    lo = X.min(axis=0).astype(np.int64)
    hi = X.max(axis=0).astype(np.int64)
    cols = [st.integers(int(lo[c]), int(hi[c]), m) for c in range(X.shape[1])]
    return np.stack(cols, axis=1).astype(np.int32)


def checksum(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a, dtype=np.int32)
        h.update(np.asarray(a.shape, dtype=np.int64).tobytes())
        h.update(a.tobytes())
    return h.hexdigest()[:16]


@dataclass
class Dataset:
    """n x p int32 data X and m x p int32 queries Zq (row-major)."""
    X: np.ndarray
    Zq: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.X.shape[0])

    @property
    def p(self):
        return int(self.X.shape[1])

    @property
    def m(self):
        return int(self.Zq.shape[0])

    def sweeps(self):
        """Top-level subsets of Algorithm 1 per query, C(n, p-2) (upper bound)."""
        return comb(self.n, self.p - 2) if self.p >= 2 else 1

    def checksum(self):
        return checksum(self.X, self.Zq)


def w1(seed=0):
    st = Stream(seed)
    n, p = 300, 3
    X = st.integers(-LIM, LIM, n * p).reshape(n, p).astype(np.int32)
    rows = X[st.choice(n, 8)]
    unif = st.integers(-LIM, LIM, 8 * p).reshape(8, p).astype(np.int32)
    return Dataset(X, np.vstack([rows, unif]).astype(np.int32), "W1 p=3 n=300 uniform, 16 queries")


def w2(seed=1):
    st = Stream(seed)
    n, p = 1000, 4
    X = _round_clip(40.0 * st.normal(n * p)).reshape(n, p)
    rows = X[st.choice(n, 32)]
    med = np.sort(X, axis=0)[n // 2 - 1][None, :]
    unif = _bbox_uniform(st, X, 31)
    return Dataset(X, np.vstack([rows, med, unif]).astype(np.int32),
                   "W2 p=4 n=1000 gaussian x40, 64 queries")


def _w3_shape(st):
    p = int(st.integers(3, 5, 1)[0])
    n = int(round(float(np.exp(np.log(100.0) + st.uniform(1)[0] * (np.log(2000.0) - np.log(100.0))))))
    while comb(n, p - 2) * n > 4_000_000_000:
        n -= 1
    return n, p


def w3(seed=2, count=256, queries=16):
    out = []
    for d in range(count):
        st = Stream(seed, sub=d + 1)
        n, p = _w3_shape(st)
        if st.uniform(1)[0] < 0.5:
            X = _round_clip(40.0 * st.normal(n * p)).reshape(n, p)
            kind = "gaussian"
        else:
            X = st.integers(-LIM, LIM, n * p).reshape(n, p).astype(np.int32)
            kind = "uniform"
        h = queries // 2
        rows = X[st.choice(n, h)]
        unif = _bbox_uniform(st, X, queries - h)
        out.append(Dataset(X, np.vstack([rows, unif]).astype(np.int32),
                           "W3[%d] p=%d n=%d %s" % (d, p, n, kind), {"index": d}))
    return out


def w4(seed=3):
    st = Stream(seed)
    n, p = 200, 5
    g = st.normal(n * p).reshape(n, p)
    chi = (st.normal(n * 3).reshape(n, 3) ** 2).sum(axis=1) / 3.0
    X = _round_clip(20.0 * g / np.sqrt(chi)[:, None])
    perm = st.choice(n, 50)
    dup_dst, dup_src, hyp = perm[:20], perm[20:40], perm[40:50]
    X[dup_dst] = X[dup_src]
    a = st.integers(-2, 2, p - 1)
    c = int(st.integers(-20, 20, 1)[0])
    for i in hyp:
        while True:
            g4 = st.normal(p - 1)
            ch = (st.normal(3) ** 2).sum() / 3.0
            head = _round_clip(20.0 * g4 / np.sqrt(ch)).astype(np.int64)
            last = c - int(np.dot(a, head))
            if abs(last) <= LIM:
                X[i, : p - 1] = head
                X[i, p - 1] = last
                break
    special = np.concatenate([dup_dst, dup_src, hyp])
    others = np.setdiff1d(np.arange(n), special)
    pick = others[st.choice(len(others), 128 - len(special))]
    rows = X[np.concatenate([special, pick])]
    unif = _bbox_uniform(st, X, 128)
    return Dataset(X, np.vstack([rows, unif]).astype(np.int32),
                   "W4 p=5 n=200 t3 x20 with copies and a hyperplane, 256 queries",
                   {"hyperplane_a": a.tolist() + [1], "hyperplane_c": c})


def w5_request(seed, index):
    st = Stream(seed, sub=index + 1)
    p = int(st.integers(3, 6, 1)[0])
    n = int(st.integers(50, 120 if p == 6 else 1000, 1)[0])
    q = int(st.integers(1, 64, 1)[0])
    X = st.integers(-LIM, LIM, n * p).reshape(n, p).astype(np.int32)
    h = q // 2
    rows = X[st.choice(n, h)] if h > 0 else np.zeros((0, p), np.int32)
    unif = _bbox_uniform(st, X, q - h)
    return Dataset(X, np.vstack([rows, unif]).astype(np.int32),
                   "W5[%d] p=%d n=%d q=%d" % (index, p, n, q), {"index": index})


def w5(seed=4, count=64):
    return [w5_request(seed, i) for i in range(count)]


def small_random(seed, n, p, lim=LIM, queries=8, data_queries=None):
    """A small uniform dataset for tests: queries = data rows then uniform points."""
    st = Stream(seed, sub=7)
    X = st.integers(-lim, lim, n * p).reshape(n, p).astype(np.int32)
    h = queries // 2 if data_queries is None else data_queries
    h = min(h, n)
    rows = X[st.choice(n, h)] if h > 0 else np.zeros((0, p), np.int32)
    unif = st.integers(-lim, lim, (queries - h) * p).reshape(queries - h, p).astype(np.int32)
    return Dataset(X, np.vstack([rows, unif]).astype(np.int32), "small p=%d n=%d" % (p, n))


def w6(seed=5, m=16384):
    st = Stream(seed)
    n, p = 2000, 2
    X = _round_clip(40.0 * st.normal(n * p)).reshape(n, p)
    half = m // 2
    rows = X[st.integers(0, n - 1, half)]
    unif = _bbox_uniform(st, X, m - half)
    return Dataset(X, np.vstack([rows, unif]).astype(np.int32),
                   "W6 p=2 n=2000 gaussian x40, %d queries" % m)


def ties6(seed, n, lim, queries=4):
    """p = 6 with ties, for the largest subset size of Algorithm 1 (K = 4):
    uniform integers in [-lim, lim], then a tenth of the rows overwritten by
    copies of other rows and up to five rows placed on the line through two
    data rows (integer steps that stay inside the box); queries: a copied
    data row, another data row, the lower coordinate-wise median, then
    uniform points of the middle half of the bounding box (deep and shallow
    points alike; uniform points of the whole box are mostly outside the
    hull at p = 6)."""
    st = Stream(seed, sub=11)
    p = 6
    X = st.integers(-lim, lim, n * p).reshape(n, p).astype(np.int64)
    k = max(1, n // 10)
    src = st.integers(0, n - 1, k)
    dst = st.integers(0, n - 1, k)
    X[dst] = X[src]
    a, b = X[0].copy(), X[1].copy()
    step = b - a
    placed = 0
    for t in range(2, 40):
        if placed == 5:
            break
        v = a + t * step // 8 if t % 2 else a - t * step // 8
        if np.all(np.abs(v) <= lim):
            X[2 + placed] = v
            placed += 1
    X = X.astype(np.int32)
    med = np.sort(X, axis=0)[n // 2 - 1][None, :]
    mid = (X.min(axis=0).astype(np.int64) + X.max(axis=0)) // 2
    quarter = (X.max(axis=0).astype(np.int64) - X.min(axis=0)) // 4
    centre = np.stack([st.integers(int(mid[c] - quarter[c]), int(mid[c] + quarter[c]), max(0, queries - 3))
                       for c in range(p)], axis=1)
    Zq = np.vstack([X[dst[:1]], X[st.choice(n, 1)], med, centre])[:queries].astype(np.int32)
    return Dataset(X, Zq, "ties6 n=%d lim=%d" % (n, lim), {"seed": seed, "n": n, "lim": lim})


W7_SHAPES = ((3, 1280), (4, 640), (5, 160), (6, 80))
W7_ALPHAS = (0.0, 0.4, 0.8, 1.2)


def w7(seed=6, reps=10):
    out = []
    for si, (p, n) in enumerate(W7_SHAPES):
        for r in range(reps):
            st = Stream(seed, sub=100 * (si + 1) + r)
            X = _round_clip(40.0 * st.normal(n * p)).reshape(n, p)
            Zq = np.array([[int(round(40 * a))] * p for a in W7_ALPHAS], dtype=np.int32)
            out.append(Dataset(X, Zq, "W7[p=%d n=%d rep=%d]" % (p, n, r), {"p": p, "n": n, "rep": r}))
    return out


WORKLOADS = {"W1": w1, "W2": w2, "W4": w4, "W6": w6}
