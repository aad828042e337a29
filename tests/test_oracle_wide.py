"""Pins of the full-range oracle (oracle/tukey_wide.py): int32 data of any
magnitude, where the C oracle's 128-bit arithmetic gives out.

  - On inputs both accept it equals the C oracle (itself pinned by the brute
    forces of test_oracle.py).
  - At full-range magnitudes it equals the sign-vector brute force of Eq. (1)
    (tests/bruteforce.py, Python integers throughout).
  - Eq. (1) is invariant under positive scaling of the centred data and
    under invertible linear maps: in-range data scaled up to the int32 range,
    or mapped by an integer unimodular matrix with large entries, keeps the
    C oracle's count of the original data.
"""
import numpy as np
import pytest

import oracle
from bruteforce import depth_bruteforce
from oracle import tukey_wide as wide

INT32_MAX = 2 ** 31 - 1


def _ties(rng, p, n, lim):
    X = rng.integers(-lim, lim + 1, size=(n, p)).astype(np.int64)
    X[-2:] = X[:2]                                   # duplicates
    return X


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_wide_oracle_equals_c_oracle_in_range(p):
    rng = np.random.default_rng(600 + p)
    n = {1: 20, 2: 20, 3: 14, 4: 11, 5: 10, 6: 9}[p]
    for trial in range(6):
        X = _ties(rng, p, n, int(rng.choice([2, 5, 40]))).astype(np.int32)
        z = X[trial % n] if trial % 2 else rng.integers(-3, 4, size=p).astype(np.int32)
        assert wide.depth(X, z) == oracle.depth(X, z)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_wide_oracle_equals_bruteforce_at_full_range(p):
    rng = np.random.default_rng(650 + p)
    n = {2: 10, 3: 9, 4: 8, 5: 8}[p]
    for trial in range(4):
        X = rng.integers(-INT32_MAX, INT32_MAX, size=(n, p), dtype=np.int64)
        X[-1] = X[0]                                 # a duplicate
        X[-2] = X[1] if trial % 2 else -X[1]         # a repeat or a mirror image
        z = X[2] if trial < 2 else rng.integers(-INT32_MAX, INT32_MAX, size=p, dtype=np.int64)
        z = np.asarray(z, np.int64)
        if trial == 3:
            z = np.zeros(p, np.int64)
            X[3] = -X[4]                             # collinear with z
        assert wide.depth(X, z) == depth_bruteforce(X, z), (p, trial)


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_wide_oracle_scaling_and_unimodular_invariance(p):
    """Centred data scaled by a positive integer up to the int32 range, and
    mapped by a unimodular matrix with entries up to ~2^20, keep the count."""
    rng = np.random.default_rng(700 + p)
    n = {3: 12, 4: 10, 5: 9, 6: 8}[p]
    for trial in range(3):
        lim = 6
        X = _ties(rng, p, n, lim)
        z = X[0] if trial == 0 else rng.integers(-2, 3, size=p)
        want = oracle.depth(X.astype(np.int32), np.asarray(z, np.int32))
        x = X - z
        k = (INT32_MAX - 4) // (2 * lim + 4)         # |z + k x| < 2^31
        Xs = z + k * x
        assert np.abs(Xs).max() > 2 ** 28
        assert wide.depth(Xs, z) == want
        # an integer unimodular map: identity plus one large upper entry, then
        # a permutation; applied to the centred data (entries stay in int32)
        U = np.eye(p, dtype=np.int64)
        U[0, p - 1] = int(rng.integers(2 ** 18, 2 ** 20))
        U = U[rng.permutation(p)]
        Xu = x @ U.T
        assert np.abs(Xu).max() < 2 ** 31
        assert wide.depth(Xu, np.zeros(p, np.int64)) == want
