"""Helpers shared by the GPU parity tests."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def load_golden(name):
    path = os.path.join(GOLDEN, name + ".json")
    if not os.path.exists(path):
        pytest.skip("golden file %s.json not generated" % name)
    with open(path) as f:
        return json.load(f)


def random_case(rng, p, n, lim, tie_rate=0.3):
    X = rng.integers(-lim, lim + 1, size=(n, p))
    if n > 2 and rng.random() < tie_rate:
        k = int(rng.integers(1, max(2, n // 5)))
        src = rng.integers(0, n, size=k)
        dst = rng.integers(0, n, size=k)
        X[dst] = X[src]
    return X.astype(np.int32)
