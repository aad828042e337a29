"""The stored expected values under tests/golden/ against the generators and
the oracle (CPU): every file's input checksum must match the regenerated
workload, and the affordable part of each file is recomputed by the oracle."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1409_3901_gb300 import workloads as W

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(HERE, name + ".json")) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["W1", "W2", "W4", "W6"])
def test_checksums_match_generators(name):
    g = _load(name)
    d = W.WORKLOADS[name]()
    assert g["checksum"] == d.checksum()
    assert len(g["T"]) == d.m
    assert all(0 <= t <= d.n for t in g["T"])


def test_w1_recomputed():
    g = _load("W1")
    d = W.w1()
    assert np.array_equal(oracle.depth_many(d.X, d.Zq), np.array(g["T"]))


def test_w6_sample_recomputed():
    g = _load("W6")
    d = W.w6()
    idx = np.arange(0, d.m, d.m // 256)
    assert np.array_equal(oracle.depth_many(d.X, d.Zq[idx]), np.array(g["T"])[idx])


@pytest.mark.parametrize("name", ["W3S", "W5S"])
def test_sampled_items(name):
    g = _load(name)
    sets = W.w3() if name == "W3S" else W.w5()
    from math import comb
    items = sorted(g["items"], key=lambda it: comb(it["n"], max(it["p"] - 2, 0)) * it["n"] * it["m"])
    assert items
    for it in g["items"]:
        assert sets[it["index"]].checksum() == it["checksum"]
    # recompute the two cheapest
    for it in items[:2]:
        d = sets[it["index"]]
        assert np.array_equal(oracle.depth_many(d.X, d.Zq), np.array(it["T"]))
