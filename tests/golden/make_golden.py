"""Write the stored expected depth counts under tests/golden/ (CPU only).

Every value written here comes from the CPU oracle (``oracle/``) applied to the
seeded workloads of ``paper_1409_3901_gb300.workloads``; each file records the
input checksum so that a test on another machine first checks that it
regenerated the same inputs.  Queries are spread over worker processes
(``spawn`` start method); the oracle code is the same in each.

    python tests/golden/make_golden.py W1 W2 W4 W6 W3S W5S W3L P6 SHARDS W1A W2A W7A W3SA W5SA [--procs 8]

W3S and W5S are bounded samples of the batched and stream workloads: every
query of the datasets (requests) whose full oracle cost is small.  W3L covers
the W3 datasets that W3S leaves out (the large p = 4 and p = 5 ones): the
largest-n dataset of each p with queries 0, 1 (data rows) and 8, 9 (uniform
points), and a seeded stratified sample of the others (two per third of each
p's n range) with queries 0 and 8.  Each of its queries is split into
contiguous ranges of subset positions, evaluated by oracle.depth_range in
parallel, and merged by an exact minimum (the minimum over a partition of the
positions is the depth).  P6 holds every query of two p = 6 sets with ties
(workloads.ties6: n = 64 in [-4, 4], n = 120 in [-127, 127]).  SHARDS holds
Z + min V(S) over sampled contiguous ranges of the library's colex subset
positions (tests/subsets.py) where a whole query is too costly for the
oracle: the p = 6 tie set with n = 300 and the three costliest p = 5
requests among the first 400 of the W5 stream; each value comes from
oracle.subset_min over the subsets of the range.  W1A, W2A,
W7A, W3SA and W5SA hold the counts of Algorithm 3 (ADIA, the oracle's
oracle.adia) on W1, W2, W7, the first 40 datasets of W3S and the first 30
requests of W5S.
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time
from math import comb

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

from paper_1409_3901_gb300 import workloads as W  # noqa: E402

# per-query oracle cost budget for the sampled workloads (point-subset slots)
SAMPLE_COST = 6e7


def _one(args):
    import oracle
    X, z = args
    return oracle.depth(X, z)


def _one_adia(args):
    import oracle
    X, z = args
    return oracle.adia(X, z)[0]


def _one_range(args):
    import oracle
    X, z, lo, hi = args
    return oracle.depth_range(X, z, lo, hi)[0]


def _positions(args):
    import oracle
    X, z = args
    return oracle.depth_range(X, z, 0, 0)[1]


# W3L: queries of the largest datasets and of the stratified sample, and
# ranges per query
W3L_QUERIES_MAX = (0, 1, 8, 9)
W3L_QUERIES = (0, 8)
W3L_CHUNKS = 16


def w3l_pick(sets, covered):
    """The W3 datasets of W3L: for p = 4 and 5, among those not in `covered`,
    the largest n (queries W3L_QUERIES_MAX) and two per third of the n-sorted
    rest (seeded, queries W3L_QUERIES).  Returns [(index, queries)]."""
    rng = np.random.default_rng(7)
    picks = []
    for p in (4, 5):
        cand = sorted((d.n, i) for i, d in enumerate(sets) if d.p == p and i not in covered)
        picks.append((cand[-1][1], W3L_QUERIES_MAX))
        rest = cand[:-1]
        for stratum in np.array_split(np.arange(len(rest)), 3):
            for c in sorted(rng.choice(stratum, size=2, replace=False)):
                picks.append((rest[c][1], W3L_QUERIES))
    return sorted(picks)


def _run_ranges(pool, jobs):
    """jobs: [(key, X, z)] -> {key: depth}, each query split into W3L_CHUNKS
    ranges of subset positions and merged by the minimum."""
    npos = pool.map(_positions, [(X, z) for _, X, z in jobs], chunksize=1)
    tasks, keys = [], []
    for (key, X, z), n in zip(jobs, npos):
        step = max(1, -(-n // W3L_CHUNKS))
        for lo in range(0, max(n, 1), step):
            tasks.append((X, z, lo, min(n, lo + step)))
            keys.append(key)
    best = {}
    done = 0
    for key, part in zip(keys, pool.imap(_one_range, tasks, chunksize=1)):
        done += 1
        if part is not None:
            best[key] = min(best.get(key, part), part)
        if done % 64 == 0:
            print("  %d / %d ranges" % (done, len(tasks)), flush=True)
    for key, X, z in jobs:
        if key not in best:          # no independent subset anywhere: the oracle's other branches
            best[key] = _one((X, z))
    return best


def _one_subsets(args):
    import oracle
    X, z, subs = args
    return oracle.subset_min(X, z, subs)[0]


P6_SETS = ((61, 64, 4), (62, 120, 127))
SHARD_COUNT = 4096          # ranges per query of the sampled items
SHARD_PICKS = 8             # ranges sampled per query: the first, the last and 6 seeded


def shard_items():
    """(name, Dataset, query indices, shard indices) of the SHARDS file."""
    rng = np.random.default_rng(8)
    picks = lambda: sorted({0, SHARD_COUNT - 1} | set(int(v) for v in rng.choice(SHARD_COUNT - 2, 6,
                                                                                    replace=False) + 1))
    out = [("ties6 n=300", W.ties6(63, 300, 60), [0, 1, 2, 3], picks())]
    reqs = [(comb(d.n, d.p - 2) * d.n, i, d) for i, d in enumerate(W.w5(count=400)) if d.p == 5]
    for _, i, d in sorted(reqs, reverse=True)[:3]:
        qs = [0, d.m - 1] if d.m > 1 else [0]
        out.append(("W5[%d]" % i, d, qs, picks()))
    return out


def _run(pool, X, Zq, fn=_one):
    return [int(v) for v in pool.map(fn, [(X, z) for z in Zq], chunksize=1)]


def _cost(d):
    return comb(d.n, max(d.p - 2, 0)) * d.n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+")
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    a = ap.parse_args()
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool:
        for name in a.names:
            t0 = time.time()
            if name in ("W1", "W2", "W4", "W6"):
                d = W.WORKLOADS[name]()
                out = {"workload": name, "description": d.name, "checksum": d.checksum(),
                       "n": d.n, "p": d.p, "m": d.m, "T": _run(pool, d.X, d.Zq)}
            elif name in ("W1A", "W2A"):
                d = W.WORKLOADS[name[:2]]()
                out = {"workload": name[:2], "algorithm": "Algorithm 3 (ADIA)", "description": d.name,
                       "checksum": d.checksum(), "n": d.n, "p": d.p, "m": d.m,
                       "T": _run(pool, d.X, d.Zq, _one_adia)}
            elif name == "W3SA":
                sets = W.w3()
                base = json.load(open(os.path.join(HERE, "W3S.json")))
                items = []
                for it in base["items"][:40]:
                    d = sets[it["index"]]
                    items.append({"index": it["index"], "checksum": d.checksum(), "n": d.n, "p": d.p,
                                  "m": d.m, "T": _run(pool, d.X, d.Zq, _one_adia)})
                out = {"workload": "W3", "algorithm": "Algorithm 3 (ADIA)",
                       "sample": "the first 40 datasets of W3S", "items": items}
            elif name == "W5SA":
                base = json.load(open(os.path.join(HERE, "W5S.json")))
                items = []
                for it in base["items"][:30]:
                    d = W.w5_request(4, it["index"])
                    items.append({"index": it["index"], "checksum": d.checksum(), "n": d.n, "p": d.p,
                                  "m": d.m, "T": _run(pool, d.X, d.Zq, _one_adia)})
                out = {"workload": "W5", "algorithm": "Algorithm 3 (ADIA)",
                       "sample": "the first 30 requests of W5S", "items": items}
            elif name == "W7A":
                items = []
                for i, d in enumerate(W.w7()):
                    items.append({"index": i, "checksum": d.checksum(), "n": d.n, "p": d.p, "m": d.m,
                                  "T": _run(pool, d.X, d.Zq, _one_adia)})
                out = {"workload": "W7", "algorithm": "Algorithm 3 (ADIA)", "items": items}
            elif name == "W3L":
                sets = W.w3()
                covered = {it["index"] for it in json.load(open(os.path.join(HERE, "W3S.json")))["items"]}
                picks = w3l_pick(sets, covered)
                jobs = [((i, q), sets[i].X, sets[i].Zq[q]) for i, qs in picks for q in qs]
                got = _run_ranges(pool, jobs)
                items = []
                for i, qs in picks:
                    d = sets[i]
                    items.append({"index": i, "checksum": d.checksum(), "n": d.n, "p": d.p, "m": d.m,
                                  "queries": list(qs), "T": [int(got[(i, q)]) for q in qs]})
                out = {"workload": "W3", "sample": "datasets not in W3S: the largest n for p = 4 and "
                       "p = 5 (queries %s) and two per third of the rest of each p's n range "
                       "(seed 7; queries %s)" % (list(W3L_QUERIES_MAX), list(W3L_QUERIES)), "items": items}
            elif name == "P6":
                sets = [W.ties6(*a) for a in P6_SETS]
                got = _run_ranges(pool, [((j, q), d.X, d.Zq[q]) for j, d in enumerate(sets) for q in range(d.m)])
                out = {"workload": "ties6 (p = 6 with ties)", "items": [
                    {"args": list(a), "checksum": d.checksum(), "n": d.n, "p": d.p, "m": d.m,
                     "T": [int(got[(j, q)]) for q in range(d.m)]} for j, (a, d) in enumerate(zip(P6_SETS, sets))]}
            elif name == "SHARDS":
                from subsets import colex_range, shard_range
                items, tasks = [], []
                for label, d, qs, shards in shard_items():
                    for q in qs:
                        z = d.Zq[q]
                        nnz = int(d.n - np.all(d.X == z, axis=1).sum())
                        for s_ in shards:
                            lo, hi = shard_range(nnz, d.p - 2, s_, SHARD_COUNT)
                            tasks.append((d.X, z, np.array(colex_range(d.p - 2, lo, hi), np.int32)))
                            items.append({"dataset": label, "checksum": d.checksum(), "query": q,
                                          "shard_index": s_, "shard_count": SHARD_COUNT, "lo": lo, "hi": hi})
                vals = pool.map(_one_subsets, tasks, chunksize=1)
                for it, v in zip(items, vals):
                    it["value"] = None if v is None else int(v)
                out = {"sample": "Z + min V(S) over colex ranks [lo, hi) of the nonzero points, shard "
                       "shard_index of shard_count (tests/subsets.py)", "items": items}
            elif name in ("W3S", "W5S"):
                sets = W.w3() if name == "W3S" else W.w5()
                items = []
                for i, d in enumerate(sets):
                    if _cost(d) <= SAMPLE_COST:
                        items.append({"index": i, "checksum": d.checksum(), "n": d.n, "p": d.p,
                                      "m": d.m, "T": _run(pool, d.X, d.Zq)})
                out = {"workload": name[:2], "sample": "every query of the datasets with "
                       "C(n,p-2)*n <= %.0e" % SAMPLE_COST, "items": items}
            else:
                raise SystemExit("unknown workload " + name)
            out["source"] = "oracle/tukey_oracle.c via tests/golden/make_golden.py"
            path = os.path.join(HERE, name + ".json")
            with open(path, "w") as f:
                json.dump(out, f, indent=1)
            print("%s written in %.1f s" % (path, time.time() - t0), flush=True)


if __name__ == "__main__":
    main()
