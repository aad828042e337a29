"""Write the stored expected depth counts under tests/golden/ (CPU only).

Every value written here comes from the CPU oracle (``oracle/``) applied to the
seeded workloads of ``paper_1409_3901_gb300.workloads``; each file records the
input checksum so that a test on another machine first checks that it
regenerated the same inputs.  Queries are spread over worker processes
(``spawn`` start method); the oracle code is the same in each.

    python tests/golden/make_golden.py W1 W2 W4 W6 W3S W5S W1A W2A W7A W3SA W5SA [--procs 8]

W3S and W5S are bounded samples of the batched and stream workloads: every
query of the datasets (requests) whose full oracle cost is small.  W1A, W2A,
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
