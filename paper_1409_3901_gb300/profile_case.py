"""A small, fixed case for profiling the kernels under ncu.

    python -m paper_1409_3901_gb300.profile_case [--workload W2|W4] [--queries 4]
                                                 [--algorithm rcom|adia|critical]

Runs td_depth twice on a few queries of a benchmark workload (the first call
captures the CUDA graph, the second is the one to profile).

- rcom (Algorithm 1): with p = 4 the second call's launches are setup, tiles,
  td_k_filtered<2>, <3>, <4>, finalize, so `ncu -k regex:td_k_filtered -s 5
  -c 1` selects the p = 4 sweep kernel of the second call; with p = 5 use
  `-s 7`.
- adia (Algorithm 3): each call launches the search kernels td_k_adia<3>,
  <4> before the sweep, so with p = 4 `-k regex:td_k_adia -s 3 -c 1` selects
  the p = 4 search of the second call.
- critical (Proposition 1, r = p - 1): one td_k_critical launch per query and
  call, so with one query `-k regex:td_k_critical -s 1 -c 1` selects the
  second call's.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="W2")
    ap.add_argument("--queries", type=int, default=4)
    ap.add_argument("--algorithm", choices=["rcom", "adia", "critical"], default="rcom")
    a = ap.parse_args()
    from paper_1409_3901_gb300 import tukey, workloads as W
    d = W.WORKLOADS[a.workload]()
    pick = [0, 40, 50, 63] if a.queries == 4 and d.m == 64 else list(range(0, d.m, max(1, d.m // a.queries)))[: a.queries]
    Z = d.Zq[pick]
    alg = {"rcom": tukey.TD_ALG_RCOM, "adia": tukey.TD_ALG_ADIA, "critical": tukey.TD_ALG_CRITICAL}[a.algorithm]
    ctx = tukey.Context(0, algorithm=alg)
    ctx.depth(d.X, Z)
    out = ctx.depth(d.X, Z)
    print(out.tolist(), ctx.last_stats.as_dict())


if __name__ == "__main__":
    main()
