"""Multi-rank path.  On the CPU: two gloo ranks split each query's subset
loop (Algorithm 1, Section 3) into contiguous position ranges, compute their
partial minima with the oracle, and merge them with an all-reduce MIN; the
merge must give the depth.  A rank that drops out before the merge is
detected on the host (the barrier times out) and never yields a partial
result.  On the GPU: the product path itself (tukey.depth_sharded), two
gloo ranks each running the library's shard on device 0 (kernels that never
wait on each other) and merging with the MIN all-reduce."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _shard_range(npos, s, S):
    """Contiguous shard s of S over positions [0, npos) (as in the set-up kernel)."""
    return npos * s // S, npos * (s + 1) // S


def _worker(rank, world, port, X, Zq, out_path, drop):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    if drop and rank == 1:
        os._exit(0)  # leaves between steps, before the merge
    parts = []
    for z in Zq:
        _, npos, _ = oracle.depth_range(X, z, 0, 1)
        lo, hi = _shard_range(npos, rank, world)
        part, _, _ = oracle.depth_range(X, z, lo, hi)
        parts.append(np.iinfo(np.int32).max if part is None else part)
    t = torch.tensor(parts, dtype=torch.int64)
    try:
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        ok = True
    except Exception:
        ok = False
    if rank == 0:
        np.save(out_path, t.numpy() if ok else np.array([-1]))
    try:
        dist.destroy_process_group()
    except Exception:
        pass


def _case():
    rng = np.random.default_rng(21)
    X = rng.integers(-6, 7, size=(18, 4)).astype(np.int32)
    X[3] = X[7]
    Zq = np.vstack([X[:2], rng.integers(-4, 5, size=(2, 4))]).astype(np.int32)
    return X, Zq


def test_two_gloo_ranks_merge_to_depth(tmp_path):
    import oracle
    X, Zq = _case()
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_worker, args=(2, _free_port(), X, Zq, out, False), nprocs=2, start_method="spawn")
    merged = np.load(out)
    assert np.array_equal(merged, oracle.depth_many(X, Zq))


def test_rank_dropout_gives_no_result(tmp_path):
    X, Zq = _case()
    out = str(tmp_path / "merged.npy")
    try:
        mp.start_processes(_worker, args=(2, _free_port(), X, Zq, out, True), nprocs=2, start_method="spawn")
    except Exception:
        pass
    if os.path.exists(out):
        assert np.array_equal(np.load(out), np.array([-1]))


def test_shard_ranges_partition():
    for npos in (1, 7, 499500, 1313400):
        for S in (1, 2, 3, 8):
            rs = [_shard_range(npos, s, S) for s in range(S)]
            assert rs[0][0] == 0 and rs[-1][1] == npos
            assert all(a[1] == b[0] for a, b in zip(rs[:-1], rs[1:]))


def _lib_worker(rank, world, port, X, Zq, out_path):
    import torch
    import torch.distributed as dist
    from paper_1409_3901_gb300 import tukey
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    merged = tukey.depth_sharded(X, Zq, device=0)
    ctx = tukey.Context(0, shard_index=rank, shard_count=world)
    own = ctx.depth(X, Zq)                     # this rank's shard alone
    np.save(out_path + ".%d.npy" % rank, np.stack([merged, own]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.gpu
def test_library_shards_on_two_ranks_merge_to_depth(tmp_path):
    """tukey.depth_sharded on two gloo ranks sharing device 0: the merged MIN
    equals the oracle's depth on both ranks, and so does the minimum of the
    two ranks' own shards (W1, p = 3, and a p = 4 tie case)."""
    import oracle
    from gpu_common import load_golden
    from paper_1409_3901_gb300 import workloads as W
    g = load_golden("W1")
    d = W.w1()
    assert d.checksum() == g["checksum"]
    rng = np.random.default_rng(22)
    X4 = rng.integers(-8, 9, size=(40, 4)).astype(np.int32)
    X4[5:9] = X4[0]
    Z4 = np.vstack([X4[:3], rng.integers(-5, 6, size=(3, 4))]).astype(np.int32)
    for X, Zq, want in ((d.X, d.Zq, np.array(g["T"])), (X4, Z4, oracle.depth_many(X4, Z4))):
        out = str(tmp_path / "m")
        mp.start_processes(_lib_worker, args=(2, _free_port(), X, Zq, out), nprocs=2, start_method="spawn")
        r0, r1 = np.load(out + ".0.npy"), np.load(out + ".1.npy")
        assert np.array_equal(r0[0], want) and np.array_equal(r1[0], want)
        assert np.array_equal(np.minimum(r0[1], r1[1]), want)
