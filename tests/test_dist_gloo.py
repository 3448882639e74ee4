"""The N > 1 path on CPU: world_size-2 gloo ranks shard the shots, decode their share (with the
oracle, standing in for each rank's GPU), and reduce counters and timing exactly like bench.py."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2508_15743_gb300 import dist as VD  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import oracle
    from paper_2508_15743_gb300 import dem as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, 16, 2)
    syn, obs = D.sample(dm, 600, 77)
    lo, hi = VD.shard_range(len(syn), rank, world)
    r = oracle.decode(dm, perms, syn[lo:hi], 30, 0.625, 5, nthreads=1, want_soft=False)
    fails = int((r["logical"] != obs[lo:hi]).any(axis=1).sum())
    counters = [hi - lo, fails, int(r["stats"]["lsd_invoked"].sum())]
    tot = VD.reduce_sum_counters(counters)
    tmax = VD.reduce_max(float(rank + 1))
    # gather the shards' corrections on rank 0 to compare with one process doing all shots
    parts = [None] * world
    dist.all_gather_object(parts, (lo, hi, r["corrections"]))
    if rank == 0:
        np.save(out_path, np.array([*tot, tmax], dtype=np.float64))
        corr = np.concatenate([p[2] for p in sorted(parts, key=lambda x: x[0])])
        np.save(out_path + ".corr.npy", corr)
    dist.destroy_process_group()


def test_shard_range_partitions():
    for total in [0, 1, 7, 1000, 1001]:
        for world in [1, 2, 3, 8]:
            spans = [VD.shard_range(total, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [h - l for l, h in spans]
            assert max(sizes) - min(sizes) <= 1
    assert VD.rank_seed(2, 0) == 2 and VD.rank_seed(2, 3) != VD.rank_seed(2, 2)


def test_two_gloo_ranks_match_one_process(tmp_path):
    import oracle
    from paper_2508_15743_gb300 import dem as D
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    tot = np.load(out)
    corr = np.load(out + ".corr.npy")
    dm = D.build_workload("cc666_d9_pheno")
    perms = D.schedules(dm.n, 16, 2)
    syn, obs = D.sample(dm, 600, 77)
    r = oracle.decode(dm, perms, syn, 30, 0.625, 5, nthreads=2, want_soft=False)
    assert np.array_equal(corr, r["corrections"])
    assert tot[0] == 600
    assert tot[1] == (r["logical"] != obs).any(axis=1).sum()
    assert tot[2] == r["stats"]["lsd_invoked"].sum()
    assert tot[3] == 2.0   # max over ranks of (rank + 1)
