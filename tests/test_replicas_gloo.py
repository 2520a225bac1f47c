"""Multi-process replica logic on CPU with the gloo backend (world size 2):
ranks draw distinct shards, the timer is reduced with max over ranks, and the
whole-job rate counts every rank's angles."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    from paper_2502_10831_gb300 import replicas as R
    from paper_2502_10831_gb300 import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = R.rank_env()
    x = W.bandwidth(1 << 12, seed=R.shard_seed(W.SEED, r))
    local_ms = 10.0 + 5.0 * r  # pretend rank 1 is slower
    dist.barrier()
    worst = R.max_over_ranks(local_ms, dist)
    rate = R.job_throughput(x.size, w, worst * 1e-3)
    out[rank] = (r, w, lr, float(x[:8].sum()), worst, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert sorted(res) == [0, 1]
    (r0, w0, l0, s0, m0, q0), (r1, w1, l1, s1, m1, q1) = res[0], res[1]
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert s0 != s1  # distinct shards
    assert m0 == m1 == 15.0  # both ranks see the slowest rank's time
    assert q0 == q1 == pytest.approx(2 * (1 << 12) / 15e-3)


def test_single_process_defaults():
    from paper_2502_10831_gb300 import replicas as R
    assert R.max_over_ranks(3.5) == 3.5
    assert R.job_throughput(100, 1, 2.0) == 50.0
    assert R.shard_seed(7, 3) == 10
    assert np.isfinite(R.job_throughput(1, 8, 1e-3))
