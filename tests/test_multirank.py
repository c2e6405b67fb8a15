"""Host logic of the multi-process benchmark path, on CPU with the gloo backend and
world_size 2: every rank solves its own problem instance (weak scaling, no data-path
collective), the step time is the maximum over ranks, and the job's throughput counts
the units of all ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench._dist()
    P, _ = bench._problem("uniform", seed_offset=r)
    t = 10.0 + 5.0 * r  # this rank's step time in ms
    t_max = bench.reduce_max(t, w, "cpu")
    v = bench.job_value(P["gas_xyz"].shape[1], w, t_max)
    q.put((r, w, local, t_max, v, float(P["gas_xyz"][0, 0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, t0, v0, x0), (r1, w1, l1, t1, v1, x1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert t0 == t1 == 15.0  # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 4096 / 15e-3)
    assert x0 != x1  # independent problem instances (seed + rank)


def test_single_rank_passthrough():
    import bench
    assert bench.reduce_max(3.5, 1, "cpu") == 3.5
    assert bench.job_value(100, 1, 10.0) == pytest.approx(1e4)
    assert np.isfinite(bench.job_value(4096, 4, 1.0))
