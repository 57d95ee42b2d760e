"""Host logic of the multi-GPU benchmark (replicas, weak scaling) on CPU ranks
over gloo: the timed region is the max over ranks and the whole-job value
counts every rank's lattice updates."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 2.0 * rank
    t = bench.reduce_max_ms(local_ms, dist, "cpu")
    q.put((rank, t, bench.job_mlups(1000, 5, world, t), bench.env_rank()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [12.0, 12.0]
    assert res[0][2] == pytest.approx(1000 * 5 * 2 / 12e-3 / 1e6)
    assert res[0][3][:2] == (0, 2) and res[1][3][:2] == (1, 2)
