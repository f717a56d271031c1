"""The replica timing logic over a real 2-rank gloo process group on CPU:
every rank sees the slowest rank's time and the same whole-job rate."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2302_05662_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = 10.0 + 5.0 * rank          # rank 1 is slower
        t = replicas.max_over_ranks(local_ms)
        rate = replicas.whole_job_rate(1e6, 4, world, t)
        out[rank] = (t, rate)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_max_and_rate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    t, rate = out[0]
    assert t == 15.0
    assert rate == pytest.approx(1e6 * 4 * 2 / 0.015)


def test_single_process_identity():
    from paper_2302_05662_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.whole_job_rate(10, 2, 1, 1000.0) == 20.0
