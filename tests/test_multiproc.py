"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The data path has no collective (replicas); the ranks only agree on the
slowest rank's time, and a rank that dies is noticed on the host.
"""

import datetime
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port, timeout_s=20):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))


def _max_worker(rank, world, port, q):
    _init(rank, world, port)
    import bench
    v = bench.max_over_ranks(torch, 10.0 * (rank + 1), torch.device("cpu"))
    q.put((rank, v, bench.whole_job_gbs(8e8, world, v * 1e-3)))
    dist.destroy_process_group()


def _dying_worker(rank, world, port, q):
    _init(rank, world, port, timeout_s=5)
    import bench
    if rank == 1:
        os._exit(3)  # leaves between steps, before the next collective
    try:
        bench.max_over_ranks(torch, 1.0, torch.device("cpu"))
        q.put((rank, "no error"))
    except Exception as e:  # noqa: BLE001 - the point is that it is noticed
        q.put((rank, type(e).__name__))


def _run(target, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    out = []
    while not q.empty():
        out.append(q.get())
    for p in procs:
        if p.is_alive():
            p.kill()
    return out, [p.exitcode for p in procs]


def test_max_over_ranks_and_whole_job_value():
    out, codes = _run(_max_worker)
    assert codes == [0, 0]
    assert sorted(r for r, _, _ in out) == [0, 1]
    for _, v, gbs in out:
        assert v == 20.0  # the slowest rank's time
        assert gbs == pytest.approx(8e8 * 2 / 20e-3 / 1e9)


def test_dead_rank_is_detected_on_the_host():
    out, codes = _run(_dying_worker)
    assert codes[1] == 3
    assert out and out[0][0] == 0 and out[0][1] != "no error"


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(torch, 3.5, torch.device("cpu")) == 3.5
