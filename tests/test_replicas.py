"""Host logic of the multi-GPU bench path (replicas only), on CPU.

The bench runs one independent replica of the workload per rank and reports
the whole-job figure from the slowest rank: `max_over_ranks` must give every
rank the maximum, `barrier` must hold ranks together, and a rank that fails
before the collective must make the others' collective fail instead of hang.
Two ranks over gloo on 127.0.0.1.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, ws: int, port: int, fail_rank: int, out):
    import datetime

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=10))
    try:
        bench.barrier(ws)
        if rank == fail_rank:
            raise RuntimeError("rank leaves before the collective")
        v = bench.max_over_ranks(float(rank + 1) * 1.5, ws)
        out.put((rank, "ok", v))
    except Exception as e:   # reported to the parent, never swallowed
        out.put((rank, "error", type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(ws, fail_rank):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, fail_rank, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung"
    res = {}
    while not q.empty():
        r, status, v = q.get()
        res[r] = (status, v)
    return res


def test_max_over_ranks_gives_every_rank_the_maximum():
    res = _run(2, fail_rank=-1)
    assert res == {0: ("ok", 3.0), 1: ("ok", 3.0)}


def test_a_rank_that_fails_before_the_collective_does_not_hang_the_other():
    res = _run(2, fail_rank=1)
    assert res[1] == ("error", "RuntimeError")
    assert res[0][0] == "error"      # its all-reduce ends with an error (peer gone or timeout)


def test_single_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(2.5, 1) == 2.5
