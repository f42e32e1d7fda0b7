"""The multi-rank path of the benchmark on CPU: two gloo ranks run the same
host logic as the GPU job (process group, barrier, slowest-rank time, band
per rank, job throughput)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init(ws, backend="gloo")
    step_ms = 10.0 + 5.0 * r                     # rank 1 is the slow one
    slowest = bench.max_over_ranks(step_ms, w)
    bench.barrier(w)
    band = bench.rank_channels(r, 64)
    value = bench.job_value(w, 1000.0, slowest)
    q.put((r, w, local, slowest, band, value))
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_two_gloo_ranks(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == list(range(ws))
    assert all(r[1] == ws and r[2] == r[0] for r in res)
    assert all(r[3] == 15.0 for r in res)                       # max over ranks
    bands = [r[4] for r in res]
    assert bands == [(0, 64), (64, 128)]                       # disjoint bands
    assert all(r[5] == pytest.approx(ws * 1000.0 / 15e-3) for r in res)


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A(), 2, 1) is None
