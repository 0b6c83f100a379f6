"""The benchmark's multi-rank logic on CPU: world_size 2 over gloo (127.0.0.1).  Replicas
share no data; the only collectives are the timing barrier and the max over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from tests.conftest import ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": "2",
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup(2, backend="gloo")
    bench.barrier(ws)
    elapsed = 1.0 + r            # rank 1 is the slow replica
    m = bench.max_over_ranks(ws, elapsed)
    rate = bench.whole_job_rate(ws, 10.0, elapsed)
    out.put((r, ws, local, m, rate))
    dist.destroy_process_group()


def test_two_rank_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, ws, local, m, rate) in enumerate(res):
        assert rank == r and ws == 2 and local == r
        assert m == 2.0                      # max over ranks
        assert rate == pytest.approx(10.0)   # 2 replicas x 10 units / 2 s


def test_reference_arm_only_rank0_prints(capsys, monkeypatch):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        gpus, steps, warmup = 2, 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
