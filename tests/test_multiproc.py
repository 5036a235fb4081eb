"""The multi-rank path of the benchmark on CPU: two gloo ranks over
127.0.0.1.  Each rank solves its own instance (replicas, weak scaling), the
job time is the maximum over ranks of each rank's timed total, the value is
that time over all ranks' instances, and only rank 0 reports; the reference
arm does no work on other ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local = 10.0 * (rank + 1) + 0.5
    total = bench.job_time_ms(local, ws)
    got_ws, got_rank, got_local = bench.dist_env()
    out[rank] = (total, bench.job_value(total, ws, 3), got_ws, got_rank, got_local)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    ws, port = 2, _free_port()
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for rank in range(ws):
        total, value, got_ws, got_rank, got_local = out[rank]
        assert total == 20.5  # the slower rank's total
        assert value == pytest.approx(20.5 / (ws * 3))
        assert (got_ws, got_rank, got_local) == (ws, rank, rank)


def test_reference_arm_does_no_work_off_rank_0(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 1, 2
    # returns before importing or running the oracle
    assert bench.run_reference(A()) is None


def test_replica_instances_differ_by_rank():
    sys.path.insert(0, ROOT)
    import bench
    a, b = bench.make_instance(seed=0, side=64), bench.make_instance(seed=1, side=64)
    assert a.dims == b.dims and a.conn == b.conn == 8
    assert (a.cs != b.cs).any()


def test_batch_replicas_differ_by_rank_and_reference_covers_the_batch():
    sys.path.insert(0, ROOT)
    import bench
    a = bench.batch_instances(batch_seed=0, only=[3, 400])
    b = bench.batch_instances(batch_seed=1, only=[3, 400])
    assert a[0].conn == 4 and a[1].conn == 6
    assert (a[0].dims != b[0].dims) or (a[0].cs.shape != b[0].cs.shape) or (a[0].cs != b[0].cs).any()
    for steps in (1, 3, 20, 600):
        shares = bench.reference_shares(512, steps)
        flat = sorted(i for sh in shares for i in sh)
        assert flat == list(range(512)) and len(shares) == steps
