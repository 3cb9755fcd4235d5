"""The bench's multi-rank path on the host: two gloo ranks on CPU (one process per
GPU on a GPU machine). Each rank runs its own replica; the job value is the pushes of all
ranks over the slowest rank's time, and only rank 0 of the reference arm does work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    r, w, _ = bench.dist_setup(n_gpus=world)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = bench.max_over_ranks(10.0 + r, w)          # rank 1 is the slower one
    pushes = bench.sum_over_ranks(1000.0 * (r + 1), w)
    q.put((r, w, ms, pushes, bench.job_value(pushes, ms)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    out = sorted(q.get(timeout=5) for _ in range(2))
    for r, w, ms, pushes, value in out:
        assert w == 2
        assert ms == 11.0 and pushes == 3000.0
        assert value == pytest.approx(3000.0 / 0.011)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")

    class Args:
        nx, ny, workload, total, steps, warmup, gpus = 2048, 512, "lwfa", 0, 1, 1, 2

    assert bench.reference_arm(Args()) is None
    assert capsys.readouterr().out == ""
