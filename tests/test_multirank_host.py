"""Host-side logic of the multi-rank benchmark path on CPU (gloo, world size 2): replicas only,
no collective on the data path; the timing reduction takes the max over ranks and the
whole-job value counts every rank's work. The reference arm prints on rank 0 only."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    total_ms = 1000.0 + 500.0 * rank  # rank 1 is slower
    per_rank = bench.gather_rank_times(total_ms, world)
    value, ms_per_step = bench.aggregate(per_rank, pairs_per_step=1e10, steps=4)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, per_rank, value, ms_per_step))


def test_rank_times_max_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, per_rank, value, ms_per_step in out:
        assert per_rank == [1000.0, 1500.0]
        # 2 ranks x 4 steps x 1e10 pairs over the slowest rank's 1.5 s
        assert abs(value - 2 * 4 * 1e10 / 1.5) < 1e-3 * value
        assert ms_per_step == 1500.0 / 4


def test_reference_arm_silent_on_other_ranks(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-rows", "8"])
    assert rc == 0 and buf.getvalue() == ""
