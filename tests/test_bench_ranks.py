"""The multi-rank path of bench.py on the CPU: two gloo ranks (world size 2,
as torchrun would start them) agree on the slowest rank's time, the
whole-job rate counts every rank's replica, only rank 0 prints, and the
reference arm's non-zero ranks exit without work."""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, _, w = bench.dist_env()
    ms = bench.max_over_ranks(100.0 + 40.0 * rank, w, "cpu")  # rank 1 is slower
    e2e = bench.max_over_ranks(0.2 - 0.05 * rank, w, "cpu")   # rank 0 is slower
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.emit({"rank": r, "value": bench.whole_job_rate(w, ms * 1e-3)}, r)
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, w, ms, e2e, buf.getvalue()))


def test_two_gloo_ranks_agree_on_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[:2] for x in res] == [(0, 2), (1, 2)]
    assert all(x[2] == 140.0 for x in res)           # max over ranks of the step time
    assert all(abs(x[3] - 0.2) < 1e-15 for x in res)  # and of the end-to-end time
    printed = [x[4] for x in res]
    assert printed[1] == ""                           # rank 1 prints nothing
    line = json.loads(printed[0])
    assert line["rank"] == 0 and abs(line["value"] - 2 / 0.140) < 1e-12


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(1, 0.25) == 4.0


def test_reference_arm_non_zero_rank_exits_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        n = 512
        steps = 1
        warmup = 0
        gpus = 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args()) == 0
    assert buf.getvalue() == ""
