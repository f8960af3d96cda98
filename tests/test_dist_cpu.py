"""The multi-process plumbing of bench.py on the CPU: two ranks over gloo,
set up from the environment torchrun gives (RANK, WORLD_SIZE, LOCAL_RANK,
MASTER_ADDR = 127.0.0.1). Every rank steps its own replica (the method has
no data-path exchange, so there is no collective on the step); the timing
collectives are a barrier and the maximum over ranks; the reference arm
runs on rank 0 only, the other ranks return without work."""
import importlib.util
import multiprocessing as mp
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location(
        "bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    try:
        bench = load_bench()

        class Args:
            gpus = ws
            steps = 1
            warmup = 0

        import torch.distributed as dist
        ref = None
        if rank != 0:
            # the reference arm sets up the group and, off rank 0, returns
            # without work (on rank 0 it would time the oracle)
            ref = bench.run_reference(Args)
            assert dist.is_initialized()
            got_ws, got_rank = dist.get_world_size(), dist.get_rank()
        else:
            got_ws, got_rank, _ = bench.dist_init(Args)
        bench.barrier(got_ws)
        mx = bench.max_over_ranks(10.0 + rank, got_ws)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, got_ws, got_rank, mx, ref))
    except Exception as e:  # report to the parent
        q.put((rank, "error", repr(e)))


def test_two_ranks_gloo():
    torch = pytest.importorskip("torch")
    assert torch.distributed.is_available()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = {o[0]: o for o in out}
    for r in range(2):
        assert res[r][1] != "error", res[r]
        _, ws, rank, mx, ref = res[r]
        assert ws == 2 and rank == r
        assert mx == 11.0  # the maximum over both ranks
        assert ref is None


def test_whole_job_value():
    bench = load_bench()
    # two replicas of 4.6 M fluid nodes, 1000 steps in 0.7 s on the slowest
    v = bench.whole_job_value(2, 4_600_000, 1000, 700.0)
    assert v == pytest.approx(2 * 4.6e6 * 1000 / 0.7 / 1e6)
    assert bench.whole_job_value(1, 10, 5, 1.0) == pytest.approx(0.05)
