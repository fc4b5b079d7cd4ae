"""The N-replica path of bench.py on CPU ranks (gloo, world size 2): the
step time is the slowest rank's, the value the whole job's, and the
reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    td.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist() == (ws, rank, rank)
        ms, value = bench.aggregate(100.0 + 50.0 * rank, ws)   # rank 1 is the slower replica
        bench.barrier(ws)

        class Args:
            warmup, steps, gpus = 3, 1, ws
        out = None
        if rank != 0:
            out = bench.run_reference(Args())  # non-zero ranks return without work
        q.put((rank, ms, value, out))
    finally:
        td.destroy_process_group()


def test_two_cpu_ranks_aggregate_and_gate():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, ms, value, out in res:
        assert ms == 150.0
        assert value == pytest.approx(2 * 1e3 / 150.0)
        assert out is None


def test_failing_extra_is_recorded_not_raised():
    """An extra workload that raises is reported as an error entry, so the
    bench's headline line is still printed."""
    import bench

    def bad(*_):
        raise RuntimeError("out of memory on the extra workload")
    assert bench.run_extra(lambda a, b: {"n_it": a + b}, 1, 2) == {"n_it": 3}
    got = bench.run_extra(bad, None, None)
    assert set(got) == {"error"} and got["error"].startswith("RuntimeError: out of memory")
