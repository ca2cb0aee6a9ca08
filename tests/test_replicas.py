"""The multi-GPU form is replicas only (independent pairs per rank, no
data-path collective): the benchmark's cross-rank timing reduction and
whole-job throughput, exercised with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as d
    import bench
    d.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r took (r + 1) ms for the device loop and (10 - r) ms end to end
        ms, ms_e2e = bench.replica_reduce(d, [rank + 1.0, 10.0 - rank], "cpu")
        out.put((rank, ms, ms_e2e, bench.replica_value(ws, 5, ms)))
    finally:
        d.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, ms_e2e, value in res:
        assert ms == 2.0 and ms_e2e == 10.0  # max over ranks, on every rank
        assert value == pytest.approx(2 * 5 / 2e-3)  # both replicas' units over the slowest time


def test_single_process_needs_no_group():
    import bench
    assert bench.replica_reduce(None, [3.0, 4.0], "cpu") == [3.0, 4.0]
    assert bench.replica_value(1, 50, 25.0) == pytest.approx(2000.0)
