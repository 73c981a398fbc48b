"""The N > 1 benchmark path (independent replicas) on two gloo ranks on the CPU:
the slowest rank's time and the job throughput reach every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = torch.distributed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, ms_per_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2103_03348_b300 import replicas
        replicas.barrier()
        value, ms = replicas.aggregate_throughput(1.0e10, ms_per_rank[rank])
        out.put((rank, value, ms, replicas.world()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_slowest_rank():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms = [7.0, 9.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, m, w in res:
        assert w == 2 and m == 9.0
        assert abs(value - 2 * 1.0e10 / 9.0e-3) <= 1e-6 * value


def test_single_process_is_identity():
    from paper_2103_03348_b300 import replicas
    value, ms = replicas.aggregate_throughput(1.0e10, 5.0)
    assert ms == 5.0 and abs(value - 2.0e12) <= 1e-3
