"""Host side of the sharded evaluation, on the CPU: the shard ranges partition
the events and the exchange buffer, bad arguments are refused before any
pointer is touched, and the record all-gather between gloo ranks leaves every
rank with every shard's records."""
import ctypes
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = torch.distributed


@pytest.fixture(scope="module")
def shard():
    from paper_2103_03348_b300 import build, shard
    build.build()
    return shard


@pytest.mark.parametrize("n", [2, 127, 128, 129, 1000, 23422, 100_000])
@pytest.mark.parametrize("k", [1, 2, 3, 7, 16])
def test_ranges_partition_events_and_records(shard, n, k):
    tiles = (n + 127) // 128
    assert shard.n_records(n) == tiles
    ev_end, rec_end = 0, 0
    for s in range(k):
        a, b, r0, r1 = shard.shard_range(n, s, k)
        assert a == ev_end and r0 == rec_end and a <= b and r0 <= r1
        assert a == min(r0 * 128, n) and b == min(r1 * 128, n)
        ev_end, rec_end = b, r1
    assert ev_end == n and rec_end == tiles
    sizes = [shard.shard_range(n, s, k)[3] - shard.shard_range(n, s, k)[2] for s in range(k)]
    assert max(sizes) - min(sizes) <= 1


def test_bad_arguments_are_refused(shard):
    from paper_2103_03348_b300 import hawkes
    L = shard._lib()
    z = ctypes.c_int64()
    assert L.hawkes_shard_range(100, 2, 2, ctypes.byref(z), None, None, None) == hawkes.EINVAL
    assert L.hawkes_shard_range(100, -1, 2, None, None, None, None) == hawkes.EINVAL
    assert L.hawkes_shard_range(1, 0, 1, None, None, None, None) == hawkes.EINVAL
    assert L.hawkes_shard_exchange_size(1) == 0
    pa = (ctypes.c_double * 6)(0.5, 0.1, 0.05, 0.3, 10.0, 0.02)
    fake = ctypes.c_void_p(1 << 20)
    big = ctypes.c_size_t(1 << 40)
    args = [fake, fake, fake, fake, 1000, pa, 1, 2]
    # shard index out of range, misaligned exchange buffer, exchange buffer too small
    assert L.hawkes_shard_rows(*args, 3, 2, fake, big, fake, big, fake, None) == hawkes.EINVAL
    assert L.hawkes_shard_rows(*args, 0, 2, fake, big, ctypes.c_void_p((1 << 20) + 8), big, fake,
                               None) == hawkes.EINVAL
    assert L.hawkes_shard_rows(*args, 0, 2, fake, big, fake, ctypes.c_size_t(64), fake, None) == hawkes.EWORKSPACE
    bad = (ctypes.c_double * 6)(0.5, -0.1, 0.05, 0.3, 10.0, 0.02)
    assert L.hawkes_shard_cols(fake, fake, fake, fake, 1000, bad, 1, 2, 0, 2, fake, big, fake, big, fake, fake,
                               fake, fake, None) == hawkes.EINVAL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _records(n, rank, world):
    """What rank `rank` would have after its row phase: its own records only."""
    from paper_2103_03348_b300 import shard
    t = shard.n_records(n)
    buf = torch.full((t, shard.RECORD_DOUBLES), float("nan"), dtype=torch.float64)
    _, _, r0, r1 = shard.shard_range(n, rank, world)
    for rec in range(r0, r1):
        buf[rec] = torch.arange(shard.RECORD_DOUBLES, dtype=torch.float64) + 1000.0 * rec
    return buf


def _worker(rank, world, port, n, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2103_03348_b300 import shard
        buf = shard.allgather_records(_records(n, rank, world), n, rank, world)
        out.put((rank, buf.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 1000), (3, 300)])
def test_record_allgather_between_gloo_ranks(world, n):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    t = (n + 127) // 128
    want = np.arange(144)[None, :] + 1000.0 * np.arange(t)[:, None]
    for r in range(world):
        np.testing.assert_array_equal(res[r], want)


def _fake_shard_cls():
    """A Shard whose row and column phases are host arithmetic instead of
    kernels: the row phase writes record j of its slice as (j + 1) * [1, 2, 3,
    ...]; the column phase needs every record (after the exchange) and writes
    loglik = sum of the records' first entries and, for each owned event e,
    grad[6 + e] = loglik + e and hdiag[6 + e] = -e.  So distributed_evaluate's
    composition (exchange, column phase, entry gather, status reduction) is
    checked on gloo ranks without a GPU."""
    from paper_2103_03348_b300 import shard

    class FakeShard(shard.Shard):
        def rows(self, x, y, t, r, params, mode="hess"):
            for j in range(self.rec0, self.rec1):
                self.xbuf[j] = (j + 1.0) * torch.arange(1, shard.RECORD_DOUBLES + 1, dtype=torch.float64)

        def cols(self, x, y, t, r, params, out, mode="hess"):
            assert not torch.isnan(self.xbuf).any()
            ll = float(self.xbuf[:, 0].sum())
            out["loglik"].fill_(ll)
            out["grad"][:6] = torch.arange(6, dtype=torch.float64)
            out["hdiag"][:6] = -torch.arange(6, dtype=torch.float64)
            e = torch.arange(self.first, self.end, dtype=torch.float64)
            out["grad"][6 + self.first:6 + self.end] = ll + e
            out["hdiag"][6 + self.first:6 + self.end] = -e

    return FakeShard


def _dist_worker(rank, world, port, n, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2103_03348_b300 import shard
        fake = _fake_shard_cls()(n, "fp32c", rank, world, device="cpu")
        fake.xbuf.fill_(float("nan"))  # only the own slice is written by the row phase
        z = torch.zeros(n, dtype=torch.float64)
        ll, g, h = shard.distributed_evaluate(z, z, z, z, (1, 1, 1, 1, 1, 1), "fp32c", "hess", shard=fake)
        out.put((rank, float(ll), g.numpy(), h.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 1000), (3, 300), (2, 100)])
def test_distributed_evaluate_composition_on_gloo_ranks(world, n):
    """Every rank ends with every rank's column entries, computed after the
    record exchange gave it every record (n = 100 with two ranks: one rank
    owns no events)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dist_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        rank, ll, g, h = q.get(timeout=120)
        res[rank] = (ll, g, h)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    t = (n + 127) // 128
    ll_want = float(sum(j + 1.0 for j in range(t)))
    e = np.arange(n, dtype=float)
    for r in range(world):
        ll, g, h = res[r]
        assert ll == ll_want
        np.testing.assert_array_equal(g, np.concatenate([np.arange(6.0), ll_want + e]))
        np.testing.assert_array_equal(h, np.concatenate([-np.arange(6.0), -e]))
