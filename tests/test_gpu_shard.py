"""The sharded evaluation (row shards, record exchange, column shards; run in
sequence on one GPU with a workspace per shard) equals the unsharded call bit
for bit, in every precision and mode, including shards that own no events."""
import numpy as np
import pytest

from paper_2103_03348_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.tensor(np.asarray(a, float), dtype=torch.float64, device="cuda")


def unsharded(x, y, t, r, params, precision, mode):
    from paper_2103_03348_b300 import hawkes
    if mode == "hess":
        return hawkes.hess_diag(x, y, t, r, params, precision)
    if mode == "grad":
        ll, g = hawkes.grad(x, y, t, r, params, precision)
        return ll, g, None
    return hawkes.loglik(x, y, t, r, params, precision), None, None


def same(a, b):
    if a is None or b is None:
        return a is None and b is None
    return torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "fp32c", "fp32c_band"])
@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_sharded_hess_is_bitwise_unsharded(precision, k):
    from paper_2103_03348_b300 import build, shard
    build.build()
    w = synth.make("ebola_like")
    x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
    a = unsharded(x, y, t, r, w.params, precision, "hess")
    b = shard.evaluate(x, y, t, r, w.params, precision, n_shards=k, mode="hess")
    assert same(a[0], b[0]) and same(a[1], b[1]) and same(a[2], b[2])
    assert torch.isfinite(b[2]).all()


@pytest.mark.parametrize("mode", ["loglik", "grad"])
@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_sharded_other_modes(precision, mode):
    from paper_2103_03348_b300 import build, shard
    build.build()
    w = synth.make_uniform(8, 1000, r_sd=0.4)
    x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
    a = unsharded(x, y, t, r, w.params, precision, mode)
    b = shard.evaluate(x, y, t, r, w.params, precision, n_shards=3, mode=mode)
    assert same(a[0], b[0]) and same(a[1], b[1])


def test_more_shards_than_tiles_and_identical_globals():
    """Ragged 300 events (3 tiles) over 5 shards: two shards own nothing; every
    shard reports the same loglik and global entries."""
    from paper_2103_03348_b300 import build, shard
    build.build()
    w = synth.make_uniform(4, 300, r_sd=0.5)
    x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
    n, k = w.n, 5
    shards = [shard.Shard(n, "fp32c", s, k) for s in range(k)]
    assert sum(sh.end - sh.first for sh in shards) == n
    assert sum(1 for sh in shards if sh.end == sh.first) == 2
    for sh in shards:
        sh.rows(x, y, t, r, w.params)
    shard.exchange_local(shards)
    outs = []
    for sh in shards:
        out = {"loglik": torch.empty((), dtype=torch.float64, device="cuda"),
               "grad": torch.zeros(6 + n, dtype=torch.float64, device="cuda"),
               "hdiag": torch.zeros(6 + n, dtype=torch.float64, device="cuda")}
        sh.cols(x, y, t, r, w.params, out)
        outs.append(out)
    for o in outs[1:]:
        assert torch.equal(o["loglik"], outs[0]["loglik"])
        assert torch.equal(o["grad"][:6], outs[0]["grad"][:6])
        assert torch.equal(o["hdiag"][:6], outs[0]["hdiag"][:6])
    a = unsharded(x, y, t, r, w.params, "fp32c", "hess")
    b = shard.evaluate(x, y, t, r, w.params, "fp32c", n_shards=k)
    assert same(a[0], b[0]) and same(a[1], b[1]) and same(a[2], b[2])


def test_status_of_one_shard_reaches_all():
    """An event far from every other has zero intensity; it sits in shard 1's
    rows, and after the exchange every shard reports it."""
    from paper_2103_03348_b300 import build, hawkes, shard
    build.build()
    w = synth.make_uniform(6, 600, box=50.0, t_max=30.0, r_sd=0.3, params=(0.8, 6.0, 4.0, 0.6, 0.5, 3.0))
    xs = w.x.copy()
    xs[450] = 1.0e7  # tile 3 of 5: shard 1 of 2 owns tiles [2, 5)
    x, y, t, r = dev(xs), dev(w.y), dev(w.t), dev(w.r)
    shards = [shard.Shard(w.n, "fp64", s, 2) for s in range(2)]
    assert shards[1].first <= 450 < shards[1].end
    for sh in shards:
        sh.rows(x, y, t, r, w.params)
    shard.exchange_local(shards)
    for sh in shards:
        out = {"loglik": torch.empty((), dtype=torch.float64, device="cuda"),
               "grad": torch.zeros(6 + w.n, dtype=torch.float64, device="cuda"),
               "hdiag": torch.zeros(6 + w.n, dtype=torch.float64, device="cuda")}
        sh.cols(x, y, t, r, w.params, out)
        assert int(sh.status.item()) == hawkes.EZERO


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_worker(rank, world, port, name, precision, q):
    """One rank on cuda:0: distributed_evaluate over gloo (records and entries
    staged through host memory) against the unsharded call on the same GPU."""
    import os
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    try:
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        from paper_2103_03348_b300 import shard
        w = synth.make(name) if name != "ragged" else synth.make_uniform(5, 1001, r_sd=0.4)
        x, y, t, r = dev(w.x), dev(w.y), dev(w.t), dev(w.r)
        ll, g, h = shard.distributed_evaluate(x, y, t, r, w.params, precision, "hess")
        a = unsharded(x, y, t, r, w.params, precision, "hess")
        ok = torch.equal(ll, a[0]) and torch.equal(g, a[1]) and torch.equal(h, a[2])
        q.put((rank, ok, ""))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, False, repr(e)))


@pytest.mark.parametrize("name,precision,world", [("ebola_like", "fp32c", 2), ("ebola_like", "fp64", 2),
                                                  ("ragged", "fp32c_band", 3)])
def test_distributed_ranks_are_bitwise_unsharded(name, precision, world):
    """The cross-rank evaluation (each rank's row phase, the record all-gather,
    each rank's column phase, the entry all-gather) run by `world` processes on
    this GPU over gloo equals hawkes_hess_diag bit for bit on every rank.  The
    ranks' kernels never wait on one another: the exchange is host-side."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, world, port, name, precision, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
    assert all(ok for _, ok, _ in res), res
    assert all(p.exitcode == 0 for p in procs)
