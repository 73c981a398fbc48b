"""Sampler checkpoints on the CPU: the state written by save_state comes back
unchanged (tensors, random-stream states, draws), and the write is atomic
(a crash while writing leaves the previous checkpoint intact)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_state_round_trip(tmp_path):
    from paper_2103_03348_b300 import hmc
    gen = torch.Generator()
    gen.manual_seed(7)
    torch.randn(5, generator=gen)
    rng = np.random.default_rng(3)
    rng.uniform(size=4)
    state = {"it": 12, "q": torch.randn(9, dtype=torch.float64), "eps": 0.123, "gen_state": gen.get_state(),
             "rng_state": rng.bit_generator.state, "draws": np.arange(12.0).reshape(3, 4),
             "dual_averaging": {"mu": 0.5, "hbar": -0.1, "t": 4}}
    path = str(tmp_path / "ck.pt")
    hmc.save_state(path, state)
    back = hmc.load_state(path)
    assert back["it"] == 12 and back["eps"] == 0.123 and back["dual_averaging"] == state["dual_averaging"]
    assert torch.equal(back["q"], state["q"]) and np.array_equal(back["draws"], state["draws"])
    g2 = torch.Generator()
    g2.set_state(back["gen_state"])
    assert torch.equal(torch.randn(3, generator=g2), torch.randn(3, generator=gen))
    r2 = np.random.default_rng(0)
    r2.bit_generator.state = back["rng_state"]
    assert r2.uniform() == rng.uniform()


def test_atomic_write_keeps_previous_checkpoint(tmp_path, monkeypatch):
    from paper_2103_03348_b300 import hmc
    path = str(tmp_path / "ck.pt")
    hmc.save_state(path, {"it": 1})

    def broken(obj, f):
        with open(f, "wb") as fh:
            fh.write(b"partial")
        raise OSError("disk full")

    monkeypatch.setattr(hmc.torch, "save", broken)
    with pytest.raises(OSError):
        hmc.save_state(path, {"it": 2})
    monkeypatch.undo()
    assert hmc.load_state(path)["it"] == 1
    assert os.path.exists(path)
