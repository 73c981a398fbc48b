"""The usage example in README.md runs as written."""
import os
import re

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_python_example_runs():
    from paper_2103_03348_b300 import build
    build.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks
    env = {}
    exec(compile(blocks[0], "README.md", "exec"), env)
    assert torch.isfinite(env["ll"]).item()
    assert torch.equal(env["ll"], env["ll4"]) and torch.equal(env["hdiag"], env["hdiag4"])
    assert env["chain"].draws.shape[0] == 500
    assert int(env["sims"]["status"].max()) == 0
