"""The usage example of the README runs as written (on the GPU), and its
outputs are consistent: sorted pairs, a finite loss, a gradient of the image's
shape that is nonzero only at birth and death pixels."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "no Python example in the README"
    ns = {}
    exec(compile(blocks[0], "README.md", "exec"), ns)
    d, x, loss, grad = ns["d"], ns["x"], ns["loss"], ns["grad"]
    p = d.numpy()
    assert len(p) > 0 and (p["dim"][:-1] <= p["dim"][1:]).all()
    assert torch.isfinite(loss).all() and torch.isfinite(ns["birth"]).all()
    g = x.grad
    assert g.shape == x.shape and torch.isfinite(g).all()
    touched = set(p["birth_pixel"].tolist()) | set(p["death_pixel"].tolist())
    nz = set(torch.nonzero(g.flatten()).flatten().tolist())
    assert nz <= touched
    assert grad.numel() == 512 * 384 + 64 * 80 * 96
