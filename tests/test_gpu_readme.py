"""The README's Python examples run as written (needs a GPU), with the training loop cut
to a few steps: they use the public binding, so an API change that leaves them stale
fails here."""
import pathlib
import re

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = pathlib.Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def gwx():
    import paper_2407_19048_gb300 as m
    from paper_2407_19048_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    m.init()
    return m


def _blocks():
    text = (ROOT / "README.md").read_text()
    return re.findall(r"```python\n(.*?)```", text, flags=re.S)


def test_readme_examples_run(gwx):
    blocks = _blocks()
    assert len(blocks) >= 2
    code = "\n".join(blocks)
    assert "range(6000)" in code
    code = code.replace("range(6000)", "range(3)")
    ns = {}
    exec(compile(code, "README.md", "exec"), ns)
    torch.cuda.synchronize()
    lnl, theta_s, ess = ns["lnl"], ns["theta_s"], ns["ess"]
    assert theta_s.shape == (11, 20000) and lnl.shape == (20000,)
    assert np.isfinite(lnl.cpu().numpy()).mean() > 0.99
    assert float(ess.cpu()[0]) >= 1.0
    assert gwx._lib.load().gwx_device_status() == 0
