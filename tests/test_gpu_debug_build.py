"""The debug build (libgwx_debug.so, GWX_DEBUG=1; needs a GPU): index checks in the hot
kernels and guards after the binding's workspaces.  A small run of the whole pipeline
(background, Welch PSD, the fused batch, both likelihoods, importance weights) in a child
process with the debug library gives no recorded out-of-range access, leaves every guard
intact and the same numbers bit for bit as the normal build; a guard byte overwritten
outside the library is reported."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PIPELINE = r"""
import sys, numpy as np, torch
sys.path.insert(0, %r)
import workloads
import paper_2407_19048_gb300 as gwx
import paper_2407_19048_gb300.simulator
assert gwx._lib.load().gwx_debug_build() == (1 if gwx._lib.DEBUG else 0)
gwx.init()
wl = workloads.workload("small_nonspinning", B=40)
sim = gwx.simulator.Simulator(wl)
y, th, off = sim.step(3)
offs = torch.tensor([0, 7, 7, 30], dtype=torch.int64, device="cuda")
samp, _ = gwx.sample_prior(wl["prior"], 5, 1, 30, wl["L"], wl["N"])
lnl = gwx.log_likelihood(y[:3].contiguous(), sim.psd, wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0, samp, offs)
lnm = gwx.log_likelihood_tmarg(y[:3].contiguous(), sim.psd, wl["seg_len"], wl["fs"], wl["f_lo"], wl["dets"], 0.0,
                               *workloads.tc_grid(wl), samp, offs)
w, ess, eff, lnz = gwx.importance_weights(lnm, offs)
gwx.debug_check()
out = [y, sim.psd, lnl, lnm, w]
np.savez(sys.argv[1], *[t.detach().cpu().numpy() for t in out])
if gwx._lib.DEBUG:
    # overwrite one guard byte of a live workspace with a torch op: the check must see it
    ref, ptr, nbytes = gwx._guards[-1]
    ws = ref()
    ws[ptr - ws.data_ptr() + nbytes + 3] ^= 0xFF
    try:
        gwx.debug_check()
        print("GUARD_NOT_SEEN")
    except gwx.GwxError as e:
        print("GUARD_SEEN", e)
print("PIPELINE_OK")
"""


def _run(tmp_path, debug):
    out = str(tmp_path / ("debug.npz" if debug else "normal.npz"))
    env = dict(os.environ, GWX_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, "-c", PIPELINE % ROOT, out], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "PIPELINE_OK" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
    return np.load(out), r.stdout


def test_debug_build_runs_clean_and_matches_the_normal_build(tmp_path):
    from paper_2407_19048_gb300 import build
    build.build()
    build.build(debug=True)
    normal, _ = _run(tmp_path, False)
    debug, text = _run(tmp_path, True)
    assert "GUARD_SEEN" in text and "past the end" in text
    for k in normal.files:
        assert np.array_equal(normal[k], debug[k]), k
