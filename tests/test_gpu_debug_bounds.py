"""The debug build (libgw_debug.so, GW_DEBUG_BOUNDS): its kernels check their
indices against their buffers, record a failed check in the plan's device
status word and skip the access.  On valid inputs no check may fire, and the
results must be those of the release build: gridding (binned and direct),
degridding (staged and gather) and the banded read-back, against the FP64
oracle.  Run in a child process, which loads the debug library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import synthetic as syn
from oracle.cgrid import Oracle
from oracle.wkernel import Params
import paper_2111_04141_gb300 as gw
from paper_2111_04141_gb300 import _lib
assert _lib.LIB_PATH.endswith("libgw_debug.so"), _lib.LIB_PATH
dev = torch.device("cuda", 0)
def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
for npol, smax in ((4, 21), (3, 13), (1, 31)):
    obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=npol, grid_n=128, s_min=7,
                         s_max=smax, n_w=5, diameter_m=1500.0)
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    ref = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis)
    rng = np.random.default_rng(5)
    g0 = (rng.normal(size=ref.shape) + 1j * rng.normal(size=ref.shape)).astype(np.complex64)
    vref = orc.degrid(obs.uvw_m, obs.freq_hz, g0.astype(np.complex128))
    uvw = torch.from_numpy(obs.uvw_m).to(dev)
    freq = torch.from_numpy(obs.freq_hz).to(dev)
    vis = torch.from_numpy(obs.vis).to(dev)
    with gw.Plan.from_observation(obs) as plan:
        for gk in (1, 2):
            plan.set_tuning(**dict(plan.get_tuning(), grid_kernel=gk))
            g = plan.grid(uvw, freq, vis).cpu().numpy().astype(np.complex128)
            plan.device_status()
            assert rel(g, ref) <= 1e-5, (npol, gk, rel(g, ref))
        for dk in (1, 2):
            plan.set_tuning(**dict(plan.get_tuning(), degrid_kernel=dk))
            v = plan.degrid(uvw, freq, torch.from_numpy(g0).to(dev)).cpu().numpy()
            plan.device_status()
            v = v.reshape(vref.shape).astype(np.complex128)
            assert rel(v, vref) <= 1e-5, (npol, dk, rel(v, vref))
        d_nrow = torch.tensor([obs.nrow], dtype=torch.int64, device=dev)
        out = plan.new_grid()
        host = torch.empty(out.shape, dtype=torch.complex64).pin_memory()
        plan.grid_devcount_readback(uvw, freq, d_nrow, vis, out, host, n_bands=3)
        plan.device_status()
        assert rel(host.numpy().astype(np.complex128), ref) <= 1e-5
print("debug-bounds ok")
"""


def test_debug_build_checks_fire_on_nothing_and_results_match():
    if not __import__("torch").cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build(debug=True)
    env = dict(os.environ, GW_DEBUG_BOUNDS="1")
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=900)
    assert out.returncode == 0, (out.stdout[-2000:], out.stderr[-4000:])
    assert "debug-bounds ok" in out.stdout
