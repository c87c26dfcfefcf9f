"""The allocation-free degridding entry point (gw_degrid_vis_static) gives
the same visibilities as gw_degrid_vis, on two calls in a row, through the
C ABI.  It is meant for callers that cannot allocate device memory while
running; its scratch is a fixed array inside the library, which every call
reuses, so the second call must not be disturbed by the first one's leftovers.
Kept in a file of its own that pytest collects last."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
TOL = 1e-5   # the relative-L2 tolerance of the FP32 degridding parity tests


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_degrid_matches_degrid_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build()
    import paper_2111_04141_gb300 as gw
    cases = [syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                            s_max=21, n_w=5, diameter_m=1500.0),
             syn.small_case(n_ant=6, n_times=12, n_chan=2, npol=2, grid_n=96, s_min=5,
                            s_max=13, n_w=3, diameter_m=900.0, beta=4, seed=4)]
    rng = np.random.default_rng(12)
    for obs in cases:
        N = obs.grid_n
        with gw.Plan.from_observation(obs) as plan:
            uvw = torch.from_numpy(obs.uvw_m).to(DEV)
            freq = torch.from_numpy(obs.freq_hz).to(DEV)
            for call in range(2):
                g = (rng.normal(size=(obs.npol, N, N))
                     + 1j * rng.normal(size=(obs.npol, N, N))).astype(np.complex64)
                grid = torch.from_numpy(g).to(DEV)
                ref, dref = plan.degrid(uvw, freq, grid, return_dropped=True)
                out = torch.full_like(ref, 7.0 + 7.0j)     # caller-owned output, dirty
                got, dgot = plan.degrid_static(uvw, freq, grid, out=out, return_dropped=True)
                assert dgot == dref
                assert rel(got.cpu().numpy(), ref.cpu().numpy()) <= TOL, (obs.name, call)


def test_static_degrid_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2111_04141_gb300 as gw
    obs = syn.small_case(n_ant=4, n_times=4, n_chan=1, npol=1, grid_n=64, s_min=7, s_max=7,
                         n_w=1, diameter_m=500.0)
    with gw.Plan.from_observation(obs) as plan:
        n = 65536 + 1
        uvw = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
        freq = torch.from_numpy(obs.freq_hz).to(DEV)
        grid = plan.new_grid()
        with pytest.raises(gw.GwError, match="static scratch limit"):
            plan.degrid_static(uvw, freq, grid)


_FRESH = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import torch
import synthetic as syn
import paper_2111_04141_gb300 as gw
from paper_2111_04141_gb300 import plan as P
dev = torch.device("cuda", 0)
obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7, s_max=21,
                     n_w=5, diameter_m=1500.0)
with torch.cuda.device(dev):
    plan = gw.Plan.from_observation(obs)            # allocating is still allowed here
    uvw = torch.from_numpy(obs.uvw_m).to(dev)
    freq = torch.from_numpy(obs.freq_hz).to(dev)
    grid = torch.ones((obs.npol, obs.grid_n, obs.grid_n), dtype=torch.complex64, device=dev)
    out = plan.new_vis(obs.nrow, obs.nchan)
    torch.cuda.synchronize(dev)
    f0, b0 = torch.cuda.mem_get_info(dev)[0], P.live_bytes()
    plan.degrid_static(uvw, freq, grid, out=out)     # the first call in this process
    torch.cuda.synchronize(dev)
    f1, b1 = torch.cuda.mem_get_info(dev)[0], P.live_bytes()
    plan.degrid_static(uvw, freq, grid, out=out)
    torch.cuda.synchronize(dev)
    f2 = torch.cuda.mem_get_info(dev)[0]
    print(json.dumps({"free": [f0, f1, f2], "live_bytes": [b0, b1]}))
    plan.close()
"""


def test_static_degrid_first_call_allocates_nothing():
    """In a fresh process, the first allocation-free call finds everything it
    needs already loaded by plan creation: free device memory and the
    library's own allocations are the same before and after it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    f0, f1, f2 = res["free"]
    assert f1 == f0 and f2 == f0, res
    assert res["live_bytes"][0] == res["live_bytes"][1], res
