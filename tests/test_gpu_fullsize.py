"""Full-size parity: the 4-pol W-projection workload (8.26M visibilities,
4096^2 x 4 grid, 32 w-planes, support 7->63, oversampling 8) through the
same Plan.grid / Plan.degrid calls the benchmark times, checked against the
FP64 oracle on sampled outputs: a lattice of grid points spanning the whole
grid, and a random subset of degridded visibilities.  Tolerance: relative
L2 <= 1e-5."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.wkernel import Params

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build()
    import paper_2111_04141_gb300 as gw
    obs = syn.config_wproj()
    orc = Oracle(Params(**obs.plan_kwargs()))
    plan = gw.Plan.from_observation(obs)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    yield obs, orc, plan, t(obs.uvw_m), t(obs.freq_hz), t(obs.vis)
    plan.close()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_fullsize_grid_lattice(setup):
    obs, orc, plan, uvw, freq, vis = setup
    g, dropped = plan.grid(uvw, freq, vis, return_dropped=True)
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    assert dropped == int((~idx["valid"]).sum())
    for off, step in ((5, 31), (1000, 17)):
        m = (obs.grid_n - off + step - 1) // step
        ref = orc.grid_lattice(obs.uvw_m, obs.freq_hz, obs.vis, off, step, m, idx=idx)
        pts = torch.arange(off, obs.grid_n, step, device=DEV)
        got = g[:, pts][:, :, pts].cpu().numpy().astype(np.complex128)
        assert np.count_nonzero(ref) > 1000
        assert rel(got, ref) <= 1e-5


def test_fullsize_degrid_sample(setup):
    obs, orc, plan, uvw, freq, vis = setup
    rng = np.random.default_rng(1)
    N = obs.grid_n
    grid = (rng.standard_normal((obs.npol, N, N), dtype=np.float32)
            + 1j * rng.standard_normal((obs.npol, N, N), dtype=np.float32)).astype(np.complex64)
    out = plan.degrid(uvw, freq, torch.from_numpy(grid).to(DEV)).cpu().numpy()
    rows = np.sort(rng.choice(obs.nrow, 3000, replace=False))
    ref = orc.degrid(obs.uvw_m[rows], obs.freq_hz, grid)
    got = out[rows].reshape(ref.shape).astype(np.complex128)
    assert rel(got, ref) <= 1e-5
