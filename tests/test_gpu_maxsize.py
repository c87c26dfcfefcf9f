"""The largest grid the plan accepts (N = 32768, the gw_plan_desc limit) with
4 polarisations: 4 x 2^30 complex values, so grid offsets pass 2^31 and
every offset computation must be 64-bit.  A small observation spread over
the whole grid (several w-planes, supports 7-15) is gridded by the binned and
the direct gridder and compared with the FP64 oracle on a lattice of grid
points; the degridders are checked through the adjoint identity
<G, grid(V)> = <degrid(G), V>, which holds at any size, with G drawn on the
device."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.wkernel import Params

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
N_MAX = 32768


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build()
    import paper_2111_04141_gb300 as gw
    obs = syn.small_case(n_ant=8, n_times=8, n_chan=2, npol=4, grid_n=N_MAX, s_min=7, s_max=15,
                         n_w=3, diameter_m=100e3, seed=41)
    orc = Oracle(Params(**obs.plan_kwargs()))
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    yield gw, obs, orc, t(obs.uvw_m), t(obs.freq_hz), t(obs.vis)
    torch.cuda.empty_cache()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kernel", [1, 2], ids=["binned", "direct"])
def test_max_grid_lattice_matches_oracle(setup, kernel):
    gw, obs, orc, uvw, freq, vis = setup
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    off, step = 3, 13
    m = (N_MAX - off + step - 1) // step
    ref = orc.grid_lattice(obs.uvw_m, obs.freq_hz, obs.vis, off, step, m, idx=idx)
    assert np.count_nonzero(ref) > 500
    with gw.Plan.from_observation(obs) as plan:
        plan.set_tuning(grid_kernel=kernel)
        g, dropped = plan.grid(uvw, freq, vis, return_dropped=True)
        assert dropped == int((~idx["valid"]).sum())
        pts = torch.arange(off, N_MAX, step, device=DEV)
        got = g[:, pts][:, :, pts].cpu().numpy().astype(np.complex128)
        del g
    torch.cuda.empty_cache()
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("kernel", [1, 2], ids=["staged", "gather"])
def test_max_grid_degrid_is_the_adjoint(setup, kernel):
    gw, obs, orc, uvw, freq, vis = setup
    gen = torch.Generator(device=DEV).manual_seed(43)
    with gw.Plan.from_observation(obs) as plan:
        plan.set_tuning(degrid_kernel=kernel, grid_kernel=1)
        G = torch.randn((obs.npol, N_MAX, N_MAX), dtype=torch.complex64, device=DEV,
                        generator=gen)
        g = plan.grid(uvw, freq, vis)
        # <G, grid(V)> per polarisation plane (each below 2^31 elements)
        lhs = sum(complex(torch.vdot(G[p].reshape(-1), g[p].reshape(-1)).item())
                  for p in range(obs.npol))
        del g
        d = plan.degrid(uvw, freq, G).cpu().numpy().astype(np.complex128)
        del G
    torch.cuda.empty_cache()
    rhs = complex(np.vdot(d.reshape(-1), obs.vis.astype(np.complex128).reshape(-1)))
    assert abs(lhs - rhs) <= 1e-5 * abs(rhs)
    # and the degridded values themselves on the records the oracle keeps
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    assert np.all(d.reshape(-1, obs.npol)[~idx["valid"]] == 0)
