"""W-stacking on the GPU (gw_grid_vis_wstack, gw_wstack_combine) against the
oracle's w-stacking: layer grids relative L2 <= 1e-5, and the corrected
w-stacked image over the central half <= 2e-5 (FP32 cuFFT included)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.image import nudft_image
from oracle.wkernel import C0, Params, corrector
from oracle.wstack import grid_layers, image_wstack

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def gw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build()
    import paper_2111_04141_gb300 as gw
    return gw


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case():
    obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=2, grid_n=128, s_min=9,
                         s_max=9, n_w=1, diameter_m=1500.0)
    wext = float(np.max(np.abs(obs.uvw_m[:, 2])) * obs.freq_hz.max() / C0)
    return obs, Params(**obs.plan_kwargs()), wext


@pytest.mark.parametrize("n_layers", [1, 7])
def test_layer_grids_match_oracle(gw, n_layers):
    obs, prm, wext = case()
    orc = Oracle(prm)
    wt = syn.random_weights(obs)
    ref = grid_layers(orc, obs.uvw_m, obs.freq_hz, obs.vis, n_layers, -wext, wext, weight=wt)
    with gw.Plan.from_observation(obs, max_vis_per_call=41 * obs.nchan) as plan:
        got, dropped = plan.grid_wstack(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis), n_layers,
                                        -wext, wext, weight=dev(wt), return_dropped=True)
    assert dropped == int((~orc.index(obs.uvw_m, obs.freq_hz)["valid"]).sum())
    assert rel_l2(got.cpu().numpy().astype(np.complex128), ref) <= 1e-5


def test_wstacked_image_matches_oracle(gw):
    from paper_2111_04141_gb300.imaging import dirty_image_wstack
    obs, prm, wext = case()
    orc = Oracle(prm)
    L = 9
    ref = image_wstack(orc, obs.uvw_m, obs.freq_hz, obs.vis, L, -wext, wext, corrector(prm))
    with gw.Plan.from_observation(obs) as plan:
        img = dirty_image_wstack(plan, dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis), L,
                                 -wext, wext, normalise=False).cpu().numpy()
    N = prm.grid_n
    c = slice(N // 4, 3 * N // 4)
    assert rel_l2(img[:, c, c].astype(np.complex128), ref[:, c, c]) <= 2e-5


# (3000, 17): w-screen phases beyond 100 rad and a screen recursion that
# crosses two re-anchoring layers
@pytest.mark.parametrize("w_max,L", [(300.0, 5), (3000.0, 17)])
def test_wstacked_image_matches_direct_sum_for_layer_exact_records(gw, w_max, L):
    from paper_2111_04141_gb300.imaging import dirty_image_wstack
    N = 64
    kw = dict(grid_n=N, cell_rad=0.3 / N, support_min=15, support_max=15, oversample=8,
              n_wplanes=1, w_max_lambda=0.0, npol=1)
    prm_w = Params(**{**kw, "n_wplanes": 2, "w_max_lambda": w_max})
    rng = np.random.default_rng(6)
    n, span = 20, 32 - 15 // 2 - 2
    field = 0.3
    fu = rng.integers(-span * 8, span * 8, n) / 8
    fv = rng.integers(-span * 8, span * 8, n) / 8
    w = -w_max + (2 * w_max / (L - 1)) * rng.integers(0, L, n)
    uvw = np.stack([fu / field, fv / field, w], 1)
    vis = (rng.normal(size=(n, 1, 1)) + 1j * rng.normal(size=(n, 1, 1))).astype(np.complex64)
    ref = nudft_image(uvw, np.array([C0]), vis, prm_w)
    with gw.Plan(**kw) as plan:
        img = dirty_image_wstack(plan, dev(uvw), dev(np.array([C0])), dev(vis), L, -w_max, w_max,
                                 normalise=False).cpu().numpy()
        # the GPU corrector includes the nearest-neighbour sinc factor; these
        # records sit on the beta-grid, so compare against the sinc-free one
        h_nn = plan.corrector()
    h0 = corrector(Params(**kw), nn_sinc=False)
    img = img * (h0[:, None] * h0[None, :]) / (h_nn[:, None] * h_nn[None, :])
    c = slice(N // 4, 3 * N // 4)
    err = np.max(np.abs(img[:, c, c] - ref[:, c, c])) / np.max(np.abs(ref[:, c, c]))
    assert err <= 2e-5
