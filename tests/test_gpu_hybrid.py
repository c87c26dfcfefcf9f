"""Hybrid Gridding on the GPU (gw_hybrid_*) against the oracle's Hybrid
Gridding step by step: fine grid and pruned grid relative L2 <= 1e-5, drop
counts exact, corrected image over the central half <= 2e-5."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle import hybrid as hy
from oracle.cgrid import Oracle
from oracle.wkernel import Params

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


# (8, 15), (8, 7), (16, 9): streaming pruner; (8, 17): shared-memory tiled pruner.
# Even npol: 16-byte atomics over polarisation pairs; odd npol: 8-byte ones.
@pytest.mark.parametrize("beta,sz,npol", [(8, 15, 2), (8, 7, 4), (16, 9, 1), (8, 17, 3)])
def test_hybrid_steps_match_oracle(gw, beta, sz, npol):
    obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=npol, grid_n=128, s_min=7, s_max=7,
                         n_w=1, diameter_m=1500.0, beta=beta)
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    wt = syn.random_weights(obs)
    fine_ref, keep = hy.fine_grid(prm, idx, obs.vis, sz, weight=wt)
    pruned_ref = hy.prune(prm, fine_ref, sz)
    img_ref = hy.image(prm, pruned_ref, sz)
    N = prm.grid_n
    with gw.Plan.from_observation(obs, max_vis_per_call=53 * obs.nchan) as plan:
        u, f = dev(obs.uvw_m), dev(obs.freq_hz)
        fine, dropped = plan.hybrid_grid(u, f, dev(obs.vis), sz, weight=dev(wt),
                                         return_dropped=True)
        pruned = plan.hybrid_prune(sz, fine)
        pr = pruned.cpu().numpy().astype(np.complex128)
        plan.hybrid_shift(pruned)
        raw = torch.fft.ifft2(pruned, norm="forward")
        img = plan.hybrid_image(sz, raw).cpu().numpy().astype(np.complex128)
        # [beta N, N, npol] (pols interleaved) -> the oracle's [npol, beta N, N]
        fine = np.moveaxis(fine.cpu().numpy().astype(np.complex128), 2, 0)
    assert dropped == int((~keep).sum())
    assert rel_l2(fine, fine_ref) <= 1e-5
    assert rel_l2(pr, pruned_ref) <= 1e-5
    c = slice(N // 4, 3 * N // 4)
    assert rel_l2(img[:, c, c], img_ref[:, c, c]) <= 2e-5


def test_hybrid_dirty_image_close_to_convolutional(gw):
    """Both gridders image the same sky; they differ by their different
    aliasing and nearest-neighbour errors (small in the central half)."""
    from paper_2111_04141_gb300.imaging import dirty_image, dirty_image_hybrid
    obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=1, grid_n=128, s_min=7, s_max=7,
                         n_w=1, diameter_m=1500.0, beta=64)
    with gw.Plan.from_observation(obs) as plan:
        u, f, v = dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)
        a = dirty_image(plan, u, f, v).cpu().numpy()
        b = dirty_image_hybrid(plan, u, f, v, 15).cpu().numpy()
    N = obs.grid_n
    c = slice(N // 4, 3 * N // 4)
    assert rel_l2(b[:, c, c], a[:, c, c]) <= 2e-3
