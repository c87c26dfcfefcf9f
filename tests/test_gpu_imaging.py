"""Imaging pipeline on the GPU (imaging.py): dirty image and model
visibilities against the oracle, and the aliasing experiment R(X) of
Section 8 for X = 0..63 on a 128^2 image against the oracle's R(X).

Tolerances: before correction the GPU image (FP32 gridding and cuFFT) and
the oracle's (FP64) agree at every pixel (X, X) to 2e-6 of the image peak:
FP32 rounding, the same at the field edge as at the centre.  The correction
multiplies that difference by h(l_X) h(m_X), so the corrected values R(X)
agree within 2e-6 peak h(l_X)^2 (peak: the uncorrected image at the centre,
about 1 / h(0)^2)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.image import centred_dft, centred_idft, correct, point_source_vis
from oracle.wkernel import Params, corrector

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


def test_rx_matches_oracle(gw):
    from paper_2111_04141_gb300.imaging import dirty_image
    N = 128
    obs = syn.config_2d()
    prm = Params(grid_n=N, cell_rad=syn.fit_cell(obs.uvw_m, obs.freq_hz, N, 7), support_min=7,
                 support_max=7, oversample=128, n_wplanes=1, w_max_lambda=0.0, npol=1)
    orc = Oracle(prm)
    h = corrector(prm)
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    nv = int(idx["valid"].sum())
    r_gpu, r_orc, raw_gpu, raw_orc = [], [], [], []
    with gw.Plan(grid_n=N, cell_rad=prm.cell_rad, support_min=7, support_max=7, oversample=128,
                 n_wplanes=1, w_max_lambda=0.0, npol=1) as plan:
        u, f = dev(obs.uvw_m), dev(obs.freq_hz)
        for x in range(64):
            v = point_source_vis(obs.uvw_m, obs.freq_hz, prm, x, x)
            vd = dev(v.reshape(obs.nrow, obs.nchan, 1).astype(np.complex64))
            img = dirty_image(plan, u, f, vd)
            r_gpu.append(abs(1.0 - float(img[0, N // 2 + x, N // 2 + x].real)))
            # the same transform without the correction step
            g = plan.grid(u, f, vd)
            plan.shift(g)
            raw = torch.fft.ifft2(g, norm="forward") / nv
            raw_gpu.append(complex(raw[0, N // 2 + x, N // 2 + x].item()))
            ref_raw = centred_idft(orc.grid(obs.uvw_m, obs.freq_hz, v, idx=idx)) / nv
            raw_orc.append(complex(ref_raw[0, N // 2 + x, N // 2 + x]))
            ref = correct(ref_raw, h)
            r_orc.append(abs(1.0 - ref[0, N // 2 + x, N // 2 + x].real))
    r_gpu, r_orc = np.array(r_gpu), np.array(r_orc)
    raw_gpu, raw_orc = np.array(raw_gpu), np.array(raw_orc)
    hx = h[N // 2 + np.arange(64)]
    peak = abs(raw_orc[0])
    print("R(X) gpu max central half %.3g, all %.3g; oracle %.3g, %.3g; raw max |diff| %.3g"
          " of the peak" % (r_gpu[:33].max(), r_gpu.max(), r_orc[:33].max(), r_orc.max(),
                             np.abs(raw_gpu - raw_orc).max() / peak))
    # the uncorrected transform agrees to FP32 rounding at every X, edge included
    assert np.all(np.abs(raw_gpu - raw_orc) <= 2e-6 * peak)
    # the corrected values differ by that, times the corrector
    assert np.all(np.abs(r_gpu - r_orc) <= 2e-6 * peak * hx ** 2 + 1e-7)


def test_dirty_image_and_model_vis_match_oracle(gw):
    from paper_2111_04141_gb300.imaging import dirty_image, model_vis
    obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                         s_max=21, n_w=5, diameter_m=1500.0)
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    h = corrector(prm)
    N = prm.grid_n
    wt = syn.random_weights(obs)
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    valid = idx["valid"]
    ref = correct(centred_idft(orc.grid(obs.uvw_m, obs.freq_hz, obs.vis, weight=wt)), h)
    ref = ref / wt.reshape(-1, prm.npol)[valid].sum(0)[:, None, None]
    rng = np.random.default_rng(2)
    model = np.zeros((prm.npol, N, N), dtype=np.complex64)
    c = slice(N // 4, 3 * N // 4)
    model[:, c, c] = (rng.normal(size=(prm.npol, N // 2, N // 2))).astype(np.complex64)
    ref_v = orc.degrid(obs.uvw_m, obs.freq_hz, centred_dft(correct(model.astype(np.complex128), h)))
    with gw.Plan.from_observation(obs) as plan:
        u, f = dev(obs.uvw_m), dev(obs.freq_hz)
        img = dirty_image(plan, u, f, dev(obs.vis), weight=dev(wt)).cpu().numpy()
        mv = model_vis(plan, u, f, dev(model)).cpu().numpy().reshape(ref_v.shape)
    assert rel_l2(img[:, c, c], ref[:, c, c]) <= 2e-5
    assert rel_l2(mv, ref_v) <= 2e-5
