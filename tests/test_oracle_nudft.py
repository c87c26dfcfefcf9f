"""End-to-end pins: oracle gridding + IFFT + correction against the
brute-force non-uniform DFT of Eq. (ID) (Section 1.7), and oracle
degridding against the measurement equation (Section 1.2)."""
import numpy as np
import pytest

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.image import centred_dft, centred_idft, correct, measurement, nudft_image
from oracle.wkernel import C0, Params, corrector, plane_w


def exact_positions(prm, n, rng, span=10):
    """Records on the beta-fine grid (no nearest-neighbour shift)."""
    beta = prm.oversample
    fu = rng.integers(-span * beta, span * beta, n) / beta
    fv = rng.integers(-span * beta, span * beta, n) / beta
    return fu, fv


def plane_exact_w(prm, n, rng):
    """w values exactly on the planes (W-projection quantises w to the
    nearest plane; records off the planes carry that quantisation error)."""
    if prm.n_wplanes == 1:
        return np.zeros(n)
    return rng.choice(plane_w(prm), n) * rng.choice([-1.0, 1.0], n)


def central(a, N):
    c = slice(N // 4, 3 * N // 4)
    return a[..., c, c]


@pytest.mark.parametrize("smin,smax,P,wmax,tol", [
    (15, 15, 1, 0.0, 1e-7),      # 2-D: only the PSWF truncation remains
    (15, 47, 2, 200.0, 1e-7),    # w-projection with a support that holds the chirp
    (15, 31, 3, 50.0, 1e-7),
])
def test_image_matches_direct_sum_exact_positions(smin, smax, P, wmax, tol):
    N = 64
    prm = Params(grid_n=N, cell_rad=0.3 / N, support_min=smin, support_max=smax, oversample=8,
                 n_wplanes=P, w_max_lambda=wmax, npol=1)
    orc = Oracle(prm)
    rng = np.random.default_rng(4)
    n = 20
    fu, fv = exact_positions(prm, n, rng, span=32 - smax // 2 - 2)
    w = plane_exact_w(prm, n, rng)
    uvw = np.stack([fu / prm.field, fv / prm.field, w], 1)
    vis = (rng.normal(size=(n, 1, 1)) + 1j * rng.normal(size=(n, 1, 1))).astype(np.complex64)
    assert orc.index(uvw, np.array([C0]))["valid"].all()
    g = orc.grid(uvw, np.array([C0]), vis)
    img = correct(centred_idft(g), corrector(prm, nn_sinc=False))
    ref = nudft_image(uvw, np.array([C0]), vis, prm)
    err = np.max(np.abs(central(img - ref, N))) / np.max(np.abs(ref))
    assert err <= tol


def test_image_random_positions_error_shrinks_with_beta():
    """Off-grid records pay the nearest-neighbour shift of up to 1/(2 beta)
    pixel (Section 2.3.6); the error falls roughly as 1/beta."""
    errs = []
    for beta in (8, 64, 512):
        obs = syn.small_case(n_ant=6, n_times=4, n_chan=2, npol=1, grid_n=64, s_min=15,
                             s_max=15, n_w=1, diameter_m=500.0, beta=beta)
        prm = Params(**obs.plan_kwargs())
        orc = Oracle(prm)
        g = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis)
        img = correct(centred_idft(g), corrector(prm))
        ref = nudft_image(obs.uvw_m, obs.freq_hz, obs.vis, prm)
        errs.append(np.sqrt(np.mean(np.abs(central(img - ref, 64)) ** 2))
                    / np.sqrt(np.mean(np.abs(ref) ** 2)))
    assert errs[0] < 0.05
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4
    assert errs[2] < 2e-3


@pytest.mark.parametrize("P,wmax", [(1, 0.0), (2, 200.0)])
def test_degrid_matches_measurement_equation(P, wmax):
    """Degridding is the adjoint of gridding; for a model inside the central
    half it reproduces the measurement equation."""
    N = 64
    prm = Params(grid_n=N, cell_rad=0.3 / N, support_min=15, support_max=47 if P > 1 else 15,
                 oversample=8, n_wplanes=P, w_max_lambda=wmax, npol=2)
    orc = Oracle(prm)
    rng = np.random.default_rng(8)
    model = np.zeros((2, N, N), dtype=np.complex128)
    for _ in range(6):
        i, j = rng.integers(N // 4 + 2, 3 * N // 4 - 2, 2)
        model[:, i, j] += rng.normal(size=2)
    n = 25
    fu, fv = exact_positions(prm, n, rng, span=32 - prm.support_max // 2 - 2)
    w = plane_exact_w(prm, n, rng)
    uvw = np.stack([fu / prm.field, fv / prm.field, w], 1)
    assert orc.index(uvw, np.array([C0]))["valid"].all()
    grid = centred_dft(correct(model, corrector(prm, nn_sinc=False)))
    v = orc.degrid(uvw, np.array([C0]), grid)
    ref = measurement(model, uvw, np.array([C0]), prm)
    assert np.max(np.abs(v - ref)) <= 1e-7 * np.max(np.abs(ref))
