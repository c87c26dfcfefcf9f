"""Differentiation through gridding and degridding (autograd.py).

The backward of gridding is degridding and vice versa.  Checked against
(a) the FP64 oracle's gradient of the same loss (oracle/chisq.py and the
oracle's grid/degrid), relative L2 <= 1e-5 on small cases and on the
sky's support (central quarter) of the 2048^2 image (FP32 FFTs of 2048^2
included), and
(b) central finite differences of the loss evaluated by the CUDA forward
(losses are quadratic, so the differences are exact up to FP32 rounding of
the forward pass).
"""
import json
import os

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.chisq import chisq_grad, predict
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


def report(name, **vals):
    print(name, json.dumps(vals))
    d = os.environ.get("GW_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "autograd.jsonl"), "a") as f:
            f.write(json.dumps({"case": name, **vals}) + "\n")


def small():
    return syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                          s_max=21, n_w=5, diameter_m=1500.0)


def sq64(t):
    return (torch.view_as_real(t).double() ** 2).sum()


def test_grid_backward_is_degridding(gw):
    """L(v) = |G v - T|^2: grad_v = 2 G^H (G v - T)."""
    from paper_2111_04141_gb300 import autograd as ag
    obs = small()
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    rng = np.random.default_rng(1)
    N = prm.grid_n
    T = (rng.normal(size=(prm.npol, N, N)) + 1j * rng.normal(size=(prm.npol, N, N))) * 0.1
    T = T.astype(np.complex64)
    with gw.Plan.from_observation(obs) as plan:
        u, f = dev(obs.uvw_m), dev(obs.freq_hz)
        v = dev(obs.vis).requires_grad_(True)
        loss = sq64(ag.grid(plan, u, f, v) - dev(T))
        loss.backward()
        got = v.grad.cpu().numpy().reshape(-1, prm.npol).astype(np.complex128)
        # finite differences of the CUDA forward on a few components
        fd_err = []
        for k in rng.choice(obs.vis.size, 6, replace=False):
            # the loss is quadratic: a unit step has no truncation error and
            # keeps the FP32 rounding of the loss small against the difference
            e = np.zeros(obs.vis.size, dtype=np.complex64)
            e[k] = 1.0
            e = dev(e.reshape(obs.vis.shape))
            with torch.no_grad():
                lp = float(sq64(ag.grid(plan, u, f, dev(obs.vis) + e) - dev(T)))
                lm = float(sq64(ag.grid(plan, u, f, dev(obs.vis) - e) - dev(T)))
            fd = (lp - lm) / 2.0
            fd_err.append(abs(fd - got.ravel()[k].real) / max(abs(got.ravel()[k].real), 1e-3))
    r = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis) - T.astype(np.complex128)
    want = 2 * orc.degrid(obs.uvw_m, obs.freq_hz, r)
    err = rel_l2(got, want)
    report("grad of |G v - T|^2", oracle_rel_l2=err, fd_max_rel=max(fd_err))
    assert err <= 1e-5
    assert max(fd_err) <= 1e-3


def test_degrid_backward_is_gridding(gw):
    """L(g) = |G^H g - d|^2: grad_g = 2 G (G^H g - d)."""
    from paper_2111_04141_gb300 import autograd as ag
    obs = small()
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    rng = np.random.default_rng(2)
    N = prm.grid_n
    g0 = (rng.normal(size=(prm.npol, N, N)) + 1j * rng.normal(size=(prm.npol, N, N)))
    g0 = (g0 * 0.01).astype(np.complex64)
    with gw.Plan.from_observation(obs) as plan:
        u, f = dev(obs.uvw_m), dev(obs.freq_hz)
        g = dev(g0).requires_grad_(True)
        loss = sq64(ag.degrid(plan, u, f, g) - dev(obs.vis))
        loss.backward()
        got = g.grad.cpu().numpy().astype(np.complex128)
    r = orc.degrid(obs.uvw_m, obs.freq_hz, g0.astype(np.complex128)) \
        - obs.vis.reshape(-1, prm.npol).astype(np.complex128)
    want = 2 * orc.grid(obs.uvw_m, obs.freq_hz, r)
    err = rel_l2(got, want)
    report("grad of |G^H g - d|^2", oracle_rel_l2=err)
    assert err <= 1e-5


def test_dirty_and_predict_are_adjoint(gw):
    from paper_2111_04141_gb300 import autograd as ag
    obs = small()
    rng = np.random.default_rng(3)
    N = obs.grid_n
    x = (rng.normal(size=(obs.npol, N, N)) + 1j * rng.normal(size=(obs.npol, N, N)))
    y = (rng.normal(size=obs.vis.shape) + 1j * rng.normal(size=obs.vis.shape))
    # the image lives on the central half, where the corrector is moderate
    c = slice(N // 4, 3 * N // 4)
    mask = np.zeros((N, N))
    mask[c, c] = 1
    with gw.Plan.from_observation(obs) as plan, torch.no_grad():
        u, f = dev(obs.uvw_m), dev(obs.freq_hz)
        px = ag.predict(plan, u, f, dev((x * mask).astype(np.complex64))).cpu().numpy()
        dy = ag.dirty(plan, u, f, dev(y.astype(np.complex64))).cpu().numpy()
    lhs = np.vdot(px.astype(np.complex128), y)
    rhs = np.vdot(x * mask, dy.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def sky_model(N, rng, n_points=200, n_blobs=12):
    """Point sources plus Gaussian blobs, all inside the central quarter
    (|l|, |m| < L/8).  With support 31 the taper's bandwidth is c = 48.7,
    so the corrector h = 1/taper reaches ~450 at |l| = L/4 and multiplies
    a model there before the FP32 FFT; inside L/8 it stays below ~5."""
    sky = np.zeros((N, N))
    lo, hi = 3 * N // 8 + 8, 5 * N // 8 - 8
    ii = rng.integers(lo, hi, n_points)
    jj = rng.integers(lo, hi, n_points)
    np.add.at(sky, (ii, jj), rng.uniform(0.1, 1.0, n_points))
    y, x = np.mgrid[0:N, 0:N]
    for _ in range(n_blobs):
        ci, cj = rng.integers(lo + 30, hi - 30, 2)
        s = rng.uniform(3.0, 12.0)
        sky += rng.uniform(0.02, 0.1) * np.exp(-((y - ci) ** 2 + (x - cj) ** 2) / (2 * s * s))
    c = np.zeros((N, N), dtype=bool)
    c[3 * N // 8:5 * N // 8, 3 * N // 8:5 * N // 8] = True
    sky[~c] = 0.0
    return sky[None].astype(np.float32)


def test_chisq_gradient_2048(gw):
    """2048^2 sky -> FFT -> degrid to 4.2M visibilities (128 antennas, 16
    w-planes, support 31) -> chi2 against noisy data (SNR ~ 10); the gradient
    by back-propagation (gridding) against the FP64 oracle gradient and
    against central differences at 32 random pixels."""
    from paper_2111_04141_gb300 import autograd as ag
    obs = syn.config_autograd()
    prm = Params(**obs.plan_kwargs())
    N = prm.grid_n
    rng = np.random.default_rng(4)
    sky = sky_model(N, rng)
    orc = Oracle(prm)
    h = corrector(prm)
    v_true = predict(orc, obs.uvw_m, obs.freq_hz, sky.astype(np.float64), h)
    sigma = float(np.sqrt(np.mean(np.abs(v_true) ** 2)) / 10.0)
    data = v_true + sigma * (rng.normal(size=v_true.shape) + 1j * rng.normal(size=v_true.shape))
    x0 = (0.7 * sky).astype(np.float32)
    want = chisq_grad(orc, obs.uvw_m, obs.freq_hz, x0.astype(np.float64), data, sigma, h)
    d_data = dev(data.reshape(obs.vis.shape).astype(np.complex64))
    with gw.Plan.from_observation(obs) as plan:
        u, f = dev(obs.uvw_m), dev(obs.freq_hz)
        x = dev(x0).requires_grad_(True)
        loss = ag.chisq(plan, u, f, x, d_data, sigma)
        loss.backward()
        got = x.grad.cpu().numpy().astype(np.float64)
        chi2 = float(loss.detach())
        # the gradient lives everywhere, but only where the taper is not tiny
        # is it resolved in FP32: in the band between L/8 and L/4 the
        # corrector (up to ~2e5 for h(l) h(m)) multiplies the FP32 inverse
        # FFT's absolute rounding.  Central quarter (the sky's support):
        # <= 1e-5; central half: <= 1e-3.
        q = slice(3 * N // 8, 5 * N // 8)
        err_q = rel_l2(got[:, q, q], want[:, q, q])
        c = slice(N // 4, 3 * N // 4)
        err = rel_l2(got[:, c, c], want[:, c, c])
        pix = np.stack([rng.integers(3 * N // 8, 5 * N // 8, 32),
                        rng.integers(3 * N // 8, 5 * N // 8, 32)], 1)
        gmax = np.abs(got[:, q, q]).max()
        fd_rel = []
        with torch.no_grad():
            for i, j in pix:
                eps = 1.0      # chi2 is quadratic: no truncation error at any step
                xp, xm = x.detach().clone(), x.detach().clone()
                xp[0, i, j] += eps
                xm[0, i, j] -= eps
                fd = (float(ag.chisq(plan, u, f, xp, d_data, sigma))
                      - float(ag.chisq(plan, u, f, xm, d_data, sigma))) / (2 * eps)
                fd_rel.append(abs(fd - got[0, i, j]) / (abs(got[0, i, j]) + 1e-4 * gmax))
    report("chi2 gradient autograd-2048-P16-S31",
           oracle_rel_l2_central_quarter=err_q, oracle_rel_l2_central_half=err,
           fd_max_rel=max(fd_rel), nvis=obs.nvis, sigma=sigma,
           chi2=chi2, chi2_per_vis=chi2 / obs.nvis)
    assert err_q <= 1e-5
    assert err <= 1e-3
    assert max(fd_rel) <= 1e-3
