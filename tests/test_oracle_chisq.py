"""Pins of the oracle's chi-squared and its gradient (oracle/chisq.py).

* predict reproduces the measurement equation (Section 1.2) for records on
  the beta-fine grid and a model inside the central half (only the PSWF
  truncation error remains);
* dirty is the adjoint of predict (dot test);
* chi2 is quadratic, so central finite differences of chi2 equal the
  gradient formula up to rounding.
"""
import numpy as np

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.chisq import chisq, chisq_grad, dirty, predict
from oracle.image import measurement
from oracle.wkernel import C0, Params, corrector, plane_w


def test_predict_is_the_measurement_equation():
    N = 64
    prm = Params(grid_n=N, cell_rad=0.3 / N, support_min=15, support_max=31, oversample=8,
                 n_wplanes=3, w_max_lambda=50.0, npol=1)
    orc = Oracle(prm)
    rng = np.random.default_rng(12)
    sky = np.zeros((1, N, N))
    for _ in range(5):
        i, j = rng.integers(N // 4 + 2, 3 * N // 4 - 2, 2)
        sky[0, i, j] += rng.uniform(0.5, 2.0)
    n, beta, span = 30, prm.oversample, 32 - 31 // 2 - 2
    fu = rng.integers(-span * beta, span * beta, n) / beta
    fv = rng.integers(-span * beta, span * beta, n) / beta
    w = rng.choice(plane_w(prm), n) * rng.choice([-1.0, 1.0], n)
    uvw = np.stack([fu / prm.field, fv / prm.field, w], 1)
    freq = np.array([C0])
    v = predict(orc, uvw, freq, sky, corrector(prm, nn_sinc=False))
    ref = measurement(sky, uvw, freq, prm)
    assert np.max(np.abs(v - ref)) <= 1e-7 * np.max(np.abs(ref))


def _case():
    obs = syn.small_case(n_ant=6, n_times=8, n_chan=2, npol=1, grid_n=64, s_min=7, s_max=15,
                         n_w=4, diameter_m=800.0)
    prm = Params(**obs.plan_kwargs())
    return obs, prm, Oracle(prm), corrector(prm)


def test_dirty_is_the_adjoint_of_predict():
    obs, prm, orc, h = _case()
    rng = np.random.default_rng(1)
    N = prm.grid_n
    x = rng.normal(size=(1, N, N)) + 1j * rng.normal(size=(1, N, N))
    y = rng.normal(size=(obs.nvis, 1)) + 1j * rng.normal(size=(obs.nvis, 1))
    lhs = np.vdot(predict(orc, obs.uvw_m, obs.freq_hz, x, h), y)
    rhs = np.vdot(x, dirty(orc, obs.uvw_m, obs.freq_hz, y, h))
    # h spans ~1e7 across the field, so the sums lose a few digits
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_gradient_matches_central_differences():
    obs, prm, orc, h = _case()
    rng = np.random.default_rng(2)
    N = prm.grid_n
    sky = np.zeros((1, N, N))
    for _ in range(6):
        i, j = rng.integers(N // 4, 3 * N // 4, 2)
        sky[0, i, j] += rng.uniform(0.5, 2.0)
    sigma = 0.1
    data = predict(orc, obs.uvw_m, obs.freq_hz, sky, h)
    data = data + sigma * (rng.normal(size=data.shape) + 1j * rng.normal(size=data.shape))
    x0 = 0.7 * sky
    g = chisq_grad(orc, obs.uvw_m, obs.freq_hz, x0, data, sigma, h)
    for i, j in [(N // 2, N // 2), (20, 40), (30, 33), (45, 19)]:
        eps = 1e-2
        xp, xm = x0.copy(), x0.copy()
        xp[0, i, j] += eps
        xm[0, i, j] -= eps
        fd = (chisq(orc, obs.uvw_m, obs.freq_hz, xp, data, sigma, h)
              - chisq(orc, obs.uvw_m, obs.freq_hz, xm, data, sigma, h)) / (2 * eps)
        assert abs(fd - g[0, i, j]) <= 1e-9 * abs(g[0, i, j])
