"""The aliasing experiment of Section 8 (R(X) = |1 - K(X)|) on the oracle:
a unit point source at pixel (X, X) from the centre of a 128^2 image,
simulated by the measurement equation in FP64, gridded (PSWF support 7,
oversampling 128), inverse transformed and corrected; K(X) is the image at
the source normalised by the number of gridded visibilities.

Pins: the point-source simulator equals the pixelised measurement equation;
R(X) stays at the level of the PSWF's aliasing over the central half and
below 1e-3 up to the field edge."""
import numpy as np
import pytest

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.image import centred_idft, correct, measurement, point_source_vis
from oracle.wkernel import Params, corrector

N = 128


def rx_params(obs):
    return Params(grid_n=N, cell_rad=syn.fit_cell(obs.uvw_m, obs.freq_hz, N, 7), support_min=7,
                  support_max=7, oversample=128, n_wplanes=1, w_max_lambda=0.0, npol=1)


def oracle_rx(obs, prm, xs):
    orc = Oracle(prm)
    h = corrector(prm)
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    nv = int(idx["valid"].sum())
    out = []
    for x in xs:
        v = point_source_vis(obs.uvw_m, obs.freq_hz, prm, x, x)
        img = correct(centred_idft(orc.grid(obs.uvw_m, obs.freq_hz, v, idx=idx)), h) / nv
        out.append(abs(1.0 - img[0, N // 2 + x, N // 2 + x].real))
    return np.array(out)


def test_point_source_simulator_is_the_measurement_equation():
    obs = syn.config_2d()
    prm = rx_params(obs)
    for x in (0, 17, 50):
        img = np.zeros((1, N, N))
        img[0, N // 2 + x, N // 2 + x] = 1.0
        ref = measurement(img, obs.uvw_m[:200], obs.freq_hz, prm)
        got = point_source_vis(obs.uvw_m[:200], obs.freq_hz, prm, x, x)
        assert np.max(np.abs(got - ref)) <= 1e-12


def test_oracle_rx_profile():
    obs = syn.config_2d()
    prm = rx_params(obs)
    xs = np.arange(0, 64, 8)
    r = oracle_rx(obs, prm, xs)
    assert np.all(r[xs <= 32] <= 1e-6), r
    assert np.all(r <= 1e-3), r
