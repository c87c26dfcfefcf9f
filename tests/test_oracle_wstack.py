"""Pins of the oracle's w-stacking (oracle/wstack.py): hand-worked layer
choices (nearest layer, ties up, clamping) and the w-stacked image against
the direct sum of Eq. (ID) with the w-term for records on the beta-grid
whose w lies on a layer (only the PSWF truncation error remains)."""
import numpy as np

from oracle.cgrid import Oracle
from oracle.image import nudft_image
from oracle.wkernel import C0, Params, corrector
from oracle.wstack import image_wstack, layer_of


def test_layer_choice():
    # 5 layers over [-100, 100]: w_l = -100, -50, 0, 50, 100
    w = np.array([-100.0, -75.0, -74.9, -0.1, 24.9, 25.0, 100.0, 130.0, -1e9, 49.99])
    uvw = np.stack([np.zeros_like(w), np.zeros_like(w), w], 1)
    got = layer_of(uvw, np.array([C0]), 5, -100.0, 100.0)
    assert list(got) == [0, 1, 1, 2, 2, 3, 4, 4, 0, 3]


def test_wstack_image_matches_direct_sum():
    N = 64
    w_max = 300.0
    L = 5
    # a 2-D plan: the kernel is the w = 0 PSWF table
    prm = Params(grid_n=N, cell_rad=0.3 / N, support_min=15, support_max=15, oversample=8,
                 n_wplanes=1, w_max_lambda=0.0, npol=1)
    prm_w = Params(grid_n=N, cell_rad=0.3 / N, support_min=15, support_max=15, oversample=8,
                   n_wplanes=2, w_max_lambda=w_max, npol=1)
    orc = Oracle(prm)
    rng = np.random.default_rng(6)
    n = 20
    span = 32 - 15 // 2 - 2
    fu = rng.integers(-span * 8, span * 8, n) / 8
    fv = rng.integers(-span * 8, span * 8, n) / 8
    w = -w_max + (2 * w_max / (L - 1)) * rng.integers(0, L, n)       # on the layers
    uvw = np.stack([fu / prm.field, fv / prm.field, w], 1)
    vis = (rng.normal(size=(n, 1, 1)) + 1j * rng.normal(size=(n, 1, 1))).astype(np.complex64)
    freq = np.array([C0])
    assert orc.index(uvw, freq)["valid"].all()
    img = image_wstack(orc, uvw, freq, vis, L, -w_max, w_max, corrector(prm, nn_sinc=False))
    ref = nudft_image(uvw, freq, vis, prm_w)          # Eq. (ID) with the w-term
    c = slice(N // 4, 3 * N // 4)
    err = np.max(np.abs(img[:, c, c] - ref[:, c, c])) / np.max(np.abs(ref[:, c, c]))
    assert err <= 1e-7
