"""W-stacking (Section 1.7.1, "Correction of the W-term in the (l,m)-plane").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Visibilities with similar w are gridded with the 2-D (w = 0) kernel onto
the grid of their w-layer; each layer's image (the centred inverse DFT of
its grid) is multiplied by the layer's w-screen ḡ_w(l, m) =
exp(+j 2 pi w_l (n - 1)) (Eq. (lmwcorr)) and the layer images are summed;
the corrector is applied once to the sum.

Reading: layers w_l = w_min + l dw, dw = (w_max - w_min)/(L - 1); a
visibility belongs to the nearest layer, ties up, clamped to [0, L - 1]:
l = clamp(floor((w_lambda - w_min)/dw + 1/2), 0, L - 1), in FP64 with the
operation order of the index stage (w_lambda = w (f/c0)).
"""
from __future__ import annotations

import numpy as np

from .image import _lmn, centred_idft, correct
from .index import chan_scale


def layer_of(uvw_m, freq_hz, n_layers: int, w_min: float, w_max: float) -> np.ndarray:
    """Layer of every visibility, (row, channel) order."""
    wl = uvw_m[:, 2][:, None] * chan_scale(freq_hz)[None, :]
    if n_layers <= 1:
        return np.zeros(wl.size, dtype=np.int64)
    dw = (w_max - w_min) / (n_layers - 1)
    t = np.floor((wl - w_min) / dw + 0.5)
    return np.clip(t, 0, n_layers - 1).astype(np.int64).reshape(-1)


def grid_layers(orc2d, uvw_m, freq_hz, vis, n_layers, w_min, w_max, weight=None):
    """[L, npol, N, N] complex128 layer grids (orc2d: an Oracle of a 2-D plan)."""
    prm = orc2d.prm
    idx = orc2d.index(uvw_m, freq_hz)
    lay = layer_of(uvw_m, freq_hz, n_layers, w_min, w_max)
    out = np.zeros((n_layers, prm.npol, prm.grid_n, prm.grid_n), dtype=np.complex128)
    for l in range(n_layers):
        sel = dict(idx)
        keep = idx["valid"] & (lay == l)
        sel["valid"] = keep
        sel["flags"] = np.where(keep, idx["flags"], 0)
        orc2d.grid(uvw_m, freq_hz, vis, weight=weight, grid=out[l], idx=sel)
    return out


def image_wstack(orc2d, uvw_m, freq_hz, vis, n_layers, w_min, w_max, h, weight=None):
    """[npol, N, N] corrected (unnormalised) w-stacked dirty image."""
    prm = orc2d.prm
    layers = grid_layers(orc2d, uvw_m, freq_hz, vis, n_layers, w_min, w_max, weight)
    _, _, nm1 = _lmn(prm)
    dw = (w_max - w_min) / (n_layers - 1) if n_layers > 1 else 0.0
    img = np.zeros((prm.npol, prm.grid_n, prm.grid_n), dtype=np.complex128)
    for l in range(n_layers):
        screen = np.exp(2j * np.pi * (w_min + l * dw) * nm1)
        img += centred_idft(layers[l]) * screen[None]
    return correct(img, h)
