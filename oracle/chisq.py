"""Chi-squared of a sky model against visibilities, and its gradient (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The thesis' imaging chain (Section 2.3, Algorithm (convgridding): gridding,
inverse FFT, correction) maps visibilities to a dirty image; its adjoint
maps a pixelised model image to visibilities, the discretised form of the
measurement equation (Section 1.2, Eq. (measurmentequation)):

  predict(x) = Degrid( centred_dft( h(m) h(l) x ) )       (model -> vis)
  dirty(r)   = h(m) h(l) centred_idft( Grid(r) )          (vis -> image)

with Grid / Degrid the oracle's w-projection gridding and its adjoint
(Section 2.4.5) and h the corrector.  dirty is exactly the adjoint of
predict (centred_idft is the adjoint of centred_dft and the correction is
real and diagonal).  For a real sky x and data d with noise sigma,

  chi2(x) = sum |predict(x) - d|^2 / sigma^2,
  grad chi2(x) = 2 Re( dirty(predict(x) - d) ) / sigma^2,

the gradient a differentiable imager gets by back-propagating through
degridding with gridding.  chi2 is quadratic, so central finite differences
reproduce the gradient exactly up to rounding (the pin used in
tests/test_oracle_chisq.py).
"""
from __future__ import annotations

import numpy as np

from .image import centred_dft, centred_idft, correct


def predict(orc, uvw_m, freq_hz, image, h) -> np.ndarray:
    """[nrow * nchan, npol] model visibilities of a [npol, N, N] image."""
    x = np.asarray(image, dtype=np.complex128)
    return orc.degrid(uvw_m, freq_hz, centred_dft(correct(x, h)))


def dirty(orc, uvw_m, freq_hz, vis, h) -> np.ndarray:
    """[npol, N, N] dirty image (adjoint of ``predict``) of visibilities."""
    g = orc.grid(uvw_m, freq_hz, np.asarray(vis, dtype=np.complex128))
    return correct(centred_idft(g), h)


def chisq(orc, uvw_m, freq_hz, sky, data, sigma, h) -> float:
    r = predict(orc, uvw_m, freq_hz, sky, h) - np.asarray(data).reshape(-1, sky.shape[0])
    return float(np.sum(np.abs(r) ** 2) / sigma ** 2)


def chisq_grad(orc, uvw_m, freq_hz, sky, data, sigma, h) -> np.ndarray:
    """Gradient of ``chisq`` with respect to a real sky [npol, N, N]."""
    r = predict(orc, uvw_m, freq_hz, sky, h) - np.asarray(data).reshape(-1, sky.shape[0])
    return 2.0 * np.real(dirty(orc, uvw_m, freq_hz, r, h)) / sigma ** 2
