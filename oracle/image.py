"""Image-domain steps: centred inverse DFT, correction, brute-force NUDFTs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``centred_idft``: I[i, j] = sum_{kv, ku} G[kv, ku]
      exp(+j 2 pi ((ku - N/2)(j - N/2) + (kv - N/2)(i - N/2)) / N),
  the IFFT Step of Algorithm (convgridding) (Section 2.3) with the origin at
  pixel N/2 on both grids.  Computed with numpy's FFT (a library primitive)
  plus index shifts; ``centred_idft_direct`` is the same sum written out,
  used to pin the shifts on tiny grids.
* ``centred_dft``: the adjoint (sign -j), used on the degridding side.
* ``correct``: the Correction Step, image[pol, i, j] *= h(m_i) h(l_j).
* ``nudft_image``: Eq. (ID) of Section 1.7 without A-terms,
  I(l, m) = sum_p V_p exp(+j 2 pi (u_p l + v_p m + w_p (n - 1))),
  at the image pixels l_j = (j - N/2) * cell.  P = 1 (2-D mode) drops w.
* ``measurement``: Eq. (measurmentequation) of Section 1.2 for a pixelised
  model, V = sum_{i,j} I[i, j] exp(-j 2 pi (u l_j + v m_i + w (n_ij - 1))).
* ``point_source_vis``: the same for one unit point source at pixel
  (N/2 + dy, N/2 + dx), the simulator of the aliasing experiment of
  Section 8 (R(X) = |1 - K(X)|, K(X) the image value at the source).
"""
from __future__ import annotations

import numpy as np

from .wkernel import C0, Params


def centred_idft(grid: np.ndarray) -> np.ndarray:
    N = grid.shape[-1]
    ax = (-2, -1)
    return (N * N) * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(grid, axes=ax), axes=ax),
                                     axes=ax)


def centred_dft(image: np.ndarray) -> np.ndarray:
    ax = (-2, -1)
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(image, axes=ax), axes=ax), axes=ax)


def centred_idft_direct(grid: np.ndarray) -> np.ndarray:
    N = grid.shape[-1]
    k = np.arange(N) - N // 2
    F = np.exp(2j * np.pi * np.outer(k, k) / N)   # F[i, k] (symmetric)
    return np.einsum("ik,...kl,lj->...ij", F, grid, F)


def correct(image: np.ndarray, h: np.ndarray) -> np.ndarray:
    return image * (h[:, None] * h[None, :])


def _lmn(prm: Params):
    N = prm.grid_n
    l = (np.arange(N, dtype=np.float64) - N // 2) * prm.cell_rad
    L, M = np.meshgrid(l, l)          # L[i, j] = l_j, M[i, j] = m_i
    r2 = L * L + M * M
    n = np.sqrt(1.0 - r2)
    return L, M, -r2 / (1.0 + n)


def nudft_image(uvw_m, freq_hz, vis, prm: Params, weight=None) -> np.ndarray:
    """[npol, N, N] dirty image by direct summation (small inputs only)."""
    Lg, Mg, nm1 = _lmn(prm)
    nrow, nchan = uvw_m.shape[0], freq_hz.shape[0]
    v = np.asarray(vis, dtype=np.complex128).reshape(nrow * nchan, prm.npol)
    if weight is not None:
        v = v * np.asarray(weight, dtype=np.float64).reshape(nrow * nchan, prm.npol)
    lam = (uvw_m[:, None, :] * freq_hz[None, :, None] / C0).reshape(-1, 3)
    use_w = prm.n_wplanes > 1
    out = np.zeros((prm.npol, prm.grid_n, prm.grid_n), dtype=np.complex128)
    for r in range(lam.shape[0]):
        u, vv, w = lam[r]
        ph = u * Lg + vv * Mg + (w * nm1 if use_w else 0.0)
        e = np.exp(2j * np.pi * ph)
        for pol in range(prm.npol):
            out[pol] += v[r, pol] * e
    return out


def measurement(image: np.ndarray, uvw_m, freq_hz, prm: Params) -> np.ndarray:
    """[nrow * nchan, npol] visibilities of a pixelised model (small inputs only)."""
    Lg, Mg, nm1 = _lmn(prm)
    lam = (uvw_m[:, None, :] * freq_hz[None, :, None] / C0).reshape(-1, 3)
    use_w = prm.n_wplanes > 1
    out = np.zeros((lam.shape[0], prm.npol), dtype=np.complex128)
    for r in range(lam.shape[0]):
        u, vv, w = lam[r]
        ph = u * Lg + vv * Mg + (w * nm1 if use_w else 0.0)
        e = np.exp(-2j * np.pi * ph)
        for pol in range(prm.npol):
            out[r, pol] = np.sum(image[pol] * e)
    return out


def point_source_vis(uvw_m, freq_hz, prm: Params, dx: int, dy: int) -> np.ndarray:
    """[nrow * nchan, npol] visibilities (FP64) of a unit point source at
    pixel (row N/2 + dy, column N/2 + dx), all polarisations equal."""
    l = dx * prm.cell_rad
    m = dy * prm.cell_rad
    r2 = l * l + m * m
    nm1 = -r2 / (1.0 + np.sqrt(1.0 - r2))
    lam = (uvw_m[:, None, :] * freq_hz[None, :, None] / C0).reshape(-1, 3)
    ph = lam[:, 0] * l + lam[:, 1] * m + (lam[:, 2] * nm1 if prm.n_wplanes > 1 else 0.0)
    v = np.exp(-2j * np.pi * ph)
    return np.repeat(v[:, None], prm.npol, axis=1)
