"""Imaging pipeline around the gridder: dirty images and model visibilities.

The imaging chain of Section 2.3 (Algorithm (convgridding)): gridding, the
inverse FFT of the grid and the correction step, giving the dirty image
(Eq. (ID) of Section 1.7 up to the approximation of the method); and its
adjoint, model image -> visibilities.  Gridding, degridding, the origin
shift and the correction run in libgw's kernels; the FFTs are cuFFT calls
through torch.fft (unnormalised, so the two operators are exact adjoints).

The dirty image is normalised by the sum of the weights of the visibilities
that were gridded (dropped records excluded), so a unit point source
observed by every visibility images to 1 at its pixel.
"""
from __future__ import annotations

from typing import Optional

import torch


def dirty_image(plan, uvw, freq, vis, weight: Optional[torch.Tensor] = None,
                normalise: bool = True, stream=None) -> torch.Tensor:
    """[npol, N, N] complex64 dirty image (the real part is the image)."""
    g, dropped = plan.grid(uvw, freq, vis, weight=weight, stream=stream, return_dropped=True)
    plan.shift(g, stream=stream)
    img = torch.fft.ifft2(g, norm="forward")          # sum_k G_k exp(+j 2 pi k x / N)
    plan.correct(img, direction=+1, stream=stream)
    if normalise:
        nrow, nchan = uvw.shape[0], freq.shape[0]
        if weight is None:
            wsum = float(nrow * nchan - dropped)
        else:
            # drops are visibilities whose footprint leaves the grid: their
            # weights are excluded through the index records' valid flags
            raw, _ = plan.index(uvw, freq, stream=stream)
            valid = ((raw[:, 3] >> 16) & 1).to(torch.float32)
            w = weight.reshape(nrow * nchan, -1) * valid[:, None]
            ws = w.sum(0).to(torch.float64).clamp_min(1e-30)     # per polarisation
            img /= ws.to(img.real.dtype)[:, None, None]
            return img
        img /= max(wsum, 1e-30)
    return img


def model_vis(plan, uvw, freq, image: torch.Tensor, stream=None) -> torch.Tensor:
    """Visibilities [nrow, nchan, npol] of a [npol, N, N] model image: the
    adjoint of the unnormalised dirty image (correct, FFT, shift, degrid)."""
    x = image.to(torch.complex64).contiguous().clone()
    plan.correct(x, direction=-1, stream=stream)
    g = torch.fft.fft2(x, norm="backward").contiguous()  # sum_x I_x exp(-j 2 pi k x / N)
    plan.shift(g, stream=stream)
    return plan.degrid(uvw, freq, g, stream=stream)


def dirty_image_wstack(plan, uvw, freq, vis, n_layers: int, w_min: float, w_max: float,
                       normalise: bool = True, stream=None) -> torch.Tensor:
    """Dirty image by w-stacking (Section 1.7.1): a 2-D plan grids every
    visibility onto the grid of its w-layer; each layer grid is inverse
    transformed, re-centred, multiplied by its w-screen
    exp(+j 2 pi w_l (n - 1)) and summed (gw_wstack_combine, which also does
    the re-centring); the sum is corrected once."""
    layers, dropped = plan.grid_wstack(uvw, freq, vis, n_layers, w_min, w_max, stream=stream,
                                       return_dropped=True)
    imgs = torch.fft.ifft2(layers, norm="forward")
    del layers
    img = plan.new_grid()
    plan.wstack_combine(imgs, w_min, w_max, img, stream=stream)
    plan.correct(img, direction=+1, stream=stream)
    if normalise:
        img /= max(float(uvw.shape[0] * freq.shape[0] - dropped), 1e-30)
    return img


def dirty_image_hybrid(plan, uvw, freq, vis, sz: int = 15, normalise: bool = True,
                       stream=None) -> torch.Tensor:
    """Dirty image by Hybrid Gridding (Section 2.4, Algorithm (hybrid)) with a
    2-D plan: Gridding Step onto beta N v-rows, column pruning to 2N rows,
    inverse FFT of the 2N x N grid, central N rows corrected."""
    fine, dropped = plan.hybrid_grid(uvw, freq, vis, sz, stream=stream, return_dropped=True)
    pruned = plan.hybrid_prune(sz, fine, stream=stream)
    del fine
    plan.hybrid_shift(pruned, stream=stream)
    raw = torch.fft.ifft2(pruned, norm="forward")
    img = plan.hybrid_image(sz, raw, stream=stream)
    if normalise:
        img /= max(float(uvw.shape[0] * freq.shape[0] - dropped), 1e-30)
    return img
