"""Hybrid Gridding with a column pruner (Section 2.4, Algorithm (hybrid)).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For the 2-D (w-free) problem the thesis splits the two grid axes:

* Gridding Step: each record is convolved along u with the oversampled 1-D
  GCF C_co (support S, oversampling beta) and sampled on the integer u
  grid, while along v it is mapped to the nearest row of a v-axis grid
  oversampled by beta (Eq. (hybridgriddingstep)): an N (u) x beta N (v)
  "fine" grid.
* Pruning Step: each column is sampled down by beta/2 through a convolution
  with the pruning GCF Z (Eq. (hybridpruner)), onto a v-axis grid
  oversampled by 2: N x 2N.
* IFFT Step, then the Correction Step cuts out the central N rows and
  applies h_hy(l, m) = h_co(l) h_pr(m) (Eq. (hhy)), with
  h_pr = 1 / ([z(m/2) * Ш_{beta/2}] sinc_beta) (Eq. (hpr)).

Readings (the thesis' pruning GCF is a least-misfit function whose tables
are not available): Z is the zeroth-order PSWF with odd support S_z on the
2x grid, Z(x) = psi_0(pi S_z / 2, 2x / S_z), normalised so its taps at zero
offset sum to 1.  A fine row at q (units of 1/beta pixel) sits at 2q/beta on
the 2x grid: k0 = floor((2q + beta/2) / beta), offset o = 2q - k0 beta (even,
in [-beta/2, beta/2)), and contributes with Z(t - o/beta) to rows k0 + t,
|t| <= (S_z - 1)/2.  The realised transform of Z averages the beta/2
offsets: zhat(x) = (2/beta) sum_o sum_t Z(t - o/beta) cos(pi (t - o/beta) x),
x = (i - N/2)/N.  A record is kept when the convolutional gridder keeps it
(support S in u and v) and its pruning window lies inside the 2N rows.
"""
from __future__ import annotations

import numpy as np

from .pswf import PSWF0, taper_bandwidth
from .wkernel import Params, corrector, kernel_fine_1d


def kernel_u(prm: Params) -> np.ndarray:
    """c[o + beta/2, t + h]: the normalised 1-D GCF at t - o/beta."""
    beta = prm.oversample
    S = prm.support_min
    h = (S - 1) // 2
    f, C = kernel_fine_1d(prm, S, PSWF0(taper_bandwidth(prm.support_min)))
    C = np.real(C)
    norm = sum(C[beta * t - f[0]] for t in range(-h, h + 1))
    out = np.empty((beta, S))
    for a in range(beta):
        o = a - beta // 2
        out[a] = [C[beta * t - o - f[0]] / norm for t in range(-h, h + 1)]
    return out


def prune_table(beta: int, sz: int) -> np.ndarray:
    """Z[(o + beta/2)/2, t + hz] for even offsets o in [-beta/2, beta/2)."""
    hz = (sz - 1) // 2
    psi = PSWF0(np.pi * sz / 2.0)
    offs = np.arange(-beta // 2, beta // 2, 2)
    t = np.arange(-hz, hz + 1)
    x = (t[None, :] - offs[:, None] / beta) * (2.0 / sz)
    Z = psi(np.clip(x, -1.0, 1.0))
    return Z / np.sum(psi(t * (2.0 / sz)))


def prune_window(q, beta):
    """(k0, offset row of the Z table) of fine rows q."""
    q2 = 2 * np.asarray(q, dtype=np.int64)
    k0 = np.floor_divide(q2 + beta // 2, beta)
    o = q2 - k0 * beta
    return k0, (o + beta // 2) // 2


def fine_grid(prm: Params, idx: dict, vis, sz: int, weight=None):
    """(fine grid [npol, beta N, N] complex128, kept mask) of the Gridding Step."""
    beta, N, npol = prm.oversample, prm.grid_n, prm.npol
    S = prm.support_min
    h = (S - 1) // 2
    hz = (sz - 1) // 2
    c = kernel_u(prm)
    n = idx["ku"].shape[0]
    v = np.asarray(vis, dtype=np.complex128).reshape(n, npol)
    if weight is not None:
        v = v * np.asarray(weight, dtype=np.float64).reshape(n, npol)
    q = idx["kv"] * beta + idx["ov"]
    k0, _ = prune_window(q, beta)
    keep = idx["valid"] & (k0 - hz >= 0) & (k0 + hz <= 2 * N - 1)
    out = np.zeros((npol, beta * N, N), dtype=np.complex128)
    for i in np.nonzero(keep)[0]:
        w = c[idx["ou"][i] + beta // 2]
        cols = idx["ku"][i] + np.arange(-h, h + 1)
        for p in range(npol):
            out[p, q[i], cols] += w * v[i, p]
    return out, keep


def prune(prm: Params, fine: np.ndarray, sz: int) -> np.ndarray:
    """Pruning Step: [npol, beta N, N] -> [npol, 2N, N]."""
    beta, N = prm.oversample, prm.grid_n
    hz = (sz - 1) // 2
    Z = prune_table(beta, sz)
    P = np.zeros((2 * N, beta * N))
    q = np.arange(beta * N)
    k0, row = prune_window(q, beta)
    for t in range(-hz, hz + 1):
        k = k0 + t
        ok = (k >= 0) & (k < 2 * N)
        P[k[ok], q[ok]] += Z[row[ok], t + hz]
    return np.einsum("kr,prn->pkn", P, fine)


def corrector_pr(prm: Params, sz: int, nn_sinc: bool = True) -> np.ndarray:
    beta, N = prm.oversample, prm.grid_n
    hz = (sz - 1) // 2
    Z = prune_table(beta, sz)
    offs = np.arange(-beta // 2, beta // 2, 2)
    t = np.arange(-hz, hz + 1)
    d = (t[None, :] - offs[:, None] / beta).reshape(-1)
    x = (np.arange(N, dtype=np.float64) - N / 2) / N
    zhat = (np.cos(np.pi * d[None, :] * x[:, None]) @ Z.reshape(-1)) * (2.0 / beta)
    if not nn_sinc:
        return 1.0 / zhat
    a = np.pi * x / beta
    sinc = np.where(a == 0.0, 1.0, np.sin(a) / np.where(a == 0.0, 1.0, a))
    return 1.0 / (zhat * sinc)


def image(prm: Params, pruned: np.ndarray, sz: int, nn_sinc: bool = True) -> np.ndarray:
    """IFFT and Correction Steps: [npol, 2N, N] -> corrected [npol, N, N]."""
    N = prm.grid_n
    ax = (-2, -1)
    raw = (2 * N * N) * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(pruned, axes=ax),
                                                     axes=ax), axes=ax)
    raw = raw[:, N // 2:N // 2 + N, :]
    hu = corrector(prm, nn_sinc=nn_sinc)
    hv = corrector_pr(prm, sz, nn_sinc=nn_sinc)
    return raw * (hv[:, None] * hu[None, :])
