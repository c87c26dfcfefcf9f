"""W-projection kernel tables and the grid corrector, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

W-projection (Section 1.7.1, after Eq. (v00) of Section 1.3) projects each
record onto the w = 0 plane by convolving it with Gbar_w, the Fourier
transform of gbar_w(l, m) = exp(+j 2 pi w (sqrt(1 - l^2 - m^2) - 1))
(Eq. (gw) and its inverse), merged into the gridding convolution function.
The anti-aliasing taper is the prolate spheroidal psi_0 (Section 2.3.4), and
the merged function is stored beta-oversampled and looked up by nearest
neighbour (Section 2.3.6).

Readings (the thesis is silent on these):

* planes uniform in sqrt|w|: w_p = w_max (p / (P - 1))^2, p = 0 .. P-1;
* support of plane p: the odd integer nearest
  y_p = S_min + (S_max - S_min) p / (P - 1)   (= sqrt(w_p / w_max)),
  ties upward, i.e. S_p = 2 floor(y_p / 2) + 1;
* taper T(t) = psi_0(c, t), c = pi S_min / 2, on the normalised field
  coordinate t = 2 l / L in [-1, 1], L = N * cell (field of view);
* kernel of plane p at uv offset (du, dv) pixels:
      K_p(du, dv) = int int_{[-1,1]^2} T(t_l) T(t_m)
                     exp(+j 2 pi w_p (n - 1)) exp(-j pi (du t_l + dv t_m)) dt_l dt_m,
      n = sqrt(1 - (L/2)^2 (t_l^2 + t_m^2)),
  the continuous Fourier transform of taper x w-screen over the field of
  view, evaluated with Gauss-Legendre quadrature (Q_p nodes per axis, from
  the phase-rate rule in ``quad_nodes``);
* oversampled table: offsets o in [-beta/2, beta/2), taps t in [-h, h],
  h = (S_p - 1) / 2, entry (o_v, o_u, t_v, t_u) = K_p(t_u - o_u/beta,
  t_v - o_v/beta) times one global scale chosen so that the w = 0 plane's
  o = 0 slice sums to 1 over its taps; no renormalisation after truncation;
* records with w < 0 use conj(K_p) (the screen is even in l and m, so
  K_{-w} = conj(K_w));
* corrector: h(l) = 1 / (chat(l) * sinc_beta(l)), with
  chat(l) = (1/beta) sum_o sum_t C(t - o/beta) cos(2 pi (t - o/beta) l),
  C the normalised one-dimensional w = 0 kernel and l the pixel position in
  units of the field of view, (i - N/2) / N.  This is Eq. (hco) of
  Section 2.4.5 with [c * Sha_beta] replaced by the transform actually
  realised by the truncated, oversampled table; without truncation it
  equals Eq. (hco).

Pins: w = 0 plane against the PSWF self-Fourier closed form; quadrature
convergence; symmetries (tests/test_oracle_kernels.py); the brute-force
NUDFT pins in tests/test_oracle_nudft.py exercise the whole chain.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import roots_legendre

from .pswf import PSWF0, taper_bandwidth

C0 = 299_792_458.0


@dataclasses.dataclass(frozen=True)
class Params:
    grid_n: int
    cell_rad: float
    support_min: int
    support_max: int
    oversample: int
    n_wplanes: int
    w_max_lambda: float
    npol: int = 1

    @property
    def field(self) -> float:
        """L = N * cell, the field of view in direction-cosine units."""
        return float(self.grid_n) * float(self.cell_rad)


def params_from(obs_or_kwargs) -> Params:
    if isinstance(obs_or_kwargs, dict):
        return Params(**obs_or_kwargs)
    return Params(**obs_or_kwargs.plan_kwargs())


def plane_w(prm: Params) -> np.ndarray:
    P = prm.n_wplanes
    if P == 1:
        return np.zeros(1)
    p = np.arange(P, dtype=np.float64)
    return prm.w_max_lambda * (p / (P - 1)) ** 2


def plane_support(prm: Params) -> np.ndarray:
    P = prm.n_wplanes
    if P == 1:
        return np.array([prm.support_min], dtype=np.int64)
    out = []
    for p in range(P):
        # y * (P - 1) is an integer; S = 2 floor(y / 2) + 1
        Y = prm.support_min * (P - 1) + (prm.support_max - prm.support_min) * p
        out.append(2 * (Y // (2 * (P - 1))) + 1)
    return np.array(out, dtype=np.int64)


def quad_nodes(prm: Params, w: float, support: int) -> int:
    """Gauss-Legendre node count per axis for one plane.

    kappa bounds the phase rate of the integrand on t in [-1, 1]: the
    w-screen contributes 2 pi |w| (L/2)^2 / n_min, the Fourier kernel
    pi (h + 1/2) and the taper's own band c.
    """
    half = 0.5 * prm.field
    n_min = math.sqrt(1.0 - 2.0 * half * half)
    h = (support - 1) // 2
    c = taper_bandwidth(prm.support_min)
    kappa = 2.0 * math.pi * abs(w) * half * half / n_min + math.pi * (h + 0.5) + c
    return int(math.ceil(0.75 * kappa)) + 40


def fine_offsets(beta: int, support: int) -> np.ndarray:
    """All f = beta * t - o for t in [-h, h], o in [-beta/2, beta/2), ascending."""
    h = (support - 1) // 2
    return np.arange(-beta * h - beta // 2 + 1, beta * h + beta // 2 + 1, dtype=np.int64)


def kernel_fine(prm: Params, w: float, support: int, taper: PSWF0, n_nodes: int | None = None):
    """K(f_v / beta, f_u / beta) for all fine offsets f of one plane, unscaled.

    Returns (f, Kf) with Kf[i_v, i_u] for f[i_v], f[i_u].
    """
    beta = prm.oversample
    Q = quad_nodes(prm, w, support) if n_nodes is None else int(n_nodes)
    t, wt = roots_legendre(Q)
    half = 0.5 * prm.field
    Tw = wt * taper(t)
    # image-domain integrand A[j (m axis), i (l axis)]
    r2 = (half * half) * (t[:, None] ** 2 + t[None, :] ** 2)
    n = np.sqrt(1.0 - r2)
    n_minus_1 = -r2 / (1.0 + n)
    A = (Tw[:, None] * Tw[None, :]) * np.exp(2j * np.pi * w * n_minus_1)
    f = fine_offsets(beta, support)
    E = np.exp(-1j * np.pi * (f[:, None].astype(np.float64) / beta) * t[None, :])
    Kf = E @ A @ E.T
    return f, Kf


def kernel_fine_1d(prm: Params, support: int, taper: PSWF0, n_nodes: int | None = None):
    """One-dimensional w = 0 kernel C(f / beta) on the fine offsets of ``support``."""
    beta = prm.oversample
    Q = quad_nodes(prm, 0.0, support) if n_nodes is None else int(n_nodes)
    t, wt = roots_legendre(Q)
    f = fine_offsets(beta, support)
    E = np.exp(-1j * np.pi * (f[:, None].astype(np.float64) / beta) * t[None, :])
    return f, E @ (wt * taper(t))


class KernelTables:
    """The oversampled W-kernel table of every plane, FP64 complex.

    ``planes[p]`` has shape [beta, beta, S_p, S_p] and is indexed
    [o_v + beta/2, o_u + beta/2, t_v + h, t_u + h].
    """

    def __init__(self, prm: Params, n_nodes: int | None = None):
        self.prm = prm
        self.beta = prm.oversample
        self.w = plane_w(prm)
        self.support = plane_support(prm)
        self.taper = PSWF0(taper_bandwidth(prm.support_min))
        fines = []
        for p in range(prm.n_wplanes):
            f, Kf = kernel_fine(prm, float(self.w[p]), int(self.support[p]), self.taper, n_nodes)
            fines.append((f, Kf))
        # global scale: w = 0 plane, o = 0 slice sums to 1
        f0, K0 = fines[0]
        h0 = (int(self.support[0]) - 1) // 2
        idx = np.array([self.beta * t - f0[0] for t in range(-h0, h0 + 1)])
        s = np.sum(K0[np.ix_(idx, idx)])
        self.scale = 1.0 / float(np.real(s))
        self.planes = [self._slice_table(f, Kf * self.scale, int(self.support[p]))
                       for p, (f, Kf) in enumerate(fines)]

    def _slice_table(self, f, Kf, support):
        beta = self.beta
        h = (support - 1) // 2
        tab = np.empty((beta, beta, support, support), dtype=np.complex128)
        t = np.arange(-h, h + 1)
        for a in range(beta):
            ov = a - beta // 2
            iv = beta * t - ov - f[0]
            for b in range(beta):
                ou = b - beta // 2
                iu = beta * t - ou - f[0]
                tab[a, b] = Kf[np.ix_(iv, iu)]
        return tab

    def flat(self):
        """(concatenated table, per-plane offsets in complex elements)."""
        offs = np.zeros(len(self.planes) + 1, dtype=np.int64)
        for p, tab in enumerate(self.planes):
            offs[p + 1] = offs[p] + tab.size
        return np.concatenate([t.ravel() for t in self.planes]), offs


def corrector(prm: Params, n_nodes: int | None = None, nn_sinc: bool = True) -> np.ndarray:
    """h(l_i) for image pixels i = 0 .. N-1 (l_i = (i - N/2) / N).

    ``nn_sinc=False`` leaves out the sinc_beta factor, which compensates the
    average amplitude loss of nearest-neighbour offsets; records that sit
    exactly on the beta-fine grid suffer no such loss.
    """
    beta = prm.oversample
    S = int(plane_support(prm)[0])
    taper = PSWF0(taper_bandwidth(prm.support_min))
    f, C = kernel_fine_1d(prm, S, taper, n_nodes)
    h = (S - 1) // 2
    idx = np.array([beta * t - f[0] for t in range(-h, h + 1)])
    Cn = np.real(C) / np.sum(np.real(C[idx]))
    N = prm.grid_n
    l = (np.arange(N, dtype=np.float64) - N / 2) / N
    chat = np.cos(2.0 * np.pi * (f[None, :].astype(np.float64) / beta) * l[:, None]) @ Cn / beta
    if not nn_sinc:
        return 1.0 / chat
    x = np.pi * l / beta
    sinc = np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
    return 1.0 / (chat * sinc)
