"""Pins for the oracle's w-kernel tables and corrector (oracle/wkernel.py)."""
import numpy as np
import pytest

from oracle.pswf import PSWF0, taper_bandwidth
from oracle.wkernel import (KernelTables, Params, fine_offsets, kernel_fine, plane_support,
                            plane_w, quad_nodes)


def prm_w(**kw):
    d = dict(grid_n=128, cell_rad=0.4 / 128, support_min=7, support_max=15, oversample=8,
             n_wplanes=4, w_max_lambda=300.0, npol=1)
    d.update(kw)
    return Params(**d)


@pytest.mark.parametrize("smin,beta", [(7, 8), (9, 4), (15, 16)])
def test_w0_plane_is_self_fourier_pswf(smin, beta):
    """At w = 0 the kernel is the Fourier transform of the truncated PSWF,
    which by the PSWF's self-Fourier property is lambda_0 psi_0(2 du / S)
    psi_0(2 dv / S): a closed form independent of the quadrature."""
    prm = prm_w(support_min=smin, support_max=smin + 8, oversample=beta)
    kt = KernelTables(prm)
    p0 = PSWF0(taper_bandwidth(smin))
    S = int(kt.support[0])
    h = (S - 1) // 2
    t = np.arange(-h, h + 1)
    norm = np.sum(p0(2.0 * t / S)) ** 2
    err = 0.0
    for a in range(beta):
        o = a - beta // 2
        d = t - o / beta
        ref1 = p0(2.0 * d / S)
        for b in range(beta):
            ob = b - beta // 2
            ref = np.outer(ref1, p0(2.0 * (t - ob / beta) / S)) / norm
            err = max(err, np.max(np.abs(kt.planes[0][a, b] - ref)))
    assert err <= 1e-10


def test_quadrature_converged():
    prm = prm_w()
    kt = KernelTables(prm)
    q = 2 * max(quad_nodes(prm, w, int(s)) for w, s in zip(kt.w, kt.support))
    kt2 = KernelTables(prm, n_nodes=q)
    for a, b in zip(kt.planes, kt2.planes):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_kernel_symmetries():
    """The screen and taper are even in l and in m and symmetric under l <-> m,
    so K(du, dv) = K(-du, dv) = K(du, -dv) = K(dv, du)."""
    prm = prm_w()
    p0 = PSWF0(taper_bandwidth(7))
    f, K = kernel_fine(prm, 300.0, 15, p0)
    n = f.shape[0] - 1            # f[:-1] is symmetric about 0
    assert f[0] == -f[-2]
    Ks = K[:-1, :-1]
    assert np.max(np.abs(Ks - Ks[::-1, :])) <= 1e-13 * np.max(np.abs(K))
    assert np.max(np.abs(Ks - Ks[:, ::-1])) <= 1e-13 * np.max(np.abs(K))
    assert np.max(np.abs(K - K.T)) <= 1e-13 * np.max(np.abs(K))
    assert n > 0


def test_normalisation_and_w0_real():
    prm = prm_w()
    kt = KernelTables(prm)
    beta = prm.oversample
    assert abs(np.sum(kt.planes[0][beta // 2, beta // 2]) - 1.0) <= 1e-13
    assert np.max(np.abs(kt.planes[0].imag)) <= 1e-15
    # non-zero w makes the kernel complex
    assert np.max(np.abs(kt.planes[-1].imag)) > 1e-3


def test_plane_rules_hand_values():
    prm = Params(grid_n=4096, cell_rad=1e-4, support_min=7, support_max=63, oversample=8,
                 n_wplanes=32, w_max_lambda=31.0 ** 2, npol=4)
    S = plane_support(prm)
    assert [S[0], S[1], S[15], S[16], S[31]] == [7, 9, 35, 35, 63]
    w = plane_w(prm)
    assert w[0] == 0.0 and abs(w[1] - 1.0) < 1e-12 and w[31] == 961.0
    # ties go up: y = 8 exactly -> 9
    prm2 = Params(grid_n=64, cell_rad=1e-3, support_min=7, support_max=9, oversample=8,
                  n_wplanes=3, w_max_lambda=1.0)
    assert list(plane_support(prm2)) == [7, 9, 9]
    assert list(fine_offsets(8, 3)) == list(range(-11, 13))
