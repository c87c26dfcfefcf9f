"""Pins for the oracle's gridding / degridding loops (oracle/cgrid.c)."""
import numpy as np
import pytest

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.image import centred_idft
from oracle.pswf import PSWF0, taper_bandwidth
from oracle.wkernel import C0, Params, kernel_fine


def tiny_prm(P=3, smin=7, smax=11, N=48, beta=8, npol=2, w_max=150.0):
    return Params(grid_n=N, cell_rad=0.3 / N, support_min=smin, support_max=smax,
                  oversample=beta, n_wplanes=P, w_max_lambda=w_max if P > 1 else 0.0, npol=npol)


def exact_uvw(prm, pix_u, pix_v, w):
    """uvw (metres at f = c0) whose pixel coordinate is exactly N/2 + pix."""
    L = prm.field
    return np.array([[pu / L, pv / L, ww] for pu, pv, ww in zip(pix_u, pix_v, w)])


@pytest.mark.parametrize("w_sign", [1.0, -1.0])
def test_single_visibility_reproduces_table_slice(w_sign):
    prm = tiny_prm()
    orc = Oracle(prm)
    # pixel offset 3 + 2/8 in u, -5 - 3/8 in v, w chosen to land on plane 2
    uvw = exact_uvw(prm, [3.25], [-5.375], [w_sign * 150.0])
    idx = orc.index(uvw, np.array([C0]))
    assert idx["plane"][0] == 2 and idx["ou"][0] == 2 and idx["ov"][0] == -3
    vis = np.array([[[1.0, 2.0 - 1.0j]]], dtype=np.complex64)
    g = orc.grid(uvw, np.array([C0]), vis)
    K = orc.tables.planes[2][-3 + 4, 2 + 4]
    if w_sign < 0:
        K = np.conj(K)
    h = (K.shape[0] - 1) // 2
    ku, kv = idx["ku"][0], idx["kv"][0]
    for pol, val in enumerate([1.0, 2.0 - 1.0j]):
        win = g[pol, kv - h:kv + h + 1, ku - h:ku + h + 1]
        assert np.array_equal(win, K * val)
        rest = g[pol].copy()
        rest[kv - h:kv + h + 1, ku - h:ku + h + 1] = 0
        assert not np.any(rest)


def test_equivalence_theorem():
    """Section 2.4.2 (Algorithm equivalentalgo): gridding with the oversampled
    table equals NN interpolation onto the beta-fine grid followed by a
    convolution with the fine-sampled GCF and decimation to the coarse grid."""
    prm = tiny_prm(P=1, smin=7, smax=7, N=32, beta=4, npol=1)
    orc = Oracle(prm)
    obs = syn.small_case(n_ant=5, n_times=6, n_chan=2, npol=1, grid_n=32, s_min=7, s_max=7,
                         n_w=1, beta=4, diameter_m=500.0)
    prm = Params(**dict(obs.plan_kwargs()))
    orc = Oracle(prm)
    idx = orc.index(obs.uvw_m, obs.freq_hz)
    assert idx["valid"].all()
    g = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis)[0]
    beta, N = prm.oversample, prm.grid_n
    # NN interpolation onto the fine grid (fine index q = k beta + o)
    qu = idx["ku"] * beta + idx["ou"]
    qv = idx["kv"] * beta + idx["ov"]
    nn = np.zeros((N * beta, N * beta), dtype=np.complex128)
    np.add.at(nn, (qv, qu), obs.vis.reshape(-1).astype(np.complex128))
    # fine-sampled GCF C(f / beta), the same scale as the table
    f, Kf = kernel_fine(prm, 0.0, 7, PSWF0(taper_bandwidth(7)))
    Kf = Kf * orc.tables.scale
    fmin, fmax = f[0], f[-1]
    ref = np.zeros((N, N), dtype=np.complex128)
    nzv, nzu = np.nonzero(nn)
    for a, b in zip(nzv, nzu):
        for kv in range(N):
            fv = beta * kv - a
            if fv < fmin or fv > fmax:
                continue
            for ku in range(N):
                fu = beta * ku - b
                if fu < fmin or fu > fmax:
                    continue
                ref[kv, ku] += nn[a, b] * Kf[fv - fmin, fu - fmin]
    assert np.max(np.abs(g - ref)) <= 1e-13 * np.max(np.abs(ref))


def _obs(P=3):
    return syn.small_case(n_ant=6, n_times=5, n_chan=3, npol=2, grid_n=64, s_min=7, s_max=15,
                          n_w=P, diameter_m=700.0)


def test_linearity_and_adjoint():
    obs = _obs()
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    rng = np.random.default_rng(5)
    x1 = obs.vis.astype(np.complex128)
    x2 = (rng.normal(size=x1.shape) + 1j * rng.normal(size=x1.shape))
    a, b = 0.7 - 0.2j, -1.3
    g1 = orc.grid(obs.uvw_m, obs.freq_hz, x1)
    g2 = orc.grid(obs.uvw_m, obs.freq_hz, x2)
    g12 = orc.grid(obs.uvw_m, obs.freq_hz, a * x1 + b * x2)
    assert np.max(np.abs(g12 - (a * g1 + b * g2))) <= 1e-12 * np.max(np.abs(g12))
    # <G x, y> = <x, G^H y>
    y = rng.normal(size=g1.shape) + 1j * rng.normal(size=g1.shape)
    lhs = np.vdot(y, g1)
    gh = orc.degrid(obs.uvw_m, obs.freq_hz, y)
    rhs = np.vdot(gh, x1.reshape(gh.shape))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_hermitian_symmetry():
    """vis(-u,-v,-w) = conj(vis) makes the grid conjugate-symmetric about the
    centre pixel and the image real (records kept off half-pixel offsets so
    that the mirrored footprint uses the mirrored table slice)."""
    prm = tiny_prm(P=3, N=64, npol=1)
    orc = Oracle(prm)
    rng = np.random.default_rng(9)
    n = 12
    beta = prm.oversample
    fu = rng.integers(-10 * beta, 10 * beta, n)
    fv = rng.integers(-10 * beta, 10 * beta, n)
    fu[(fu % beta) == beta // 2] += 1
    fv[(fv % beta) == beta // 2] += 1
    w = rng.uniform(-150, 150, n)
    uvw = exact_uvw(prm, fu / beta, fv / beta, w)
    uvw = np.concatenate([uvw, -uvw])
    vis = rng.normal(size=(n, 1, 1)) + 1j * rng.normal(size=(n, 1, 1))
    vis = np.concatenate([vis, np.conj(vis)])
    g = orc.grid(uvw, np.array([C0]), vis)[0]
    N = prm.grid_n
    mirror = np.conj(g[(N - np.arange(N)) % N][:, (N - np.arange(N)) % N])
    assert np.max(np.abs(g - mirror)) <= 1e-13 * np.max(np.abs(g))
    img = centred_idft(g)
    assert np.max(np.abs(img.imag)) <= 1e-12 * np.max(np.abs(img.real))


def test_exception_equal_offsets_exact():
    """Section 2.3.3 (Exceptions): when every record has the same sub-pixel
    offset y, the corrector 1 / l_co(y, x) makes Convolutional Gridding exact
    at every pixel (no aliasing)."""
    prm = tiny_prm(P=1, smin=7, smax=7, N=32, npol=1)
    orc = Oracle(prm)
    rng = np.random.default_rng(2)
    n = 15
    yu, yv = 3 / 8, -1 / 8
    pu = rng.integers(-10, 10, n) + yu
    pv = rng.integers(-10, 10, n) + yv
    uvw = exact_uvw(prm, pu, pv, np.zeros(n))
    vis = rng.normal(size=(n, 1, 1)) + 1j * rng.normal(size=(n, 1, 1))
    g = orc.grid(uvw, np.array([C0]), vis)[0]
    img = centred_idft(g)
    N = prm.grid_n
    lpix = (np.arange(N) - N // 2) / N
    K = orc.tables.planes[0][int(round(yv * 8)) + 4, int(round(yu * 8)) + 4]
    h = (K.shape[0] - 1) // 2
    t = np.arange(-h, h + 1)
    eu = np.exp(2j * np.pi * np.outer(lpix, t - yu))     # [j, tu]
    ev = np.exp(2j * np.pi * np.outer(lpix, t - yv))     # [i, tv]
    lco = ev @ K @ eu.T                                   # [i, j]
    dft = np.zeros((N, N), dtype=np.complex128)
    for a in range(n):
        dft += vis[a, 0, 0] * np.exp(2j * np.pi * (pv[a] * lpix[:, None] + pu[a] * lpix[None, :]))
    # img = l_co * f^g exactly; compared in the multiplied (well-conditioned) form
    assert np.max(np.abs(img - lco * dft)) <= 1e-13 * np.max(np.abs(img))
