"""Pins for the oracle's index selection (oracle/index.py)."""
import os

import numpy as np

from oracle.index import FLAG_CONJ, FLAG_VALID, index_vis
from oracle.wkernel import C0, Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "index_cases.txt")


def golden_params():
    return Params(grid_n=16, cell_rad=1.0 / 16, support_min=7, support_max=11, oversample=8,
                  n_wplanes=3, w_max_lambda=4.0, npol=1)


def read_golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append(([float(f[0]), float(f[1]), float(f[2])], [int(x) for x in f[3:9]]))
    return rows


def test_golden_hand_computed_cases():
    rows = read_golden()
    uvw = np.array([r[0] for r in rows])
    exp = np.array([r[1] for r in rows])
    idx = index_vis(uvw, np.array([C0]), golden_params())
    got = np.stack([idx["ku"], idx["kv"], idx["ou"], idx["ov"], idx["plane"], idx["flags"]], 1)
    want = exp[:, [0, 1, 2, 3, 4, 5]]
    for i in range(len(rows)):
        assert list(got[i]) == list(want[i]), (rows[i], got[i])


def test_offset_range_and_reconstruction():
    """o in [-beta/2, beta/2) and k*beta + o is the nearest fine-grid point."""
    rng = np.random.default_rng(3)
    prm = Params(grid_n=256, cell_rad=1e-3, support_min=7, support_max=7, oversample=8,
                 n_wplanes=1, w_max_lambda=0.0)
    uvw = rng.uniform(-400, 400, size=(2000, 3))
    freq = np.array([1.2e8, 1.5e8])
    idx = index_vis(uvw, freq, prm)
    v = idx["valid"]
    assert v.mean() > 0.9
    for k, o, col in (("ku", "ou", 0), ("kv", "ov", 1)):
        assert np.all(idx[o][v] >= -4) and np.all(idx[o][v] < 4)
        x = ((uvw[:, col][:, None] * freq[None, :]) / C0 * prm.field + 128).reshape(-1)
        q = idx[k] * 8 + idx[o]
        assert np.all(np.abs(q[v] / 8.0 - x[v]) <= 1 / 16 + 1e-12)


def test_flags_and_invalid_zeros():
    prm = golden_params()
    uvw = np.array([[0.0, 0.0, -2.0], [100.0, 0.0, 1.0]])
    idx = index_vis(uvw, np.array([C0]), prm)
    assert idx["flags"][0] == FLAG_VALID | FLAG_CONJ
    assert idx["flags"][1] == 0
    assert idx["ku"][1] == 0 and idx["plane"][1] == 0


def test_plane_is_nearest_in_sqrt_w_exactly():
    """The threshold count equals the plane nearest in sqrt(|w|) (ties up,
    clamped to P - 1) decided in exact rational arithmetic:
    p >= j  <=>  (j - 1/2)^2 w_max <= (P - 1)^2 |w|."""
    from fractions import Fraction
    from oracle.index import plane_thresholds
    rng = np.random.default_rng(11)
    for P, wmax in ((2, 3.0), (5, 1000.0), (32, 2300.0), (129, 77.7)):
        prm = Params(grid_n=64, cell_rad=1e-3, support_min=7, support_max=15, oversample=8,
                     n_wplanes=P, w_max_lambda=wmax)
        w = np.concatenate([rng.uniform(-1.2 * wmax, 1.2 * wmax, 400),
                            rng.uniform(-wmax / P**2, wmax / P**2, 100)])
        uvw = np.stack([np.zeros_like(w), np.zeros_like(w), w], axis=1)
        got = index_vis(uvw, np.array([C0]), prm)["plane"]
        Fw = Fraction(wmax)
        for wi, pi in zip(w, got):
            a = Fraction(abs(float(wi)))
            exact = sum(1 for j in range(1, P)
                        if (Fraction(2 * j - 1, 2) ** 2) * Fw <= (P - 1) ** 2 * a)
            assert pi == exact, (P, wi, pi, exact)
        # the square-root form of the same rule agrees away from the thresholds
        T = plane_thresholds(prm)
        far = np.min(np.abs(np.abs(w)[:, None] - T[None, :]), axis=1) > 1e-9 * wmax
        s = np.sqrt(np.abs(w) / wmax) * (P - 1)
        want = np.minimum(np.floor(s + 0.5), P - 1).astype(np.int64)
        assert np.array_equal(got[far], want[far])


def test_channel_factor_is_one_division_per_channel():
    """u_lambda = u * (f / c0): with f = c0 the factor is exactly 1, so the
    coordinate in wavelengths is the metre value itself."""
    from oracle.index import chan_scale
    assert chan_scale(np.array([C0]))[0] == 1.0
    # u_lambda * lambda recovers u to rounding (two roundings, < 4 ulp)
    rng = np.random.default_rng(5)
    f = rng.uniform(5e7, 2e9, 64)
    u = rng.uniform(-2e4, 2e4, 64)
    lam_m = C0 / f
    back = (u * chan_scale(f)) * lam_m
    assert np.all(np.abs(back - u) <= 4 * np.spacing(np.abs(u)))
