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
