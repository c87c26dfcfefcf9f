"""Pins of the oracle's Hybrid Gridding (oracle/hybrid.py): for records on
the beta-grid in u and on the beta-fine rows in v (no nearest-neighbour
shift), gridding + pruning + IFFT + correction reproduces the direct sum of
Eq. (ID) over the central half up to the PSWF truncation error; the pruning
table sums to 1 at zero offset and is even; a single record's fine-grid
footprint is the 1-D GCF on its row."""
import numpy as np
import pytest

from oracle import hybrid as hy
from oracle.cgrid import Oracle
from oracle.image import nudft_image
from oracle.wkernel import C0, Params


def params(N=64, S=15, beta=8):
    return Params(grid_n=N, cell_rad=0.3 / N, support_min=S, support_max=S, oversample=beta,
                  n_wplanes=1, w_max_lambda=0.0, npol=1)


def test_prune_table():
    for beta, sz in [(8, 15), (16, 13), (4, 7)]:
        Z = hy.prune_table(beta, sz)
        hz = (sz - 1) // 2
        assert Z.shape == (beta // 2, sz)
        assert abs(Z[beta // 4].sum() - 1.0) < 1e-14          # offset 0 row
        assert np.allclose(Z[beta // 4], Z[beta // 4][::-1], atol=1e-15)


def test_single_record_footprint():
    prm = params()
    orc = Oracle(prm)
    uvw = np.array([[3.25 / prm.field, -2.5 / prm.field, 0.0]])
    idx = orc.index(uvw, np.array([C0]))
    fine, keep = hy.fine_grid(prm, idx, np.ones((1, 1, 1)), 15)
    assert keep.all()
    q = idx["kv"][0] * 8 + idx["ov"][0]
    c = hy.kernel_u(prm)[idx["ou"][0] + 4]
    row = fine[0, q]
    cols = idx["ku"][0] + np.arange(-7, 8)
    assert np.allclose(row[cols], c, atol=1e-15) and np.count_nonzero(fine) == 15


@pytest.mark.parametrize("beta", [8, 16])
def test_hybrid_image_matches_direct_sum(beta):
    prm = params(beta=beta)
    N = prm.grid_n
    orc = Oracle(prm)
    rng = np.random.default_rng(3)
    n = 25
    span = 32 - 15 // 2 - 3
    fu = rng.integers(-span * beta, span * beta, n) / beta
    fv = rng.integers(-span * beta, span * beta, n) / beta
    uvw = np.stack([fu / prm.field, fv / prm.field, np.zeros(n)], 1)
    vis = (rng.normal(size=(n, 1, 1)) + 1j * rng.normal(size=(n, 1, 1))).astype(np.complex64)
    freq = np.array([C0])
    idx = orc.index(uvw, freq)
    fine, keep = hy.fine_grid(prm, idx, vis, 15)
    assert keep.all()
    img = hy.image(prm, hy.prune(prm, fine, 15), 15, nn_sinc=False)
    ref = nudft_image(uvw, freq, vis, prm)
    c = slice(N // 4, 3 * N // 4)
    err = np.max(np.abs(img[:, c, c] - ref[:, c, c])) / np.max(np.abs(ref[:, c, c]))
    assert err <= 1e-6
