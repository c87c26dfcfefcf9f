"""Pins of the oracle's full compression (oracle/compress.py): a brute-force
dictionary grouping gives the same records and sums; gridding the compressed
records reproduces gridding the originals (linearity, FP64)."""
import numpy as np

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.compress import full_compression, record_keys
from oracle.wkernel import Params


def dense_case():
    """Every uvw row three times (different visibilities): heavy compression."""
    obs = syn.small_case(n_ant=6, n_times=8, n_chan=2, npol=2, grid_n=96, s_min=7, s_max=15,
                         n_w=4, diameter_m=900.0)
    rng = np.random.default_rng(5)
    uvw = np.repeat(obs.uvw_m, 3, axis=0)
    vis = (rng.normal(size=(uvw.shape[0], obs.nchan, obs.npol))
           + 1j * rng.normal(size=(uvw.shape[0], obs.nchan, obs.npol))).astype(np.complex64)
    return obs, uvw, vis


def test_matches_brute_force_grouping():
    obs, uvw, vis = dense_case()
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    idx = orc.index(uvw, obs.freq_hz)
    wt = np.random.default_rng(1).uniform(0.5, 1.5, size=vis.shape)
    cidx, cvis = full_compression(idx, vis, wt)
    groups = {}
    keys = record_keys(idx)
    v = vis.reshape(-1, prm.npol).astype(np.complex128) * wt.reshape(-1, prm.npol)
    for i in range(keys.shape[0]):
        if not idx["valid"][i]:
            continue
        k = tuple(int(x) for x in keys[i])
        groups[k] = groups.get(k, 0) + v[i]
    assert len(groups) == cvis.shape[0] < idx["valid"].sum()
    ck = record_keys(cidx)
    for j in range(ck.shape[0]):
        assert np.allclose(groups[tuple(int(x) for x in ck[j])], cvis[j], rtol=1e-14, atol=1e-14)


def test_gridding_compressed_equals_gridding_all():
    for obs, uvw, vis in [dense_case(), (lambda o: (o, o.uvw_m, o.vis))(
            syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                           s_max=21, n_w=5, diameter_m=1500.0))]:
        prm = Params(**obs.plan_kwargs())
        orc = Oracle(prm)
        idx = orc.index(uvw, obs.freq_hz)
        ref = orc.grid(uvw, obs.freq_hz, vis, idx=idx)
        cidx, cvis = full_compression(idx, vis)
        got = orc.grid(None, None, cvis, idx=cidx)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
