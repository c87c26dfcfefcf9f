"""Full compression on the GPU (gw_grid_vis_compressed) against the oracle:
the number of distinct records is exact (integer work), the grid matches the
oracle's grid of the uncompressed visibilities (relative L2 <= 1e-5)."""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.compress import full_compression
from oracle.wkernel import Params

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def gw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build()
    import paper_2111_04141_gb300 as gw
    return gw


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dense_case():
    obs = syn.small_case(n_ant=6, n_times=8, n_chan=2, npol=2, grid_n=96, s_min=7, s_max=15,
                         n_w=4, diameter_m=900.0)
    rng = np.random.default_rng(5)
    uvw = np.repeat(obs.uvw_m, 3, axis=0)
    vis = (rng.normal(size=(uvw.shape[0], obs.nchan, obs.npol))
           + 1j * rng.normal(size=(uvw.shape[0], obs.nchan, obs.npol))).astype(np.complex64)
    return obs, uvw, vis


@pytest.mark.parametrize("which", ["dense", "small-w"])
@pytest.mark.parametrize("weighted", [False, True])
def test_compressed_grid_and_count(gw, which, weighted):
    if which == "dense":
        obs, uvw, vis = dense_case()
    else:
        obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                             s_max=21, n_w=5, diameter_m=1500.0)
        uvw, vis = obs.uvw_m, obs.vis
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    idx = orc.index(uvw, obs.freq_hz)
    wt = np.random.default_rng(2).uniform(0.5, 1.5, size=vis.shape).astype(np.float32) \
        if weighted else None
    ref = orc.grid(uvw, obs.freq_hz, vis, weight=wt, idx=idx)
    cidx, _ = full_compression(idx, vis, wt)
    with gw.Plan.from_observation(obs) as plan:
        g, n_gridded, dropped = plan.grid_compressed(dev(uvw), dev(obs.freq_hz), dev(vis),
                                                     weight=dev(wt) if weighted else None)
        plain = plan.grid(dev(uvw), dev(obs.freq_hz), dev(vis),
                          weight=dev(wt) if weighted else None)
    assert n_gridded == cidx["ku"].shape[0]
    assert dropped == int((~idx["valid"]).sum())
    got = g.cpu().numpy().astype(np.complex128)
    assert rel_l2(got, ref) <= 1e-5
    assert rel_l2(got, plain.cpu().numpy().astype(np.complex128)) <= 1e-5


def test_compression_within_chunks(gw):
    """Compression acts within each internal chunk: the count is the sum of
    the per-chunk distinct records."""
    obs, uvw, vis = dense_case()
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    rows = 50
    expect = 0
    for r0 in range(0, uvw.shape[0], rows):
        idx = orc.index(uvw[r0:r0 + rows], obs.freq_hz)
        expect += full_compression(idx, vis[r0:r0 + rows])[0]["ku"].shape[0]
    ref = orc.grid(uvw, obs.freq_hz, vis)
    with gw.Plan.from_observation(obs, max_vis_per_call=rows * obs.nchan) as plan:
        g, n_gridded, _ = plan.grid_compressed(dev(uvw), dev(obs.freq_hz), dev(vis))
        # a second call on the same plan starts from an empty table
        g2, n2, _ = plan.grid_compressed(dev(uvw), dev(obs.freq_hz), dev(vis))
    assert n_gridded == expect == n2
    assert rel_l2(g.cpu().numpy().astype(np.complex128), ref) <= 1e-5
    assert rel_l2(g2.cpu().numpy().astype(np.complex128), ref) <= 1e-5


@pytest.mark.parametrize("which", ["dense", "small-w"])
def test_compression_decision_from_a_sample(gw, which):
    """With compress_min_gain set, the call compresses a sample first (the
    first rows, up to 2^18 visibilities) and compresses only when at least
    that share of its records merges; either way the grid is the same."""
    if which == "dense":
        obs, uvw, vis = dense_case()         # every row three times: 2/3 merge
    else:
        obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                             s_max=21, n_w=5, diameter_m=1500.0)
        uvw, vis = obs.uvw_m, obs.vis
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    idx = orc.index(uvw, obs.freq_hz)
    cidx, _ = full_compression(idx, vis)
    valid = int(idx["valid"].sum())
    merged = 1.0 - cidx["ku"].shape[0] / valid   # the sample is the whole (small) input
    ref = orc.grid(uvw, obs.freq_hz, vis, idx=idx)
    gain = 500
    with gw.Plan.from_observation(obs) as plan:
        plan.set_tuning(compress_min_gain=gain)
        g, n_gridded, dropped = plan.grid_compressed(dev(uvw), dev(obs.freq_hz), dev(vis))
    expect = cidx["ku"].shape[0] if merged * 1000 >= gain else valid
    assert (which == "dense") == (merged * 1000 >= gain)
    assert n_gridded == expect
    assert dropped == int((~idx["valid"]).sum())
    assert rel_l2(g.cpu().numpy().astype(np.complex128), ref) <= 1e-5
