"""The oracle's lattice evaluator equals the full oracle grid at those points."""
import numpy as np

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.wkernel import Params


def test_lattice_equals_full_grid():
    obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=2, grid_n=128, s_min=7, s_max=21,
                         n_w=5, diameter_m=1500.0)
    orc = Oracle(Params(**obs.plan_kwargs()))
    wt = syn.random_weights(obs)
    full = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis, weight=wt)
    for off, step in ((0, 1), (3, 7), (50, 13)):
        m = (128 - off + step - 1) // step
        lat = orc.grid_lattice(obs.uvw_m, obs.freq_hz, obs.vis, off, step, m, weight=wt)
        pts = off + step * np.arange(m)
        assert np.array_equal(lat, full[:, pts][:, :, pts])
