"""Multi-rank gridding logic on CPU (gloo, world size 2).

Gridding is linear in the visibilities, so sharding the visibilities across
ranks, gridding each shard into a per-rank grid and summing the grids once
(the all-reduce bench.py performs under torchrun) equals gridding everything
on one device.  The per-rank gridder here is the FP64 oracle; the CUDA path
is covered by the GPU tests.
"""
import os

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synthetic as syn


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.cgrid import Oracle
    from oracle.wkernel import Params
    obs = syn.small_case(n_ant=6, n_times=8, n_chan=2, npol=2, grid_n=64, s_min=7, s_max=15,
                         n_w=3, diameter_m=800.0)
    orc = Oracle(Params(**obs.plan_kwargs()))
    rows = np.array_split(np.arange(obs.nrow), world)[rank]
    g = orc.grid(obs.uvw_m[rows], obs.freq_hz, obs.vis[rows], nthreads=1)
    t = torch.from_numpy(g.view(np.float64).copy())
    dist.all_reduce(t)
    if rank == 0:
        np.save(out_path, t.numpy().view(np.complex128))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_grids_sum_to_full_grid(tmp_path):
    out = str(tmp_path / "g.npy")
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    from oracle.cgrid import Oracle
    from oracle.wkernel import Params
    obs = syn.small_case(n_ant=6, n_times=8, n_chan=2, npol=2, grid_n=64, s_min=7, s_max=15,
                         n_w=3, diameter_m=800.0)
    full = Oracle(Params(**obs.plan_kwargs())).grid(obs.uvw_m, obs.freq_hz, obs.vis)
    got = np.load(out)
    assert np.max(np.abs(got - full)) <= 1e-12 * np.max(np.abs(full))
