"""Serving on the GPU: device-count calls and their CUDA graphs, plan clones
and tuning, and the continuous-batching server (each job's result is the
same alone and in the mix).

Tolerances: degridding is deterministic (fixed reduction order), so results
agree to FP32 rounding of identical sums (relative L2 <= 1e-6); gridding
commits with atomics in a run-dependent order (relative L2 <= 1e-6).
"""
import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TOL = 1e-6


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


def rel(a, b):
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def small():
    return syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                          s_max=21, n_w=5, diameter_m=1500.0)


def test_devcount_and_graph_replay_match_plain_calls(gw):
    obs = small()
    u, f, v = dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)
    rng = np.random.default_rng(0)
    model = dev((rng.normal(size=(4, 128, 128)) + 1j * rng.normal(size=(4, 128, 128)))
                .astype(np.complex64))
    with gw.Plan.from_observation(obs) as master:
        plan = master.clone(max_vis_per_call=obs.nvis)
        d_n = torch.zeros(1, dtype=torch.int64, device=DEV)
        g = plan.new_grid()
        vo = torch.zeros_like(v)
        # device count
        for nrow in (obs.nrow, 37, 1, 0):
            d_n.fill_(nrow)
            g.zero_()
            plan.grid_devcount(u, f, d_n, v, g)
            want = master.grid(u[:nrow], f, v[:nrow]) if nrow else master.new_grid()
            assert rel(g, want) <= TOL if nrow else not torch.any(g != 0)
            vo.fill_(7)
            plan.degrid_devcount(u, f, d_n, model, vo)
            if nrow:
                want = master.degrid(u[:nrow], f, model)
                assert rel(vo[:nrow], want) <= TOL
            assert torch.all(vo[nrow:] == 7)               # rows past the count untouched
        # one captured graph, replayed for several sizes
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            d_n.fill_(obs.nrow)
            g.zero_()
            plan.grid_devcount(u, f, d_n, v, g)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            g.zero_()
            plan.grid_devcount(u, f, d_n, v, g)
        for nrow in (obs.nrow, 55, 3):
            d_n.fill_(nrow)
            graph.replay()
            torch.cuda.synchronize()
            assert rel(g, master.grid(u[:nrow], f, v[:nrow])) <= TOL
        plan.close()


def test_clone_shares_tables_and_outlives_master(gw):
    obs = small()
    u, f, v = dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)
    master = gw.Plan.from_observation(obs)
    want = master.grid(u, f, v)
    tab = master.tables()[0]
    clone = master.clone(max_vis_per_call=1000)
    assert clone.info.table_bytes == master.info.table_bytes
    assert clone.info.scratch_bytes != master.info.scratch_bytes
    master.close()                                    # the tables stay alive for the clone
    assert np.array_equal(clone.tables()[0], tab)
    assert rel(clone.grid(u, f, v), want) <= TOL      # several chunks of 1000
    clone.close()


@pytest.mark.parametrize("item_max,degrid_kernel,grid_kernel,plane_groups",
                         [(64, 2, 1, 2), (256, 1, 2, 1), (4096, 0, 0, 0), (1024, 0, 1, 3)])
def test_tuning_changes_nothing_but_speed(gw, item_max, degrid_kernel, grid_kernel, plane_groups):
    obs = small()
    u, f, v = dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)
    with gw.Plan.from_observation(obs) as plan:
        g0 = plan.grid(u, f, v)
        d0 = plan.degrid(u, f, g0)
        plan.set_tuning(item_max=item_max, degrid_kernel=degrid_kernel, grid_kernel=grid_kernel,
                        plane_groups=plane_groups)
        assert plan.get_tuning() == {"item_max": item_max, "degrid_kernel": degrid_kernel,
                                     "grid_kernel": grid_kernel, "compress_min_gain": 0,
                                     "plane_groups": plane_groups}
        assert plan.info.plane_groups == max(1, plane_groups)   # small FP32 tables: auto = 1
        assert rel(plan.grid(u, f, v), g0) <= TOL
        assert rel(plan.degrid(u, f, g0), d0) <= TOL
        with pytest.raises(gw.GwError):
            plan.set_tuning(item_max=3)
        with pytest.raises(gw.GwError):
            plan.set_tuning(grid_kernel=3)
        with pytest.raises(gw.GwError):
            plan.set_tuning(plane_groups=17)


def test_autotuner_picks_a_candidate(gw):
    from paper_2111_04141_gb300.tune import TuningCache, tune_plan
    obs = small()
    u, f, v = dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)
    with gw.Plan.from_observation(obs) as plan:
        res = tune_plan(plan, u, f, v, plan.new_grid(), reps=1, items=(256, 1024),
                        degrid=(1, 2))
        assert res["tuning"] == plan.get_tuning()
        assert len(res["timings"]) == 4
    c = TuningCache()
    c.put("x", res["tuning"])
    assert c.get("x") == res["tuning"]


@pytest.mark.parametrize("use_graphs,bands,shared", [(True, 0, False), (True, 4, False),
                                                     (False, 0, False), (True, 0, True)],
                         ids=["graphs", "graphs-readback", "plain", "graphs-shared-staging"])
def test_server_results_same_alone_and_in_the_mix(gw, use_graphs, bands, shared):
    from paper_2111_04141_gb300.serve import Server, build_stream, run_sequential
    max_vis = 60_000
    specs = syn.serving_setups(n_setups=4, max_vis=max_vis, grid_sizes=(256, 512))
    jspecs = syn.serving_jobs(specs, n_jobs=24, min_vis=500, max_vis=max_vis)
    arrivals = syn.poisson_arrivals(len(jspecs), 2000.0)       # overlapping arrivals
    setups, jobs = build_stream(specs, jspecs, arrivals, max_vis)
    rng = np.random.default_rng(3)
    models = {s.name: (rng.normal(size=(s.npol, s.grid_n, s.grid_n))
                       + 1j * rng.normal(size=(s.npol, s.grid_n, s.grid_n))).astype(np.complex64)
              for s in setups}
    mixed = {}
    staging = None
    if shared:
        # caller-provided pinned result staging (as servers that take turns share it)
        n_host = max(max(s.npol * s.grid_n ** 2, -(-max_vis // s.nchan) * s.nchan * s.npol)
                     for s in setups)
        small_bufs = [torch.empty(n_host - 1, dtype=torch.complex64, pin_memory=True)] * 3
        with pytest.raises(ValueError):
            Server(setups, DEV, budget=8 << 30, n_slots=3, max_vis=max_vis,
                   host_staging=small_bufs).warm(models)
        staging = [torch.empty(n_host, dtype=torch.complex64, pin_memory=True) for _ in range(3)]
    srv = Server(setups, DEV, budget=8 << 30, n_slots=3, max_vis=max_vis, use_graphs=use_graphs,
                 readback_bands=bands, on_result=lambda j, t: mixed.__setitem__(j.id, t.clone()),
                 host_staging=staging)
    srv.warm(models)
    if shared:
        assert all(srv.slots[k]["host"] is staging[k] for k in range(3))
    done = srv.run(jobs)
    assert len(done) == len(jobs) and len(mixed) == len(jobs)
    assert all(j.t_done >= j.t_admit >= j.arrival for j in done)
    slots_used = {j.slot for j in done}
    assert len(slots_used) > 1
    # every job alone: the setup's master plan, plain calls, one at a time
    alone = {}
    for j in jobs:
        j.arrival = 0.0
    run_sequential(setups, srv.plans, srv.models, srv.freqs, jobs, DEV,
                   on_result=lambda j, t: alone.__setitem__(j.id, t.clone()),
                   host_buf=staging[0] if shared else None)
    for j in jobs:
        assert rel(mixed[j.id], alone[j.id]) <= TOL, (j.id, j.kind, j.setup)
    srv.close()


@pytest.mark.parametrize("n_bands", [1, 3, 8, 64])
def test_grid_readback_matches_devcount(gw, n_bands):
    """Banded gridding with read-back (gw_grid_vis_devcount_readback): the
    host copy equals the device grid it leaves behind, both match plain
    device-count gridding, for band counts from 1 to more than the tile rows;
    and the call replays from a CUDA graph with another row count."""
    obs = syn.small_case(n_ant=10, n_times=24, n_chan=3, npol=4, grid_n=160, s_min=7,
                         s_max=31, n_w=6, diameter_m=1500.0, seed=4)
    uvw, freq, vis = dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)
    with gw.Plan.from_observation(obs) as plan:
        d_nrow = torch.tensor([obs.nrow], dtype=torch.int64, device=DEV)
        ref = plan.grid_devcount(uvw, freq, d_nrow, vis, plan.new_grid())
        g = plan.new_grid()
        host = torch.empty(g.shape, dtype=torch.complex64).pin_memory()
        plan.grid_devcount_readback(uvw, freq, d_nrow, vis, g, host, n_bands=n_bands)
        torch.cuda.synchronize()
        assert torch.equal(host, g.cpu())
        assert rel(g, ref) <= TOL
        # captured once, replayed for a different row count
        s = torch.cuda.Stream()
        g2 = plan.new_grid()
        host2 = torch.empty(g.shape, dtype=torch.complex64).pin_memory()

        def body():
            g2.zero_()
            plan.grid_devcount_readback(uvw, freq, d_nrow, vis, g2, host2, n_bands=n_bands)

        with torch.cuda.stream(s):
            body()
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            body()
        half = obs.nrow // 2
        d_nrow.fill_(half)
        ref_half = plan.grid_devcount(uvw, freq, d_nrow, vis, plan.new_grid())
        host2.zero_()
        with torch.cuda.stream(s):
            graph.replay()
        s.synchronize()
        assert torch.equal(host2, g2.cpu())
        assert rel(host2.to(DEV), ref_half) <= TOL
        with pytest.raises(gw.GwError):
            plan.grid_devcount_readback(uvw, freq, d_nrow, vis, g, host, n_bands=0)


def test_hugepage_pinned_buffers(gw):
    """Page-locked host buffers from hostmem: pinned, exact round trips
    through the device, released on request; small ones use the ordinary
    page-locked allocator."""
    from paper_2111_04141_gb300 import hostmem
    n = (hostmem.MIN_HUGE_BYTES // 8) * 2
    before = hostmem.live_bytes()
    t = hostmem.pinned_empty((n,), torch.complex64)
    assert t.is_pinned() and tuple(t.shape) == (n,) and t.dtype == torch.complex64
    src = torch.randn(n, dtype=torch.complex64, device=DEV)
    t.copy_(src, non_blocking=True)
    back = torch.empty_like(src)
    back.copy_(t, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(back, src)
    grew = hostmem.live_bytes() - before
    assert grew in (0, n * 8)          # 0 where the host has no huge pages
    hostmem.release(t)
    assert hostmem.live_bytes() == before
    small = hostmem.pinned_empty((1000, 3), torch.float64)
    assert small.is_pinned() and tuple(small.shape) == (1000, 3)
    assert hostmem.live_bytes() == before
