"""Error paths of the C ABI under injected allocation failures.

The library's test hook (gw_debug_fail_alloc) makes the n-th allocation from
now fail on the host, as if the device or host were out of memory; nothing
faulty ever reaches the GPU.  For every allocation a call makes, the call
must return GW_ENOMEM, free what it had allocated (live plans and the
library's live device bytes back where they were) and leave the plan usable: the next call
succeeds and gives the reference result."""
import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
GW_ENOMEM = -2


def _setup():
    from paper_2111_04141_gb300 import build as b
    b.build()
    import paper_2111_04141_gb300 as gw
    from paper_2111_04141_gb300 import plan as P
    obs = syn.small_case(n_ant=6, n_times=8, n_chan=3, npol=2, grid_n=96, s_min=7, s_max=15,
                         n_w=4, diameter_m=1200.0)
    return gw, P, obs


def _sweep(P, call, max_n=80):
    """Fail the 1st, 2nd, ... allocation of `call` until it succeeds; each
    failure must be GW_ENOMEM with live plans and device memory unchanged.
    Returns the number of allocations the call made."""
    import paper_2111_04141_gb300 as gw
    base_plans = P.live_plans()
    base_bytes = P.live_bytes()
    for n in range(1, max_n + 1):
        P.debug_fail_alloc(n)
        try:
            res = call()
        except gw.GwError as exc:
            P.debug_fail_alloc(0)
            assert exc.status == GW_ENOMEM, (n, str(exc))
            assert P.live_plans() == base_plans, n
            assert P.live_bytes() == base_bytes, n
            continue
        P.debug_fail_alloc(0)
        return n - 1, res
    raise AssertionError("the call kept failing")


def test_plan_create_and_clone_fail_cleanly():
    gw, P, obs = _setup()
    with torch.cuda.device(DEV):
        gw.Plan.from_observation(obs).close()          # modules loaded once
        n_alloc, plan = _sweep(P, lambda: gw.Plan.from_observation(obs))
        assert n_alloc >= 10                            # tables, scratch, plan objects
        n_clone, clone = _sweep(P, lambda: plan.clone(max_vis_per_call=4096))
        assert n_clone >= 5
        uvw = torch.from_numpy(obs.uvw_m).to(DEV)
        freq = torch.from_numpy(obs.freq_hz).to(DEV)
        vis = torch.from_numpy(obs.vis).to(DEV)
        ref = plan.grid(uvw, freq, vis)
        got = clone.grid(uvw, freq, vis)
        assert torch.equal(got, ref) or float((got - ref).abs().max()) <= 1e-6 * float(
            ref.abs().max())
        clone.close()
        plan.close()


def test_lazy_scratch_fails_cleanly_and_the_plan_stays_usable():
    """Weighted gridding, host-input gridding and full compression allocate
    their scratch on first use."""
    gw, P, obs = _setup()
    w = syn.random_weights(obs)
    with torch.cuda.device(DEV):
        plan = gw.Plan.from_observation(obs)
        uvw = torch.from_numpy(obs.uvw_m).to(DEV)
        freq = torch.from_numpy(obs.freq_hz).to(DEV)
        vis = torch.from_numpy(obs.vis).to(DEV)
        wt = torch.from_numpy(w).to(DEV)
        fresh = gw.Plan.from_observation(obs)
        ref_w = fresh.grid(uvw, freq, vis, weight=wt)
        ref = fresh.grid(uvw, freq, vis)
        ref_c = fresh.grid_compressed(uvw, freq, vis)[0]
        fresh.close()
        tol = 1e-6 * float(ref.abs().max())

        plan.set_tuning(grid_kernel=1)      # binned: weighted scratch allocated on first use
        n, g = _sweep(P, lambda: plan.grid(uvw, freq, vis, weight=wt))
        assert n == 1 and float((g - ref_w).abs().max()) <= tol
        pin_uvw = torch.from_numpy(obs.uvw_m).pin_memory()
        pin_freq = torch.from_numpy(obs.freq_hz).pin_memory()
        pin_vis = torch.from_numpy(obs.vis).pin_memory()
        n, g = _sweep(P, lambda: plan.grid_host(pin_uvw, pin_freq, pin_vis))
        assert n >= 4 and float((g - ref).abs().max()) <= tol
        n, res = _sweep(P, lambda: plan.grid_compressed(uvw, freq, vis))
        assert n >= 5 and float((res[0] - ref_c).abs().max()) <= tol
        plan.close()


def test_hook_is_off_after_firing_and_rejects_negative():
    gw, P, obs = _setup()
    with torch.cuda.device(DEV):
        P.debug_fail_alloc(1)
        with pytest.raises(gw.GwError):
            gw.Plan.from_observation(obs)
        gw.Plan.from_observation(obs).close()           # the hook fired once and is off
        with pytest.raises(gw.GwError):
            P.debug_fail_alloc(-1)


def test_device_status_word_is_clear_after_gridding():
    """The status word a bounded device wait sets when it gives up reads 0
    (GW_OK) after gridding and degridding that completed, and reading it
    leaves the plan usable."""
    gw, P, obs = _setup()
    with torch.cuda.device(DEV):
        with gw.Plan.from_observation(obs) as plan:
            uvw = torch.from_numpy(obs.uvw_m).to(DEV)
            freq = torch.from_numpy(obs.freq_hz).to(DEV)
            vis = torch.from_numpy(obs.vis).to(DEV)
            for kernel in (1, 2):
                plan.set_tuning(**dict(plan.get_tuning(), grid_kernel=kernel))
                g = plan.grid(uvw, freq, vis)
                plan.device_status()
                out = plan.degrid(uvw, freq, g)
                plan.device_status()
                assert torch.isfinite(torch.view_as_real(out)).all()
