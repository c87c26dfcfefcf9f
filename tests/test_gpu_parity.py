"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: index records, bin counts and bin membership are bit-exact;
FP32 grids and degridded visibilities within relative L2 1e-5 of the FP64
oracle; kernel tables within 2e-7 of the table's peak (FP32 storage of FP64
values); the corrector's reciprocal within 1e-12 absolute (and h within
1e-9 relative where |h| < 1e3).
"""
import os

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.image import centred_idft, correct
from oracle.index import index_vis
from oracle.wkernel import C0, KernelTables, Params, corrector, plane_support

pytestmark = pytest.mark.gpu

TOL_GRID = 1e-5
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "index_cases.txt")


@pytest.fixture(scope="module")
def gw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_04141_gb300 import build as b
    b.build()
    import paper_2111_04141_gb300 as gw
    return gw


DEV = torch.device("cuda", 0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


_ORACLES = {}


def oracle_for(prm):
    if prm not in _ORACLES:
        _ORACLES[prm] = Oracle(prm)
    return _ORACLES[prm]


CASES = {
    "2d": lambda: syn.config_2d(),
    "small-w": lambda: syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128,
                                      s_min=7, s_max=21, n_w=5, diameter_m=1500.0),
    "ragged": lambda: syn.small_case(n_ant=5, n_times=7, n_chan=5, npol=3, grid_n=90, s_min=5,
                                     s_max=13, n_w=3, diameter_m=900.0, beta=4, seed=3),
    "npol2-beta16": lambda: syn.small_case(n_ant=6, n_times=9, n_chan=2, npol=2, grid_n=160,
                                           s_min=9, s_max=9, n_w=1, diameter_m=1200.0,
                                           beta=16, seed=5),
    "bigS": lambda: syn.small_case(n_ant=6, n_times=12, n_chan=2, npol=1, grid_n=256,
                                   s_min=15, s_max=63, n_w=6, diameter_m=1500.0, seed=9),
    # staged degridding region (16 + 70)^2 x 4 pols > shared-memory budget:
    # exercises the global-gather fallback
    "wide-4pol": lambda: syn.small_case(n_ant=5, n_times=6, n_chan=2, npol=4, grid_n=256,
                                        s_min=15, s_max=71, n_w=4, diameter_m=1000.0, seed=13),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    obs = CASES[request.param]()
    return request.param, obs, Params(**obs.plan_kwargs())


# ---------------------------------------------------------------------------
# index stage (bit-exact)
# ---------------------------------------------------------------------------

def _gpu_index(gw, plan, uvw, freq):
    raw, dropped = plan.index(dev(uvw), dev(freq))
    return gw.Plan.unpack_index(raw.cpu().numpy()), dropped


def test_index_bit_exact(gw, case):
    name, obs, prm = case
    with gw.Plan.from_observation(obs) as plan:
        got, dropped = _gpu_index(gw, plan, obs.uvw_m, obs.freq_hz)
    ref = index_vis(obs.uvw_m, obs.freq_hz, prm)
    for key in ("ku", "kv", "ou", "ov", "plane", "flags"):
        assert np.array_equal(got[key], ref[key]), (name, key)
    assert dropped == int((~ref["valid"]).sum())


def test_index_golden_edges(gw):
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    uvw = np.array([[float(r[0]), float(r[1]), float(r[2])] for r in rows])
    want = np.array([[int(x) for x in r[3:9]] for r in rows])
    with gw.Plan(grid_n=16, cell_rad=1.0 / 16, support_min=7, support_max=11, oversample=8,
                 n_wplanes=3, w_max_lambda=4.0, npol=1) as plan:
        got, _ = _gpu_index(gw, plan, uvw, np.array([C0]))
    g = np.stack([got["ku"], got["kv"], got["ou"], got["ov"], got["plane"], got["flags"]], 1)
    assert np.array_equal(g, want)


def test_index_random_ties_and_extremes(gw):
    """Coordinates on exact fine-grid ties and random magnitudes."""
    rng = np.random.default_rng(17)
    prm = Params(grid_n=64, cell_rad=1.0 / 64, support_min=7, support_max=15, oversample=8,
                 n_wplanes=4, w_max_lambda=9.0, npol=1)
    n = 5000
    u = np.concatenate([rng.integers(-300, 300, n) / 16.0, rng.normal(0, 20, n)])
    v = np.concatenate([rng.integers(-300, 300, n) / 16.0, rng.normal(0, 20, n)])
    w = np.concatenate([rng.integers(-40, 40, n) / 4.0, rng.normal(0, 6, n)])
    uvw = np.stack([u, v, w], 1)
    uvw[::97, 0] = np.inf
    uvw[::89, 2] = np.nan
    uvw[::83, 1] = 1e15
    freq = np.array([C0, 0.75 * C0, 1.5 * C0])
    with gw.Plan(**prm.__dict__) as plan:
        got, _ = _gpu_index(gw, plan, uvw, freq)
    ref = index_vis(uvw, freq, prm)
    for key in ("ku", "kv", "ou", "ov", "plane", "flags"):
        assert np.array_equal(got[key], ref[key]), key


# ---------------------------------------------------------------------------
# tables and corrector
# ---------------------------------------------------------------------------

def test_tables_match_oracle(gw, case):
    name, obs, prm = case
    orc = oracle_for(prm)
    with gw.Plan.from_observation(obs) as plan:
        tab, offs, sup = plan.tables()
        h = plan.corrector()
    assert list(sup) == list(plane_support(prm))
    flat, roffs = orc.tables.flat()
    assert list(offs) == list(roffs)
    peak = np.max(np.abs(flat))
    assert np.max(np.abs(tab.astype(np.complex128) - flat)) <= 2e-7 * peak
    href = corrector(prm)
    # 1/h = chat * sinc is a sum of O(1) terms: compare it absolutely (h itself
    # reaches 1e9 at the field edge for wide tapers, where both sides lose
    # relative precision to cancellation)
    assert np.max(np.abs(1.0 / h - 1.0 / href)) <= 1e-12
    mid = np.abs(href) < 1e3
    assert np.max(np.abs(h[mid] - href[mid]) / np.abs(href[mid])) <= 1e-9


# ---------------------------------------------------------------------------
# binner
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [0, 1])
def test_bins(gw, case, mode):
    name, obs, prm = case
    ref = index_vis(obs.uvw_m, obs.freq_hz, prm)
    with gw.Plan.from_observation(obs) as plan:
        info = plan.info
    tu_, tv_ = (info.grid_tile_u, info.grid_tile_v) if mode == 0 else (info.degrid_tile,) * 2
    ntu = (prm.grid_n + tu_ - 1) // tu_
    ntv = (prm.grid_n + tv_ - 1) // tv_
    S = plane_support(prm)
    want = [[] for _ in range(ntu * ntv)]
    for i in np.nonzero(ref["valid"])[0]:
        h = int(S[ref["plane"][i]]) // 2
        ku, kv = int(ref["ku"][i]), int(ref["kv"][i])
        if mode == 1:
            want[(kv // tv_) * ntu + ku // tu_].append(i)
            continue
        for tv in range((kv - h) // tv_, (kv + h) // tv_ + 1):
            for tu in range((ku - h) // tu_, (ku + h) // tu_ + 1):
                want[tv * ntu + tu].append(i)
    with gw.Plan.from_observation(obs) as plan:
        offs, ent = plan.debug_bins(dev(obs.uvw_m), dev(obs.freq_hz), mode=mode)
    counts = np.diff(offs)
    assert list(counts) == [len(w) for w in want]
    for t in range(ntu * ntv):
        assert sorted(ent[offs[t]:offs[t + 1]].tolist()) == want[t]


@pytest.mark.parametrize("mode", [0, 1])
def test_bins_many_tiles(gw, mode):
    """More bins than one CTA scans (65536): the multi-CTA scan path.
    A 16384^2 grid has 131072 gridder tiles of 64 x 32 and 262144 degridder
    tiles of 32 x 32."""
    # 2-D (no w-term): at this grid size a w-projection field of view of a
    # small array would reach the horizon
    obs = syn.small_case(n_ant=12, n_times=20, n_chan=4, npol=1, grid_n=16384, s_min=15,
                         s_max=15, n_w=1, diameter_m=4000.0, seed=21)
    prm = Params(**obs.plan_kwargs())
    ref = index_vis(obs.uvw_m, obs.freq_hz, prm)
    S = plane_support(prm)
    with gw.Plan.from_observation(obs) as plan:
        info = plan.info
    tu_, tv_ = (info.grid_tile_u, info.grid_tile_v) if mode == 0 else (info.degrid_tile,) * 2
    ntu, ntv = 16384 // tu_, 16384 // tv_
    counts = np.zeros(ntu * ntv, dtype=np.int64)
    for i in np.nonzero(ref["valid"])[0]:
        h = int(S[ref["plane"][i]]) // 2
        ku, kv = int(ref["ku"][i]), int(ref["kv"][i])
        if mode == 1:
            counts[(kv // tv_) * ntu + ku // tu_] += 1
            continue
        for tv in range((kv - h) // tv_, (kv + h) // tv_ + 1):
            for tu in range((ku - h) // tu_, (ku + h) // tu_ + 1):
                counts[tv * ntu + tu] += 1
    with gw.Plan.from_observation(obs) as plan:
        offs, ent = plan.debug_bins(dev(obs.uvw_m), dev(obs.freq_hz), mode=mode)
    assert offs[0] == 0
    assert np.array_equal(np.diff(offs), counts)
    assert int(offs[-1]) == int(counts.sum()) == len(ent)


# ---------------------------------------------------------------------------
# gridding / degridding
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [1, 2], ids=["binned", "direct"])
def test_grid_matches_oracle(gw, case, kernel):
    name, obs, prm = case
    orc = oracle_for(prm)
    ref = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis)
    with gw.Plan.from_observation(obs) as plan:
        plan.set_tuning(grid_kernel=kernel)
        g, dropped = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis),
                               return_dropped=True)
    got = g.cpu().numpy().astype(np.complex128)
    assert rel_l2(got, ref) <= TOL_GRID, name
    assert dropped == int((~orc.index(obs.uvw_m, obs.freq_hz)["valid"]).sum())


@pytest.mark.parametrize("groups", [2, 0], ids=["two", "one-per-plane"])
def test_grid_plane_groups_match_oracle(gw, case, groups):
    """Bins keyed by (w-plane group, tile), served group by group, give the
    oracle's grid; 0 here asks for the most groups the plan allows (up to one
    per plane)."""
    name, obs, prm = case
    if prm.n_wplanes < 2:
        pytest.skip("one w-plane: nothing to group")
    orc = oracle_for(prm)
    ref = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis)
    with gw.Plan.from_observation(obs, max_vis_per_call=max(obs.nchan, obs.nvis // 3)) as plan:
        n = groups or min(prm.n_wplanes, 16)
        plan.set_tuning(grid_kernel=1, plane_groups=n)
        assert plan.info.plane_groups == n
        g = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)).cpu().numpy()
    assert rel_l2(g.astype(np.complex128), ref) <= TOL_GRID, (name, n)


@pytest.mark.parametrize("kernel", [1, 2], ids=["binned", "direct"])
def test_grid_weights_accumulate_and_chunks(gw, kernel):
    obs = CASES["small-w"]()
    prm = Params(**obs.plan_kwargs())
    orc = oracle_for(prm)
    wt = syn.random_weights(obs)
    ref = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis, weight=wt)
    # a small chunk size forces several internal chunks with a ragged last one
    with gw.Plan.from_observation(obs, max_vis_per_call=37 * obs.nchan + 1) as plan:
        plan.set_tuning(grid_kernel=kernel)
        g = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis), weight=dev(wt))
        got = g.cpu().numpy().astype(np.complex128)
        assert rel_l2(got, ref) <= TOL_GRID
        plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis), weight=dev(wt), out=g)
        assert rel_l2(g.cpu().numpy().astype(np.complex128), 2 * ref) <= TOL_GRID


@pytest.mark.parametrize("kernel", [1, 2], ids=["binned", "direct"])
def test_grid_empty_and_all_dropped(gw, kernel):
    obs = CASES["small-w"]()
    with gw.Plan.from_observation(obs) as plan:
        plan.set_tuning(grid_kernel=kernel)
        e3 = torch.zeros((0, 3), dtype=torch.float64, device=DEV)
        f = dev(obs.freq_hz)
        v = torch.zeros((0, obs.nchan, obs.npol), dtype=torch.complex64, device=DEV)
        g, dropped = plan.grid(e3, f, v, return_dropped=True)
        assert dropped == 0 and not torch.any(g != 0)
        far = obs.uvw_m * 1e6
        g, dropped = plan.grid(dev(far), f, dev(obs.vis), return_dropped=True)
        assert dropped == obs.nvis and not torch.any(g != 0)
        vo, dropped = plan.degrid(dev(far), f, plan.new_grid() + 1, return_dropped=True)
        assert dropped == obs.nvis and not torch.any(vo != 0)


def test_degrid_matches_oracle(gw, case):
    name, obs, prm = case
    orc = oracle_for(prm)
    rng = np.random.default_rng(21)
    N = prm.grid_n
    grid = (rng.normal(size=(prm.npol, N, N)) + 1j * rng.normal(size=(prm.npol, N, N)))
    grid = grid.astype(np.complex64)
    ref = orc.degrid(obs.uvw_m, obs.freq_hz, grid.astype(np.complex128))
    with gw.Plan.from_observation(obs) as plan:
        v = plan.degrid(dev(obs.uvw_m), dev(obs.freq_hz), dev(grid))
    got = v.cpu().numpy().reshape(ref.shape).astype(np.complex128)
    assert rel_l2(got, ref) <= TOL_GRID, name


@pytest.mark.parametrize("npol", [1, 3, 4])
def test_degrid_long_items_in_chunks(gw, npol):
    """Tiles holding more records than the staged degridder's metadata buffer
    (1,024) are served in several chunks from one region: with one work item
    per tile the result matches the oracle and the default item size, for
    region layouts of pairs only, pairs and a single plane, and a single
    plane."""
    obs = syn.small_case(n_ant=12, n_times=64, n_chan=4, npol=npol, grid_n=64, s_min=7,
                         s_max=15, n_w=4, diameter_m=400.0, seed=11)
    prm = Params(**obs.plan_kwargs())
    rng = np.random.default_rng(22)
    N = prm.grid_n
    grid = (rng.normal(size=(prm.npol, N, N)) + 1j * rng.normal(size=(prm.npol, N, N)))
    grid = grid.astype(np.complex64)
    ref = oracle_for(prm).degrid(obs.uvw_m, obs.freq_hz, grid.astype(np.complex128))
    with gw.Plan.from_observation(obs) as plan:
        idx, _ = _gpu_index(gw, plan, obs.uvw_m, obs.freq_hz)
        plan.set_tuning(**dict(plan.get_tuning(), item_max=1 << 20, degrid_kernel=1))
        v_long = plan.degrid(dev(obs.uvw_m), dev(obs.freq_hz), dev(grid)).cpu().numpy()
        plan.set_tuning(**dict(plan.get_tuning(), item_max=1024))
        v_def = plan.degrid(dev(obs.uvw_m), dev(obs.freq_hz), dev(grid)).cpu().numpy()
    got = v_long.reshape(ref.shape).astype(np.complex128)
    assert obs.nvis > 4 * 1024
    assert rel_l2(got, ref) <= TOL_GRID
    assert rel_l2(v_def.reshape(ref.shape).astype(np.complex128), ref) <= TOL_GRID
    # records per 16 x 16 centre tile: some tiles need more than one chunk
    ok = (idx["flags"] & 1) != 0
    tiles = (idx["kv"][ok] // 16) * (N // 16) + idx["ku"][ok] // 16
    assert np.bincount(tiles).max() > 1024


def test_adjoint_dot_gpu(gw):
    obs = CASES["small-w"]()
    rng = np.random.default_rng(3)
    N = obs.grid_n
    y = (rng.normal(size=(obs.npol, N, N)) + 1j * rng.normal(size=(obs.npol, N, N)))
    y = y.astype(np.complex64)
    with gw.Plan.from_observation(obs) as plan:
        gx = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)).cpu().numpy()
        ghy = plan.degrid(dev(obs.uvw_m), dev(obs.freq_hz), dev(y)).cpu().numpy()
    lhs = np.vdot(y.astype(np.complex128), gx.astype(np.complex128))
    rhs = np.vdot(ghy.astype(np.complex128), obs.vis.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


# ---------------------------------------------------------------------------
# correction + shift
# ---------------------------------------------------------------------------

def test_correction_pipeline_matches_oracle(gw):
    """shift -> unnormalised inverse FFT -> correct(+1) equals the oracle's
    centred IDFT x h(m) h(l).  The corrector grows towards the field edge
    (h^2 ~ 1e7 in the corners for S_min = 7), amplifying FP32 FFT rounding
    there, so the corrected image is compared over the central half (where
    the thesis evaluates images) and the uncorrected transform everywhere."""
    obs = CASES["small-w"]()
    prm = Params(**obs.plan_kwargs())
    orc = oracle_for(prm)
    ref_grid = orc.grid(obs.uvw_m, obs.freq_hz, obs.vis)
    ref_raw = centred_idft(ref_grid)
    ref_img = correct(ref_raw, corrector(prm))
    N = prm.grid_n
    c = slice(N // 4, 3 * N // 4)
    with gw.Plan.from_observation(obs) as plan:
        g = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis))
        plan.shift(g)
        img = torch.fft.ifft2(g, norm="forward")      # unnormalised inverse FFT
        raw = img.clone()
        plan.correct(img, direction=+1)
        got = img.cpu().numpy().astype(np.complex128)
        rawn = raw.cpu().numpy().astype(np.complex128)
    ii = np.arange(N)
    checker = np.where((ii[:, None] + ii[None, :]) % 2 == 1, -1.0, 1.0)
    assert rel_l2(rawn * checker, ref_raw) <= 2e-5
    assert rel_l2(got[:, c, c], ref_img[:, c, c]) <= 2e-5
    # direction 0: correction only
    x = (np.arange(prm.npol * N ** 2).reshape(prm.npol, N, N) % 7 + 1j).astype(np.complex64)
    with gw.Plan.from_observation(obs) as plan:
        t = dev(x)
        plan.correct(t, direction=0)
        h = corrector(prm)
        assert rel_l2(t.cpu().numpy(), x * (h[:, None] * h[None, :])) <= 1e-6


def test_w0_kernel_is_exactly_real(gw):
    """2-D plans grid with a real kernel (padded tables of real parts, no
    imaginary-part FMAs): that rests on the w = 0 kernel's imaginary parts
    being exactly zero, which the w-screen of zero phase gives.  The binned
    gridder on that path matches the oracle for 1 and 4 polarisations."""
    for npol in (1, 4):
        obs = syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=npol, grid_n=128, s_min=7,
                             s_max=7, n_w=1, diameter_m=1500.0, seed=31)
        prm = Params(**obs.plan_kwargs())
        ref = oracle_for(prm).grid(obs.uvw_m, obs.freq_hz, obs.vis)
        with gw.Plan.from_observation(obs) as plan:
            t, _, _ = plan.tables()
            assert np.all(t.imag == 0)
            plan.set_tuning(grid_kernel=1)
            g = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis)).cpu().numpy()
        assert rel_l2(g.astype(np.complex128), ref) <= TOL_GRID, npol


def test_launch_count_increases(gw):
    obs = CASES["2d"]()
    before = gw.launch_count()
    with gw.Plan.from_observation(obs) as plan:
        plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis))
    assert gw.launch_count() > before


def test_grid_from_host_inputs_matches_device_inputs(gw):
    """gw_grid_vis_host (pipelined host-to-device copies) gives the grid of
    gw_grid_vis on the same data, with and without weights, for ragged steps."""
    obs = CASES["small-w"]()
    wt = syn.random_weights(obs)
    for nrow in (obs.nrow, 3, 1):
        uvw, vis, w = obs.uvw_m[:nrow], obs.vis[:nrow], wt[:nrow]
        with gw.Plan.from_observation(obs, max_vis_per_call=7 * obs.nchan) as plan:
            ref, dref = plan.grid(dev(uvw), dev(obs.freq_hz), dev(vis), weight=dev(w),
                                  return_dropped=True)
            hu = torch.from_numpy(np.ascontiguousarray(uvw)).pin_memory()
            hf = torch.from_numpy(obs.freq_hz).pin_memory()
            hv = torch.from_numpy(np.ascontiguousarray(vis)).pin_memory()
            hw = torch.from_numpy(np.ascontiguousarray(w)).pin_memory()
            got, dgot = plan.grid_host(hu, hf, hv, weight=hw, return_dropped=True)
            got2 = plan.grid_host(hu, hf, hv)
            ref2 = plan.grid(dev(uvw), dev(obs.freq_hz), dev(vis))
        assert dgot == dref
        a, b = got.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)
        assert rel_l2(a, b) <= 1e-6
        a, b = got2.cpu().numpy().astype(np.complex128), ref2.cpu().numpy().astype(np.complex128)
        assert rel_l2(a, b) <= 1e-6


def test_ffma_peak_probe(gw):
    """The FP32 FMA probe runs and lands near the nominal peak (152 SMs x 128
    FMA/clk x 2 FLOP x clock: 80.5 TFLOP/s at 2.07 GHz)."""
    t = gw.ffma_peak(2048)
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    assert 0.3 * nominal <= t <= 1.1 * nominal
