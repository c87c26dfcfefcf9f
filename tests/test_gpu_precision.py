"""Mixed-precision storage on the GPU: bfloat16 / float16 kernel tables and
visibilities with FP32 sums, and compensated (TwoSum) grid commits.

Every result is checked twice against the FP64 oracle:

* parity -- the oracle run on exactly the values the 16-bit storage holds
  (tables and visibilities rounded as stored, oracle/precision.py): the
  CUDA path differs only by FP32 arithmetic, relative L2 <= 1e-5 (for
  16-bit degridded output, elementwise within the output's own rounding);
* storage error -- the oracle on the unrounded FP64 tables and FP32
  visibilities: relative L2 <= 5e-3 for bfloat16 storage and <= 1e-3 for
  float16 storage (measured values are printed).
"""
import json
import os

import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.cgrid import Oracle
from oracle.precision import BF16, F16, QuantisedTables
from oracle.wkernel import KernelTables, Params

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
TOL_PARITY = 1e-5
TOL_STORAGE = {"bf16": 5e-3, "f16": 1e-3}
UNIT = {"bf16": 2.0**-8, "f16": 2.0**-11}     # unit roundoff of each format


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


def report(name, **vals):
    """Print measured errors; also append them to $GW_REPORT_DIR/precision.jsonl if set."""
    print(name, json.dumps(vals))
    d = os.environ.get("GW_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "precision.jsonl"), "a") as f:
            f.write(json.dumps({"case": name, **vals}) + "\n")


def small():
    return syn.small_case(n_ant=7, n_times=10, n_chan=3, npol=4, grid_n=128, s_min=7,
                          s_max=21, n_w=5, diameter_m=1500.0)


_TABLES = {}


def tables_for(prm):
    if prm not in _TABLES:
        _TABLES[prm] = KernelTables(prm)
    return _TABLES[prm]


def oracle(prm, kind):
    kt = tables_for(prm)
    return Oracle(prm, kt if kind == "c64" else QuantisedTables(kt, kind))


def stored_vis(gw, vis, kind, want_held=True):
    """Host complex64 visibilities -> device tensor in the storage of ``kind``
    (torch rounds binary32 to 16-bit to nearest even) and the complex128 values held."""
    from paper_2111_04141_gb300.plan import from_storage, to_storage
    t = to_storage(torch.from_numpy(np.ascontiguousarray(vis)), kind)
    held = from_storage(t).numpy().astype(np.complex128) if want_held else None
    return t.to(DEV), held


# ---------------------------------------------------------------------------
# stored tables
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["bf16", "f16"])
def test_stored_tables_are_the_rounded_fp64_tables(gw, kind):
    obs = small()
    prm = Params(**obs.plan_kwargs())
    qt = QuantisedTables(tables_for(prm), kind)
    with gw.Plan.from_observation(obs, table_dtype=kind) as plan:
        assert plan.info.table_exp2 == qt.exp2
        raw = plan.stored_tables()
    flat, _ = qt.flat()
    want = np.stack([np.ldexp(flat.real, qt.exp2), np.ldexp(flat.imag, qt.exp2)], 1)
    if kind == "f16":
        got = raw.view(np.float16).astype(np.float64)
    else:
        got = (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    # the GPU rounds its own FP64 table (its quadrature differs from the
    # oracle's at ~1e-13 of the peak), so a rounding decision may rarely land
    # one unit in the last place apart, and entries at that noise level (the
    # imaginary part of the w = 0 plane is 0 on the GPU, ~1e-19 in the
    # oracle) may differ; everything else is identical
    p, emin, _ = F16 if kind == "f16" else BF16
    _, e = np.frexp(np.maximum(np.abs(got), np.abs(want)))
    ulp = np.ldexp(1.0, np.maximum(e - p, emin - p + 1))
    noise = 1e-12 * np.abs(want).max()
    assert np.all(np.abs(got - want) <= ulp + noise), kind
    big = np.abs(want) > noise
    assert np.mean(got[big] == want[big]) >= 0.9999, kind


# ---------------------------------------------------------------------------
# gridding / degridding with 16-bit storage
# ---------------------------------------------------------------------------

COMBOS = [("bf16", "bf16"), ("f16", "f16"), ("bf16", "c64"), ("c64", "bf16"), ("f16", "c64")]


@pytest.mark.parametrize("kernel", [1, 2], ids=["binned", "direct"])
@pytest.mark.parametrize("table_kind,vis_kind", COMBOS)
def test_grid_16bit_parity_and_storage_error(gw, table_kind, vis_kind, kernel):
    obs = small()
    prm = Params(**obs.plan_kwargs())
    vt, held = stored_vis(gw, obs.vis, vis_kind)
    ref_q = oracle(prm, table_kind).grid(obs.uvw_m, obs.freq_hz, held)
    exact = Oracle(prm, tables_for(prm)).grid(obs.uvw_m, obs.freq_hz, obs.vis)
    with gw.Plan.from_observation(obs, table_dtype=table_kind, vis_dtype=vis_kind) as plan:
        plan.set_tuning(grid_kernel=kernel)
        g = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), vt)
    got = g.cpu().numpy().astype(np.complex128)
    parity = rel_l2(got, ref_q)
    storage = rel_l2(got, exact)
    report(f"grid table={table_kind} vis={vis_kind}", parity=parity, storage_error=storage)
    assert parity <= TOL_PARITY
    worst = max(TOL_STORAGE.get(table_kind, 0), TOL_STORAGE.get(vis_kind, 0))
    assert storage <= worst


@pytest.mark.parametrize("table_kind,vis_kind", COMBOS)
def test_degrid_16bit_parity_and_storage_error(gw, table_kind, vis_kind):
    obs = small()
    prm = Params(**obs.plan_kwargs())
    rng = np.random.default_rng(5)
    N = prm.grid_n
    grid = (rng.normal(size=(prm.npol, N, N)) + 1j * rng.normal(size=(prm.npol, N, N)))
    grid = grid.astype(np.complex64)
    ref_q = oracle(prm, table_kind).degrid(obs.uvw_m, obs.freq_hz, grid.astype(np.complex128))
    exact = Oracle(prm, tables_for(prm)).degrid(obs.uvw_m, obs.freq_hz,
                                                 grid.astype(np.complex128))
    from paper_2111_04141_gb300.plan import from_storage
    with gw.Plan.from_observation(obs, table_dtype=table_kind, vis_dtype=vis_kind) as plan:
        v = plan.degrid(dev(obs.uvw_m), dev(obs.freq_hz), dev(grid))
        vs = plan.degrid_static(dev(obs.uvw_m), dev(obs.freq_hz), dev(grid))
    got = from_storage(v.cpu()).numpy().reshape(ref_q.shape).astype(np.complex128)
    got_s = from_storage(vs.cpu()).numpy().reshape(ref_q.shape).astype(np.complex128)
    if vis_kind == "c64":
        assert rel_l2(got, ref_q) <= TOL_PARITY
        assert rel_l2(got_s, ref_q) <= TOL_PARITY
    else:
        # FP32 sum rounded once to the output format
        rms = np.sqrt(np.mean(np.abs(ref_q) ** 2))
        for z in (got, got_s):
            for part in (np.real, np.imag):
                err = np.abs(part(z) - part(ref_q))
                assert np.all(err <= 2 * UNIT[vis_kind] * np.abs(part(ref_q)) + 1e-5 * rms)
    storage = rel_l2(got, exact)
    report(f"degrid table={table_kind} vis={vis_kind}", storage_error=storage,
           parity=rel_l2(got, ref_q))
    worst = max(TOL_STORAGE.get(table_kind, 0), TOL_STORAGE.get(vis_kind, 0))
    assert storage <= worst


def test_16bit_vis_with_weights(gw):
    obs = small()
    prm = Params(**obs.plan_kwargs())
    wt = syn.random_weights(obs)
    vt, held = stored_vis(gw, obs.vis, "bf16")
    ref_q = oracle(prm, "bf16").grid(obs.uvw_m, obs.freq_hz, held, weight=wt)
    with gw.Plan.from_observation(obs, table_dtype="bf16", vis_dtype="bf16",
                                  max_vis_per_call=41 * obs.nchan) as plan:
        g = plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), vt, weight=dev(wt))
    assert rel_l2(g.cpu().numpy().astype(np.complex128), ref_q) <= TOL_PARITY


# ---------------------------------------------------------------------------
# compensated commits
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", [1, 2], ids=["binned", "direct"])
def test_compensated_grid_matches_oracle(gw, kernel):
    obs = small()
    prm = Params(**obs.plan_kwargs())
    exact = Oracle(prm, tables_for(prm)).grid(obs.uvw_m, obs.freq_hz, obs.vis)
    with gw.Plan.from_observation(obs, max_vis_per_call=29 * obs.nchan) as plan:
        plan.set_tuning(grid_kernel=kernel)
        g = plan.new_grid()
        e = plan.new_grid()
        plan.grid(dev(obs.uvw_m), dev(obs.freq_hz), dev(obs.vis), out=g, err=e)
        plan.fold(g, e)
        assert not torch.any(e != 0)
    assert rel_l2(g.cpu().numpy().astype(np.complex128), exact) <= TOL_PARITY


def test_compensated_commits_recover_the_exact_sum(gw):
    """Records far apart (one record per grid point) gridded M times into one
    grid: every call commits the same FP32 value c to each point, so the
    exact sum is M c.  Plain FP32 commits drift from it by many ulps; with
    compensation grid + err (summed in FP64) equals M c to ~1e-12."""
    N, M = 512, 600
    prm = dict(grid_n=N, cell_rad=1.0 / N, support_min=7, support_max=7, oversample=8,
               n_wplanes=1, w_max_lambda=0.0, npol=1)
    rng = np.random.default_rng(8)
    # 12 x 12 records on a lattice with 32-pixel spacing (no footprint overlap)
    k = np.arange(-6, 6) * 32 + 0.3
    uu, vv = np.meshgrid(k, k)
    uvw = np.stack([uu.ravel(), vv.ravel(), np.zeros(uu.size)], 1)   # metres = wavelengths at c0
    freq = np.array([299792458.0])
    vis = (rng.normal(size=(uu.size, 1, 1)) + 1j * rng.normal(size=(uu.size, 1, 1)))
    vis = vis.astype(np.complex64)
    with gw.Plan(**prm) as plan:
        plan.set_tuning(grid_kernel=1)      # the binned kernel's per-item commits
        u, f, v = dev(uvw), dev(freq), dev(vis)
        one = plan.grid(u, f, v).cpu().numpy().astype(np.complex128)
        plain = plan.new_grid()
        g = plan.new_grid()
        e = plan.new_grid()
        for _ in range(M):
            plan.grid(u, f, v, out=plain)
            plan.grid(u, f, v, out=g, err=e)
        plain = plain.cpu().numpy().astype(np.complex128)
        comp = g.cpu().numpy().astype(np.complex128) + e.cpu().numpy().astype(np.complex128)
        plan.fold(g, e)
        folded = g.cpu().numpy().astype(np.complex128)
    want = M * one
    nz = np.abs(want) > 0
    rel = lambda x: np.max(np.abs(x[nz] - want[nz]) / np.abs(want[nz]))
    report("compensated exact-sum", plain_max_rel=rel(plain), comp_max_rel=rel(comp),
           folded_max_rel=rel(folded))
    assert rel(comp) <= 1e-11
    assert rel(plain) >= 100 * max(rel(comp), 1e-16)
    assert rel(folded) <= 2.0**-23          # one FP32 rounding of the compensated sum


# ---------------------------------------------------------------------------
# mixed precision at scale: 256 antennas, 8192^2 x 4, 128 w-planes, S <= 127
# ---------------------------------------------------------------------------

def test_precision_at_scale(gw):
    """All 133.7M visibilities: 16-bit paths against the (compensated) FP32
    path; a 1/256 row subsample against the FP64 oracle (exact and
    storage-rounded), for gridding and degridding."""
    full = syn.config_precision()
    kw = full.plan_kwargs()
    prm = Params(**kw)
    u, f = dev(full.uvw_m), dev(full.freq_hz)
    grids = {}
    with gw.Plan(**kw) as p32:
        g, e = p32.new_grid(), p32.new_grid()
        p32.grid(u, f, dev(full.vis), out=g, err=e)
        p32.fold(g, e)
        del e
        grids["c64"] = g
    for kind in ("bf16", "f16"):
        vt, _ = stored_vis(gw, full.vis, kind, want_held=False)
        with gw.Plan(**kw, table_dtype=kind, vis_dtype=kind) as p:
            grids[kind] = p.grid(u, f, vt)
        del vt
    vs_fp32 = {k: float(torch.linalg.vector_norm(grids[k] - grids["c64"]) /
                        torch.linalg.vector_norm(grids["c64"])) for k in ("bf16", "f16")}
    del grids, u, f
    torch.cuda.empty_cache()

    rows = np.arange(0, full.nrow, 256)
    uvw, freq = full.uvw_m[rows], full.freq_hz
    vis = full.vis[rows]
    del full
    kt = tables_for(prm)
    exact = Oracle(prm, kt)
    ref = exact.grid(uvw, freq, vis)
    rng = np.random.default_rng(9)
    model = (rng.normal(size=ref.shape) + 1j * rng.normal(size=ref.shape)).astype(np.complex64)
    model64 = model.astype(np.complex128)
    ref_v = exact.degrid(uvw, freq, model64)
    out = {"sample_rows": int(rows.size), "sample_vis": int(rows.size * freq.size)}
    from paper_2111_04141_gb300.plan import from_storage
    for kind in ("c64", "bf16", "f16"):
        vt, held = stored_vis(gw, vis, kind)
        orc = exact if kind == "c64" else Oracle(prm, QuantisedTables(kt, kind))
        ref_q = orc.grid(uvw, freq, held)
        with gw.Plan(**kw, table_dtype=kind, vis_dtype=kind) as p:
            g = p.grid(dev(uvw), dev(freq), vt).cpu().numpy().astype(np.complex128)
            dv = p.degrid(dev(uvw), dev(freq), dev(model))
        dv = from_storage(dv.cpu()).numpy().reshape(ref_v.shape).astype(np.complex128)
        ref_vq = orc.degrid(uvw, freq, model64)
        out[kind] = dict(grid_parity=rel_l2(g, ref_q), grid_vs_fp64=rel_l2(g, ref),
                         degrid_parity=rel_l2(dv, ref_vq), degrid_vs_fp64=rel_l2(dv, ref_v))
        del ref_q, orc
    out["grid_vs_fp32_path_all_vis"] = vs_fp32
    report("precision-8192-P128-S7to127-4pol", **out)
    assert out["c64"]["grid_vs_fp64"] <= TOL_PARITY
    assert out["c64"]["degrid_vs_fp64"] <= TOL_PARITY
    for kind in ("bf16", "f16"):
        assert out[kind]["grid_parity"] <= TOL_PARITY
        assert out[kind]["grid_vs_fp64"] <= TOL_STORAGE[kind]
        assert out[kind]["degrid_vs_fp64"] <= TOL_STORAGE[kind]
        assert vs_fp32[kind] <= TOL_STORAGE[kind]
