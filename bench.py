#!/usr/bin/env python
"""Benchmark: 4-pol W-projection gridding rate on GB300.

A step is one call of the gridding path on one batch of synthetic input:
index selection, device binning and the gridding kernel (the kernel tables
are built once per plan, as the thesis generates its GCF table once).
Workload: 64 antennas in a 5 km disk, 256 times x 16 channels (120-180 MHz)
= 8,257,536 visibilities x 4 pols; 4096^2 x 4 grid, 32 w-planes, support
7 -> 63, oversampling 8.  Inputs (vis 264 MB, grid 512 MB) exceed the
129 MB L2, so no explicit flush is done between steps.

value = grid-point polarisation updates per second (sum over visibilities of
S_p^2 x npol, divided by the device time of the step), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank grids its own batch (seeded by rank) into its own
grid; the grids are summed once (NCCL all-reduce) inside the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gridding rate (grid-point updates/s), 4-pol W-proj; p50/p99 request latency"
UNIT = "grid-point pol-updates/s"
FLOP_PER_UPDATE = 8           # complex x complex multiply-accumulate = 4 FFMA
SM_MAX_MHZ_DEFAULT = 2070.0
FFMA_PER_SM_PER_CLK = 128

# DRAM traffic of the gridding kernel from one ncu capture, valid only for the
# kernel source it was taken on (sha256 of gw_grid_kernel.cuh); null otherwise.
GRID_TRAFFIC = {"sha256": "1ee91684f8fa3ecd5a1cc714157b1691bdf3c0bbce0a8d1c95030106c9a3d36f",
                "bytes_per_launch": 0.964303e9 + 0.264140e9,
                "capture": "profiles/k_grid_wproj4096.md"}


# The thesis' own best gridding rate, context only (a different workload on
# other hardware, so no vs_baseline): Section 4's maximum-performance
# experiment, 4 polarisations.
PAPER_CONTEXT = {
    "value": 3.62e9 * 36 * 4, "unit": "grid-point pol-updates/s",
    "hardware": "Tesla P100-SXM2 at 1480 MHz, FP32",
    "workload": "real 6x6 prolate-spheroidal kernel, no w-term, every record on one pixel "
                "(3.62 GRecs/s at 4 pols, 19.7 % of the P100 FP32 peak)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # steps of the end-to-end loop: the last step's result copy is not
    # overlapped, so more steps approach the streaming steady state
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-stream measurement")
    ap.add_argument("--serving-jobs", type=int, default=256)
    ap.add_argument("--no-variants", action="store_true",
                    help="skip compression, hybrid gridding and w-stacking measurements")
    ap.add_argument("--no-imaging", action="store_true",
                    help="skip the dirty-image pipeline and R(X) measurements")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the 16-bit-storage and compensated-commit measurements")
    ap.add_argument("--no-c5", action="store_true",
                    help="skip the 8192^2, 128-plane (C5) storage-precision timing")
    ap.add_argument("--cpu-sample-rows", type=int, default=0,
                    help="rows of the workload in the CPU-baseline sample (0 = half of the rows, about 8 s of oracle work on 16 cores)")
    ap.add_argument("--times", type=int, default=256,
                    help="time steps of the workload (256 = the full workload)")
    ap.add_argument("--profile-only", nargs="?", const="grid", default=None,
                    choices=["grid", "degrid", "hybrid"],
                    help="plan + warm-up + one gridding (or degridding) call, no timing or "
                         "JSON (for ncu)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def kernel_sha(name="gw_grid_kernel.cuh"):
    p = os.path.join(ROOT, "paper_2111_04141_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7],
                                 swp=f[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(obs, rows, rows_single):
    """The FP64 oracle on bounded samples of the workload (host cores): the
    same stages as the GPU step, index selection and gridding, timed
    together; all host threads on `rows` rows, one thread on `rows_single`."""
    import numpy as np
    from oracle.cgrid import Oracle, default_threads
    from oracle.wkernel import Params, plane_support
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    S = plane_support(prm)

    def timed(nr, th):
        sub = slice(0, nr)
        t0 = time.perf_counter()
        idx = orc.index(obs.uvw_m[sub], obs.freq_hz)
        orc.grid(obs.uvw_m[sub], obs.freq_hz, obs.vis[sub], idx=idx, nthreads=th)
        dt = time.perf_counter() - t0
        taps = int(np.sum(S[idx["plane"]][idx["valid"]] ** 2))
        return taps * prm.npol / dt, dt

    th = default_threads()
    v, dt = timed(rows, th)
    v1, dt1 = timed(rows_single, 1)
    return {"value": v, "threads": th, "seconds": dt, "single_thread_value": v1,
            "single_thread_seconds": dt1, "single_thread_rows": rows_single}


def run_reference(args, world, rank):
    if rank != 0:
        return
    import numpy as np
    import synthetic as syn
    from oracle.cgrid import Oracle, default_threads
    from oracle.wkernel import Params, plane_support
    obs = syn.config_wproj()
    prm = Params(**obs.plan_kwargs())
    orc = Oracle(prm)
    rows = obs.nrow // 64
    S = plane_support(prm)
    th = default_threads()
    times, taps_tot = [], 0
    for step in range(args.warmup + args.steps):
        r0 = (step * rows) % (obs.nrow - rows)
        sub = slice(r0, r0 + rows)
        # the GPU step's stages: index selection, then gridding
        t0 = time.perf_counter()
        idx = orc.index(obs.uvw_m[sub], obs.freq_hz)
        orc.grid(obs.uvw_m[sub], obs.freq_hz, obs.vis[sub], idx=idx, nthreads=th)
        dt = time.perf_counter() - t0
        taps = int(np.sum(S[idx["plane"]][idx["valid"]] ** 2))
        if step >= args.warmup:
            times.append(dt)
            taps_tot += taps
    value = taps_tot * prm.npol / sum(times)
    sample = (f"{rows} consecutive rows (1/64 of the workload's rows, all 16 channels) per step, "
              f"FP64 oracle index selection (numpy) + gridding (C, {th} threads)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": obs.name, "rows_per_step": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "threads": th,
                         "kind": "oracle", "includes": "index+grid", "cpu_model": cpu_model(),
                         "nproc": os.cpu_count(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def measure_precision(gw, plan, obs, uvw, freq, vis, dev, stream, steps):
    """Gridding rate and error of each storage variant on the same batch:
    bfloat16 / float16 tables + visibilities (FP32 sums), and FP32 with
    compensated commits.  Errors are relative L2 against the plain FP32 grid
    of the batch (the FP64-oracle errors are measured by the test suite)."""
    import torch
    from paper_2111_04141_gb300.plan import to_storage
    ref = plan.grid(uvw, freq, vis)
    nref = torch.linalg.vector_norm(ref)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"error_basis": "relative L2 vs the FP32 grid of the same batch"}

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    plan.timing(True)
    plan.timing()
    for kind in ("bf16", "f16"):
        p2 = gw.Plan.from_observation(obs, table_dtype=kind, vis_dtype=kind)
        v2 = to_storage(vis, kind)
        g2 = p2.new_grid()
        p2.timing(True)
        ms = timed(lambda: p2.grid(uvw, freq, v2, out=g2))
        tm = p2.timing()
        one = p2.grid(uvw, freq, v2)
        taps = tm["taps"] / max(1, tm["grid_calls"])
        out[kind] = {"value": taps * obs.npol / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "grid_kernel_ms": tm["grid_ms"] / max(1, tm["grid_calls"]),
                     "rel_l2_vs_fp32": float(torch.linalg.vector_norm(one - ref) / nref),
                     "vis_bytes": v2.numel() * v2.element_size()}
        p2.close()
        del v2, g2, one
    g, e = plan.new_grid(), plan.new_grid()
    plan.timing()
    ms = timed(lambda: plan.grid(uvw, freq, vis, out=g, err=e))
    tm = plan.timing()
    plan.timing(False)
    g.zero_()
    e.zero_()
    plan.grid(uvw, freq, vis, out=g, err=e)
    plan.fold(g, e)
    taps = tm["taps"] / max(1, tm["grid_calls"])
    out["c64_compensated"] = {"value": taps * obs.npol / (ms * 1e-3), "unit": UNIT,
                              "ms_per_step": ms,
                              "grid_kernel_ms": tm["grid_ms"] / max(1, tm["grid_calls"]),
                              "rel_l2_vs_fp32": float(torch.linalg.vector_norm(g - ref) / nref)}
    return out


def measure_imaging(gw, plan, obs, uvw, freq, vis, dev, stream, steps):
    """Dirty image of the batch (grid, shift, cuFFT inverse transform, correct,
    normalise) and the aliasing experiment R(X) = |1 - K(X)| (unit point source
    at pixel (X, X), X = 0..63, 128^2 image, support 7, oversampling 128)."""
    import numpy as np
    import torch
    import synthetic as syn
    from paper_2111_04141_gb300.imaging import dirty_image
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dirty_image(plan, uvw, freq, vis)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        dirty_image(plan, uvw, freq, vis)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    # R(X): point-source visibilities from the measurement equation in FP64
    N = 128
    o2 = syn.config_2d()
    cell = syn.fit_cell(o2.uvw_m, o2.freq_hz, N, 7)
    lam = (o2.uvw_m[:, None, :] * o2.freq_hz[None, :, None] / 299792458.0).reshape(-1, 3)
    r = []
    with gw.Plan(grid_n=N, cell_rad=cell, support_min=7, support_max=7, oversample=128,
                 n_wplanes=1, npol=1) as p2:
        u2, f2 = torch.from_numpy(o2.uvw_m).to(dev), torch.from_numpy(o2.freq_hz).to(dev)
        for x in range(64):
            v = np.exp(-2j * np.pi * (lam[:, 0] + lam[:, 1]) * (x * cell))
            img = dirty_image(p2, u2, f2, torch.from_numpy(
                v.reshape(o2.nrow, o2.nchan, 1).astype(np.complex64)).to(dev))
            r.append(abs(1.0 - float(img[0, N // 2 + x, N // 2 + x].real)))
    r = np.array(r)
    return {"dirty_image_ms": ms, "images_per_s": 1e3 / ms,
            "steps": "grid + shift + inverse FFT (cuFFT) + correct + normalise, "
                     f"{obs.grid_n}^2 x {obs.npol}",
            "R_X": {"max_X_le_32": float(r[:33].max()), "max_all": float(r.max()),
                    "X": list(range(64)), "R": [float(t) for t in r],
                    "setup": "16 antennas, 3,840 vis, 128^2, support 7, oversampling 128"}}


def grid_roofline(tm, calls, npol, peak):
    """FP32-FMA roofline of the gridding kernel from a plan's stage timing."""
    ms = tm["grid_ms"] / max(1, tm["grid_calls"])
    flop = tm["taps"] / max(1, calls) * npol * FLOP_PER_UPDATE / max(1, tm["grid_calls"] / calls)
    tf = flop / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel_ms": ms, "achieved": tf, "peak": peak, "unit": "TFLOP/s",
            "frac": tf / peak}


def measure_c5(gw, dev, stream, steps, peak):
    """The 8192^2 x 4, 128-plane, support 7->127 workload (133.7M visibilities
    x 4 pols; tables far larger than L2): one gridding step (index, bin, grid)
    with FP32 storage and with bfloat16 / float16 tables and visibilities.
    Visibilities are CN(0, 1) drawn on the device (seeded); uvw, channels and
    imaging parameters come from the synthetic generator."""
    import torch
    import synthetic as syn
    from paper_2111_04141_gb300.plan import to_storage
    obs = syn.config_precision(with_vis=False)
    uvw = torch.from_numpy(obs.uvw_m).to(dev)
    freq = torch.from_numpy(obs.freq_hz).to(dev)
    gen = torch.Generator(device=dev).manual_seed(20211108)
    vis = torch.randn((obs.nrow, obs.nchan, obs.npol), dtype=torch.complex64, device=dev,
                      generator=gen)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": obs.name, "nvis": obs.nvis, "npol": obs.npol, "grid_n": obs.grid_n,
           "n_wplanes": obs.n_wplanes, "support": f"{obs.support_min}->{obs.support_max}",
           "vis": "CN(0,1) drawn on the device (torch, seeded)"}
    for kind in ("c64", "bf16", "f16"):
        with gw.Plan.from_observation(obs, table_dtype=kind, vis_dtype=kind) as p:
            v = vis if kind == "c64" else to_storage(vis, kind)
            g = p.new_grid()
            p.grid(uvw, freq, v, out=g)
            torch.cuda.synchronize(dev)
            p.timing(True)
            p.timing()
            e0.record(stream)
            for _ in range(steps):
                p.grid(uvw, freq, v, out=g)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            tm = p.timing()
            info = p.info
            out[kind] = {"value": tm["taps"] / steps * obs.npol / (ms * 1e-3), "unit": UNIT,
                         "ms_per_step": ms, "roofline": grid_roofline(tm, steps, obs.npol, peak),
                         "stage_ms_per_step": {k: tm[f"{k}_ms"] / steps
                                               for k in ("index", "bin", "grid")},
                         "table_bytes": int(info.table_bytes),
                         "plane_groups": int(info.plane_groups),
                         "mean_S2": tm["taps"] / max(1, tm["valid_vis"])}
            del g
            if kind != "c64":
                del v
        torch.cuda.empty_cache()
    return out


def measure_c1(gw, dev, stream, steps, peak):
    """The 2-D workload (16 antennas, 3,840 visibilities, 256^2, support 7,
    1 pol): one gridding step; small enough to be bound by launches."""
    import torch
    import synthetic as syn
    obs = syn.config_2d()
    uvw = torch.from_numpy(obs.uvw_m).to(dev)
    freq = torch.from_numpy(obs.freq_hz).to(dev)
    vis = torch.from_numpy(obs.vis).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with gw.Plan.from_observation(obs) as p:
        g = p.new_grid()
        for _ in range(3):
            p.grid(uvw, freq, vis, out=g)
        torch.cuda.synchronize(dev)
        p.timing(True)
        p.timing()
        e0.record(stream)
        for _ in range(steps):
            p.grid(uvw, freq, vis, out=g)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        tm = p.timing()
    return {"workload": obs.name, "nvis": obs.nvis, "value": tm["taps"] / steps * obs.npol /
            (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "roofline": grid_roofline(tm, steps, obs.npol, peak)}


def measure_next(gw, plan, obs, uvw, freq, vis, dev, stream, steps):
    """The batch through the other gridding variants: full compression with
    the w-projection plan; and with a 2-D plan (support 7, the same grid):
    convolutional gridding, Hybrid Gridding (gridding + column pruning,
    pruner support 15) and a 32-layer w-stacked dirty image."""
    import torch
    from paper_2111_04141_gb300.imaging import dirty_image, dirty_image_wstack
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, n=steps):
        fn()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    out = {}
    g = plan.new_grid()
    _, ncomp, _ = plan.grid_compressed(uvw, freq, vis, out=g)
    out["compression"] = {"records_in": obs.nvis, "records_gridded": ncomp,
                          "ratio": obs.nvis / max(ncomp, 1),
                          "ms_per_step": timed(lambda: plan.grid_compressed(uvw, freq, vis,
                                                                            out=g))}
    # with the sampled decision (compress only when >= 5 % of a sample merges)
    tun = plan.get_tuning()
    plan.set_tuning(**dict(tun, compress_min_gain=50))
    _, ncomp2, _ = plan.grid_compressed(uvw, freq, vis, out=g)
    out["compression"]["auto_min_gain_5pct"] = {
        "records_gridded": ncomp2, "compressed": ncomp2 == ncomp,
        "ms_per_step": timed(lambda: plan.grid_compressed(uvw, freq, vis, out=g))}
    plan.set_tuning(**tun)
    kw = dict(obs.plan_kwargs())
    kw.update(support_min=7, support_max=7, n_wplanes=1, w_max_lambda=0.0)
    sz = 15
    with gw.Plan(**kw) as p2:
        g2 = p2.new_grid()
        conv_ms = timed(lambda: p2.grid(uvw, freq, vis, out=g2))
        fine = torch.zeros(p2.fine_shape(), dtype=torch.complex64, device=dev)
        pruned = torch.empty((obs.npol, 2 * obs.grid_n, obs.grid_n), dtype=torch.complex64,
                             device=dev)
        hy_grid_ms = timed(lambda: p2.hybrid_grid(uvw, freq, vis, sz, out=fine))
        hy_prune_ms = timed(lambda: p2.hybrid_prune(sz, fine, out=pruned))
        del fine, pruned
        torch.cuda.empty_cache()
        upd = obs.nvis * obs.npol
        out["2d_support7"] = {
            "convolutional_grid_ms": conv_ms,
            "convolutional_updates_per_s": upd * 49 / (conv_ms * 1e-3),
            "hybrid_grid_ms": hy_grid_ms, "hybrid_prune_ms": hy_prune_ms,
            "hybrid_speedup_grid_only": conv_ms / hy_grid_ms,
            "hybrid_speedup_with_prune": conv_ms / (hy_grid_ms + hy_prune_ms),
            "pruner_support": sz}
        wmax = obs.w_max_lambda
        ws_ms = timed(lambda: dirty_image_wstack(p2, uvw, freq, vis, 32, -wmax, wmax), n=2)
        torch.cuda.empty_cache()
    wp_ms = timed(lambda: dirty_image(plan, uvw, freq, vis), n=2)
    out["wstack_vs_wproj_dirty_image_ms"] = {"wstack_32_layers_support7": ws_ms,
                                             "wproj_32_planes_support7to63": wp_ms}
    return out


def measure_serving(args, dev):
    """Mixed grid/degrid stream (256 jobs, 8 setups with 1024^2-8192^2 grids,
    support 7-63, 1 or 4 pols, 1e4-1e7 visibilities log-uniform, sorted or
    shuffled uvw) at Poisson arrivals of 0.8x the sequential capacity: the
    continuous-batching server against one-at-a-time plain launches."""
    import numpy as np
    import torch
    import synthetic as syn
    from paper_2111_04141_gb300 import hostmem
    from paper_2111_04141_gb300.serve import (Server, build_stream, latency_stats,
                                              run_sequential)
    from paper_2111_04141_gb300.tune import tune_plan
    max_vis = 10_000_000
    n_slots = 4
    specs = syn.serving_setups(n_setups=8, max_vis=max_vis)
    jspecs = syn.serving_jobs(specs, n_jobs=args.serving_jobs, max_vis=max_vis)
    setups, jobs = build_stream(specs, jspecs, np.zeros(len(jspecs)), max_vis)
    gen = torch.Generator(device=dev).manual_seed(17)
    models = {s.name: torch.randn((s.npol, s.grid_n, s.grid_n), dtype=torch.complex64,
                                  device=dev, generator=gen) for s in setups}
    # autotune each setup on a one-million-visibility sample of its own pools
    tuning, tune_ms = {}, {}
    from paper_2111_04141_gb300 import Plan
    for s, d in zip(setups, specs):
        rows = min(d["uvw_sorted"].shape[0], 1_000_000 // s.nchan)
        with Plan(**s.plan_kwargs) as p:
            u = torch.from_numpy(d["uvw_sorted"][:rows]).to(dev)
            f = torch.from_numpy(s.freq_hz).to(dev)
            v = torch.randn((rows, s.nchan, s.npol), dtype=torch.complex64, device=dev,
                            generator=gen)
            res = tune_plan(p, u, f, v, p.new_grid(), reps=2)
        tuning[s.name] = res["tuning"]
        tune_ms[s.name] = res["ms"]
    plain = {s.name: Plan(**s.plan_kwargs) for s in setups}
    # one page-locked arena of result staging (huge pages) for both servers
    # and the sequential loop, which never run at the same time
    n_host = max(max(s.npol * s.grid_n ** 2, -(-max_vis // s.nchan) * s.nchan * s.npol)
                 for s in setups)
    arena = hostmem.PinnedArena(hostmem.arena_bytes([(n_host, torch.complex64)] * n_slots))
    staging = [arena.take(n_host, torch.complex64) for _ in range(n_slots)]

    def reset(js, arrivals):
        for j, t in zip(js, arrivals):
            j.arrival, j.t_admit, j.t_done, j.slot = float(t), float("nan"), float("nan"), -1

    def seq(js, arrivals, srv):
        reset(js, arrivals)
        run_sequential(setups, plain, srv.models, srv.freqs, js, dev, host_buf=staging[0])
        return latency_stats(js)

    def served(js, arrivals, srv):
        reset(js, arrivals)
        srv.run(js)
        return latency_stats(js)

    out = {"jobs": len(jobs), "setups": [s.name for s in setups], "slots": n_slots,
           "graphs": True, "repeats": 3,
           "host_staging": f"{n_slots} x {n_host * 8 / 2**30:.1f} GiB page-locked on huge pages "
                           f"({'yes' if arena.huge else 'no'}), shared by both servers and the "
                           "sequential loop; job pools likewise in one arena"}
    zeros = np.zeros(len(jobs))
    # both servers are built and warmed before any measurement; the modes
    # then alternate within each repeat, so slow drifts hit them alike
    srvs = {}
    for label, tun in (("default", None), ("autotuned", tuning)):
        srvs[label] = Server(setups, dev, budget=96 << 30, n_slots=n_slots, max_vis=max_vis,
                             use_graphs=True, tuning=tun, host_staging=staging)
        srvs[label].warm(models)
    s0 = srvs["default"]
    seq(jobs[:8], zeros[:8], s0)                           # warm-up of the plain path
    cap_seq = seq(jobs, zeros, s0)
    rate = 0.8 * cap_seq["jobs_per_s"]
    arrivals = syn.poisson_arrivals(len(jobs), rate)
    out["arrival_rate_jobs_per_s"] = rate
    out["back_to_back"] = {"sequential": cap_seq}
    runs = {"sequential": [], "server_default": [], "server_autotuned": []}
    for _ in range(out["repeats"]):
        runs["sequential"].append(seq(jobs, arrivals, s0))
        for label, srv in srvs.items():
            runs[f"server_{label}"].append(served(jobs, arrivals, srv))
    out["poisson_0.8x"] = runs
    for label, srv in srvs.items():
        out["back_to_back"][f"server_{label}"] = served(jobs, zeros, srv)
        srv.close()
    for p in plain.values():
        p.close()
    torch.cuda.synchronize(dev)
    arena.release()
    out["tuning"] = tuning
    out["tune_ms"] = tune_ms
    med = lambda runs, k: float(np.median([r[k] for r in runs]))
    modes = ("sequential", "server_default", "server_autotuned")
    out["summary"] = {
        "p99_ms": {m: med(out["poisson_0.8x"][m], "p99_ms") for m in modes},
        "p50_ms": {m: med(out["poisson_0.8x"][m], "p50_ms") for m in modes},
        "back_to_back_jobs_per_s": {k: v["jobs_per_s"] for k, v in out["back_to_back"].items()},
        "basis": ("median over 3 repeats per mode, the modes alternating within each "
                  "repeat; Poisson arrivals at 0.8x the sequential back-to-back rate")}
    return out


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch
    import synthetic as syn
    import paper_2111_04141_gb300 as gw
    from paper_2111_04141_gb300 import build as gwbuild

    gwbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    obs = syn.config_wproj(seed_offset=rank, n_times=args.times)
    plan = gw.Plan.from_observation(obs)
    uvw = torch.from_numpy(obs.uvw_m).to(dev)
    freq = torch.from_numpy(obs.freq_hz).to(dev)
    vis = torch.from_numpy(obs.vis).to(dev)
    grid = plan.new_grid()
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(3, args.warmup)):
        plan.grid(uvw, freq, vis, out=grid)
    torch.cuda.synchronize(dev)
    if args.profile_only:
        if args.profile_only == "hybrid":
            kw = dict(obs.plan_kwargs())
            kw.update(support_min=7, support_max=7, n_wplanes=1, w_max_lambda=0.0)
            with gw.Plan(**kw) as p2:
                for _ in range(2):
                    fine = p2.hybrid_grid(uvw, freq, vis, 15)
                    p2.hybrid_prune(15, fine)
                    del fine
            torch.cuda.synchronize(dev)
            plan.close()
            return
        if args.profile_only == "degrid":
            out_vis = torch.empty_like(vis)
            for _ in range(4):
                plan.degrid(uvw, freq, grid, out=out_vis)
        else:
            plan.grid(uvw, freq, vis, out=grid)
        torch.cuda.synchronize(dev)
        plan.close()
        return
    def optional(enabled, fn):
        """A secondary measurement: its failure is reported in the line
        instead of losing the headline measurement."""
        if not (enabled and world == 1):
            return None
        try:
            return fn()
        except Exception as exc:                      # noqa: BLE001
            torch.cuda.synchronize(dev)
            return {"error": f"{type(exc).__name__}: {exc}"[:300]}
        finally:
            torch.cuda.empty_cache()

    plan.timing(True)
    plan.timing()  # reset counters

    sampler = ClockSampler(local)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    l0 = gw.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.grid(uvw, freq, vis, out=grid)
    if pg:
        pg.all_reduce(grid)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = gw.launch_count() - l0
    t_ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    tm = plan.timing()
    plan.timing(False)
    if pg:
        tt = torch.tensor([t_ms], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_ms = float(tt.item())

    npol = obs.npol
    taps_step = tm["taps"] / args.steps
    updates_step = taps_step * npol
    value = world * updates_step * args.steps / (t_ms * 1e-3)
    grid_ms = tm["grid_ms"] / max(1, tm["grid_calls"])
    flop_launch = updates_step * FLOP_PER_UPDATE / max(1, tm["grid_calls"] / args.steps)
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = (clocks or {}).get("sm_max_mhz") or SM_MAX_MHZ_DEFAULT
    peak = num_sms * FFMA_PER_SM_PER_CLK * 2 * sm_max * 1e6 / 1e12
    achieved = flop_launch / (grid_ms * 1e-3) / 1e12
    traffic = (GRID_TRAFFIC["bytes_per_launch"]
               if GRID_TRAFFIC["sha256"] == kernel_sha() else None)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "kernel": "k_grid (gw_grid_kernel.cuh)",
            "peak_basis": f"FP32 FFMA: {num_sms} SMs x {FFMA_PER_SM_PER_CLK} FFMA/clk x 2 FLOP x "
                          f"{sm_max:.0f} MHz",
            "frac_at_sampled_clock": (achieved / (num_sms * FFMA_PER_SM_PER_CLK * 2 *
                                                  clocks["sm_mhz"] * 1e-6)
                                      if clocks and clocks.get("sm_mhz") else None),
            "stage_ms_per_step": {k: tm[f"{k}_ms"] / args.steps
                                  for k in ("index", "bin", "grid")}}
    # cross-check of the nominal peak: a kernel of independent packed FMAs
    ffma = gw.ffma_peak()
    roof["peak_ffma_measured"] = ffma
    roof["frac_of_measured_ffma"] = achieved / ffma

    # ---- end to end through the public API with host buffers --------------
    pin_uvw = torch.from_numpy(obs.uvw_m).pin_memory()
    pin_freq = torch.from_numpy(obs.freq_hz).pin_memory()
    pin_vis = torch.from_numpy(obs.vis).pin_memory()
    # two result buffers: the device-to-host read of step i overlaps step i+1
    pin_out = [torch.empty(grid.shape, dtype=grid.dtype).pin_memory() for _ in range(2)]
    dgrid = [grid, torch.empty_like(grid)]
    d2h_stream = torch.cuda.Stream(dev)
    done = [torch.cuda.Event() for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    ne = max(1, args.e2e_steps)

    def e2e_step(i):
        # public API from host buffers: gw_grid_vis_host pipelines the
        # host-to-device copies of uvw / vis with the gridding of earlier rows
        b = i % 2
        stream.wait_event(done[b])          # buffer b's previous read has finished
        dgrid[b].zero_()
        plan.grid_host(pin_uvw, pin_freq, pin_vis, out=dgrid[b])
        ready[b].record(stream)
        d2h_stream.wait_event(ready[b])
        with torch.cuda.stream(d2h_stream):
            pin_out[b].copy_(dgrid[b], non_blocking=True)
            done[b].record(d2h_stream)

    for b in range(2):
        done[b].record(stream)
    e2e_step(0)
    e2e_step(1)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for i in range(ne):
        e2e_step(i)
    for b in range(2):
        stream.wait_event(done[b])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / ne
    if pg:
        tt = torch.tensor([e2e_ms], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        e2e_ms = float(tt.item())
    h2d = pin_uvw.numel() * 8 + pin_freq.numel() * 8 + pin_vis.numel() * 8
    d2h = pin_out[0].numel() * 8
    e2e = {"value": world * updates_step / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "ms_per_step": e2e_ms,
           "api": "gw_grid_vis_host (host inputs, copies pipelined with gridding); two result "
                  "grids so that step i's device-to-host read overlaps step i+1"}

    # ---- degridding (the adjoint) on the same batch -------------------------
    out_vis = torch.empty_like(vis)
    plan.degrid(uvw, freq, grid, out=out_vis)
    plan.timing(True)
    plan.timing()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    nd = max(1, min(args.steps, 10))
    for _ in range(nd):
        plan.degrid(uvw, freq, grid, out=out_vis)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dg = plan.timing()
    plan.timing(False)
    dg_ms = e0.elapsed_time(e1) / nd
    degrid = {"value": dg["taps"] / nd * npol / (dg_ms * 1e-3), "unit": UNIT,
              "ms_per_step": dg_ms, "kernel_ms": dg["degrid_ms"] / max(1, dg["degrid_calls"]),
              "achieved_tflops": dg["taps"] / nd * npol * FLOP_PER_UPDATE /
                                 (dg["degrid_ms"] / max(1, dg["degrid_calls"]) * 1e-3) / 1e12}

    # ---- serving stream (after the headline and e2e measurements: its
    # servers pin several GB of host staging memory), then the other
    # measurements on the batch
    serving = optional(not args.no_serving, lambda: measure_serving(args, dev))
    precision = optional(not args.no_precision, lambda: measure_precision(
        gw, plan, obs, uvw, freq, vis, dev, stream, nd))
    imaging = optional(not args.no_imaging, lambda: measure_imaging(
        gw, plan, obs, uvw, freq, vis, dev, stream, nd))
    variants = optional(not args.no_variants, lambda: measure_next(
        gw, plan, obs, uvw, freq, vis, dev, stream, 3))
    c1 = optional(True, lambda: measure_c1(gw, dev, stream, 50, peak))
    c5 = optional(not args.no_c5, lambda: measure_c5(gw, dev, stream, 3, peak))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = args.cpu_sample_rows or obs.nrow // 2
        rows1 = max(1, rows // 8)
        cb = cpu_baseline(obs, rows, rows1)
        cpu = {"value": cb["value"], "unit": UNIT, "cores": cb["threads"],
               "threads": cb["threads"], "kind": "oracle", "includes": "index+grid",
               "cpu_model": cpu_model(), "nproc": os.cpu_count(),
               "single_thread_value": cb["single_thread_value"],
               "sample": f"first {rows} rows (1/{obs.nrow // rows} of the workload, all "
                         f"{obs.nchan} channels): FP64 oracle index selection (numpy) + "
                         f"gridding (C, {cb['threads']} threads), {cb['seconds']:.1f} s; "
                         f"single thread on the first {rows1} rows, "
                         f"{cb['single_thread_seconds']:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": obs.name, "nvis": obs.nvis, "npol": npol,
                       "grid_n": obs.grid_n, "n_wplanes": obs.n_wplanes,
                       "support": f"{obs.support_min}->{obs.support_max}",
                       "oversample": obs.oversample,
                       "valid_vis": int(tm["valid_vis"] / args.steps),
                       "mean_S2": taps_step / max(1, tm["valid_vis"] / args.steps),
                       "vis_per_s": world * tm["valid_vis"] / args.steps * args.steps /
                                    (t_ms * 1e-3),
                       "l2": "inputs larger than L2 (vis 264 MB, grid 512 MB); no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "paper_context": PAPER_CONTEXT,
            "clocks": clocks, "degrid": degrid, "precision": precision, "imaging": imaging,
            "variants": variants, "c1": c1, "c5": c5,
            "serving": serving,
        }
        print(json.dumps(line))
    plan.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
