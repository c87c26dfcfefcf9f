"""Launch autotuner: picks a plan's work-item size and degridding kernel by
timing candidates on a sample job (CUDA events on the launching stream).

The candidates are the plan tunables (gw_tuning): records per work item,
which trades SM load balance on small or sparse jobs against commit
traffic, and the degridding kernel (shared-memory staged tiles or global
gather).  The best configuration is kept in a dict (and, optionally, a JSON
file) keyed by the setup's name or by ``plan_key(plan)``: the plan
parameters the timings depend on and the device's SM count.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional

ITEM_CANDIDATES = (256, 512, 1024, 2048, 4096)
DEGRID_CANDIDATES = (1, 2)


def _time(fn, stream, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune_plan(plan, uvw, freq, vis, grid, reps: int = 3,
              items: Iterable[int] = ITEM_CANDIDATES,
              degrid: Iterable[int] = DEGRID_CANDIDATES) -> dict:
    """Time gridding + degridding of one sample (device tensors) for each
    candidate; leaves the best tuning set on ``plan`` and returns it with
    the timings (ms)."""
    import torch
    stream = torch.cuda.current_stream(plan.device)
    out_vis = torch.empty_like(vis)
    timings = {}
    best, best_ms = None, float("inf")
    for im in items:
        for dk in degrid:
            plan.set_tuning(item_max=im, degrid_kernel=dk)

            def step():
                plan.grid(uvw, freq, vis, out=grid)
                plan.degrid(uvw, freq, grid, out=out_vis)

            ms = _time(step, stream, reps)
            timings[f"item_max={im},degrid_kernel={dk}"] = ms
            if ms < best_ms:
                best, best_ms = {"item_max": im, "degrid_kernel": dk, "grid_kernel": 0,
                                  "compress_min_gain": 0, "plane_groups": 0}, ms
    plan.set_tuning(**best)
    return {"tuning": best, "ms": best_ms, "timings": timings}


def plan_key(plan, num_sms: Optional[int] = None) -> str:
    """Cache key of a plan's tuning: grid size, support range, oversampling,
    w-planes, polarisations, storage kinds and the SM count of its device
    (a tuning found on another GPU or for other plan parameters is not
    reused)."""
    d = plan.desc
    if num_sms is None:
        import torch
        num_sms = torch.cuda.get_device_properties(plan.device).multi_processor_count
    return (f"N{d.grid_n}-S{d.support_min}-{d.support_max}-b{d.oversample}-P{d.n_wplanes}"
            f"-pol{d.npol}-vis{d.vis_dtype}-tab{d.table_dtype}-sm{int(num_sms)}")


class TuningCache:
    """Best tuning per setup name, optionally persisted as JSON."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.best: Dict[str, dict] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.best = json.load(f)

    def get(self, name: str) -> Optional[dict]:
        return self.best.get(name)

    def put(self, name: str, tuning: dict):
        self.best[name] = dict(tuning)
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.best, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
