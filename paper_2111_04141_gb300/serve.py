"""Serving loop: continuous batching of gridding and degridding jobs on one GPU.

Jobs (grid or degrid requests against one of a set of registered imaging
setups) arrive over time.  The server keeps every setup's plan and kernel
tables on the device, and each setup's model grid for degridding.  It runs
jobs in *slots*: a slot is a CUDA stream with device staging buffers and,
per setup, a plan clone (own scratch, shared tables) plus CUDA graphs of the
gridding and degridding calls captured once with a device-side row count,
so one graph serves every job size.  A job that arrives while others run is
admitted as soon as a slot is free and the HBM budget holds what the slot
still has to allocate for its setup (idle slot state of other setups is
evicted least-recently-used first); its copies and kernels then overlap on
the device with the other slots' work.  Results come back through
per-slot pinned staging buffers and a callback.

Scheduling (``Scheduler``) is host logic only and is tested on the CPU; the
GPU side (``Server``) turns its decisions into stream work.  ``run_sequential``
is the baseline: one job at a time, plain launches on one stream.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Callable, Dict, List, Optional

import numpy as np


# --------------------------------------------------------------------------
# jobs and setups
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Setup:
    """An imaging setup jobs refer to: the plan descriptor plus channels."""
    name: str
    plan_kwargs: dict
    freq_hz: np.ndarray

    @property
    def grid_n(self):
        return self.plan_kwargs["grid_n"]

    @property
    def npol(self):
        return self.plan_kwargs["npol"]

    @property
    def nchan(self):
        return int(self.freq_hz.shape[0])

    def grid_bytes(self):
        return self.npol * self.grid_n * self.grid_n * 8


@dataclasses.dataclass
class Job:
    id: int
    kind: str                 # "grid" or "degrid"
    setup: str
    nrow: int
    arrival: float            # seconds from the start of the stream
    uvw: object = None        # host [nrow, 3] float64 (pinned torch tensor)
    vis: object = None        # host [nrow, nchan, npol] complex64 (grid jobs)
    work: float = 0.0         # grid-point pol-updates (filled by the server)
    t_admit: float = math.nan
    t_done: float = math.nan
    slot: int = -1
    cancelled: bool = False   # set before admission: the job is dropped, no GPU work
    error: Optional[str] = None  # why a job finished without running (rejected or cancelled)

    @property
    def latency(self):
        return self.t_done - self.arrival


# --------------------------------------------------------------------------
# scheduling (host logic)
# --------------------------------------------------------------------------

class Scheduler:
    """FIFO continuous-batching admission under an HBM budget and, optionally,
    a compute budget.

    ``cost(slot, setup)`` is the device memory a slot still has to allocate
    to run a job of ``setup`` (0 when the slot already holds that setup's
    state).  Slot state that is idle may be evicted, least recently used
    first, to make room; the head of the queue is never overtaken (no
    starvation), and a job that cannot fit even with every idle state
    evicted waits for running jobs to finish.  A job that could not fit even
    with no slot state at all (``resident + cost > budget``) would wait
    forever: it is rejected instead, as is a job whose ``cancelled`` flag is
    set when it reaches the head; both leave the queue with ``error`` set and
    no GPU work, and ``take_rejected`` hands them to the caller.

    With ``work_cap`` (grid-point updates of a job that fills the GPU), a
    job's load is min(1, work / work_cap) and the head is admitted only while
    the running jobs' loads plus its own stay within 1 + ``work_slack``: two
    GPU-filling jobs never share the GPU (sharing only delays the first of
    them), while small jobs still overlap with a large one.  The first job
    is always admitted.
    """

    def __init__(self, n_slots: int, budget: int, resident: int = 0,
                 work_cap: Optional[float] = None, work_slack: float = 0.5):
        self.n_slots = n_slots
        self.budget = budget
        self.work_cap = work_cap
        self.work_slack = work_slack
        self.resident = resident           # bytes held outside slot state (tables, models)
        self.used = resident
        self.rejected: List[Job] = []
        self.pending: collections.deque = collections.deque()
        self.busy: Dict[int, Job] = {}
        self.state: Dict[tuple, int] = {}  # (slot, setup) -> bytes held
        self.lru: collections.OrderedDict = collections.OrderedDict()

    def arrive(self, job: Job):
        self.pending.append(job)

    def cancel(self, job_id: int) -> bool:
        """Cancel a job that has not been admitted yet; False if it is not
        pending (already running, finished or unknown)."""
        for j in self.pending:
            if j.id == job_id:
                j.cancelled = True
                return True
        return False

    def take_rejected(self) -> List[Job]:
        out, self.rejected = self.rejected, []
        return out

    def _reject(self, job: Job, why: str):
        self.pending.popleft()
        job.error = why
        self.rejected.append(job)

    def free_slots(self) -> List[int]:
        return [s for s in range(self.n_slots) if s not in self.busy]

    def _pick_slot(self, setup: str, free: List[int]) -> int:
        # prefer a slot that already holds this setup's state
        for s in free:
            if (s, setup) in self.state:
                return s
        return free[0]

    def _evictable(self, exclude_slot: int):
        busy = set(self.busy)
        return [k for k in self.lru if k[0] not in busy and k[0] != exclude_slot]

    def load(self, job: Job) -> float:
        if self.work_cap is None:
            return 0.0
        return min(1.0, job.work / self.work_cap)

    def admit(self, cost: Callable[[int, str], int]):
        """Admit queue-head jobs while possible.  Returns a list of
        (job, slot, evicted_keys, new_bytes) decisions."""
        out = []
        while self.pending:
            job = self.pending[0]
            if job.cancelled:
                self._reject(job, "cancelled before admission")
                continue
            free = self.free_slots()
            if not free:
                break
            if self.work_cap is not None and self.busy:
                inflight = sum(self.load(j) for j in self.busy.values())
                if inflight + self.load(job) > 1.0 + self.work_slack:
                    break            # wait for running work to finish
            slot = self._pick_slot(job.setup, free)
            need = cost(slot, job.setup)
            if self.resident + need > self.budget:
                self._reject(job, f"needs {need} bytes of slot state but the budget leaves "
                                  f"{self.budget - self.resident} beside the resident "
                                  f"{self.resident}")
                continue
            evicted = []
            if self.used + need > self.budget:
                # evict idle state (LRU) until the job fits, if it can
                cands = self._evictable(slot) + [k for k in self.lru
                                                 if k[0] == slot and k[1] != job.setup]
                freeable = sum(self.state[k] for k in cands)
                if self.used - freeable + need > self.budget:
                    break            # wait for running jobs to release memory
                for k in cands:
                    if self.used + need <= self.budget:
                        break
                    self.used -= self.state.pop(k)
                    self.lru.pop(k)
                    evicted.append(k)
            self.pending.popleft()
            key = (slot, job.setup)
            if need:
                self.state[key] = self.state.get(key, 0) + need
                self.used += need
            self.lru[key] = True
            self.lru.move_to_end(key)
            self.busy[slot] = job
            job.slot = slot
            out.append((job, slot, evicted, need))
        return out

    def complete(self, slot: int) -> Job:
        return self.busy.pop(slot)


def latency_stats(jobs: List[Job]) -> dict:
    lat = np.array([j.latency for j in jobs])
    t0 = min(j.arrival for j in jobs)
    t1 = max(j.t_done for j in jobs)
    work = sum(j.work for j in jobs)
    return {"jobs": len(jobs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "max_ms": float(lat.max() * 1e3), "makespan_s": float(t1 - t0),
            "updates_per_s": float(work / max(t1 - t0, 1e-9)),
            "jobs_per_s": float(len(jobs) / max(t1 - t0, 1e-9))}


# --------------------------------------------------------------------------
# GPU execution
# --------------------------------------------------------------------------

class _SlotState:
    """Per (slot, setup): plan clone, device row count and captured graphs."""

    def __init__(self, plan, d_nrow):
        self.plan = plan
        self.d_nrow = d_nrow
        self.graphs = {}

    def close(self):
        self.graphs.clear()
        self.plan.close()


class Server:
    """Continuous-batching server on one GPU (see the module docstring).

    setups      registered imaging setups (plans are built at ``warm``)
    max_vis     largest job (visibilities) any slot must hold
    budget      device bytes the server may hold (tables, models, slot state)
    work_cap    nominal grid-point updates of a GPU-filling job for the
                scheduler's compute budget; None (the default) admits by slots
                and memory only, which measured better on the mixed stream
                (p99 26 ms vs 35 ms with a 2e10 cap)
    readback_bands  with graphs, a grid job's graph grids in this many bands of
                tile rows and copies each finished band to the slot's pinned
                host buffer while the next one grids
                (gw_grid_vis_devcount_readback); 0 (the default) copies the
                grid after the gridding.  In the mixed stream the slots'
                copies already overlap other slots' work, and banding measured
                no better (p99 0.49-0.55 vs 0.47-0.50 of sequential)
    on_result   callback(job, host_tensor) called when a job's result is in
                host memory (the tensor is a slot staging buffer: copy it to keep it);
                a job that was rejected or cancelled without running gets
                host_tensor None and its reason in job.error
    host_staging  optional list of n_slots pinned complex64 host tensors used as
                the slots' result staging instead of allocating new ones (for
                servers that never run at the same time); by default the slots'
                staging is one page-locked arena on huge pages
                (``hostmem.PinnedArena``)
    """

    def __init__(self, setups: List[Setup], device, budget: int, n_slots: int = 4,
                 max_vis: int = 10_000_000, use_graphs: bool = True, tuning: Optional[dict] = None,
                 on_result: Optional[Callable] = None, work_cap: Optional[float] = None,
                 readback_bands: int = 0, host_staging: Optional[list] = None):
        import torch
        from .plan import Plan
        self.torch = torch
        self.Plan = Plan
        self.setups = {s.name: s for s in setups}
        self.device = torch.device(device)
        self.n_slots = n_slots
        self.max_vis = int(max_vis)
        self.use_graphs = use_graphs
        self.tuning = tuning or {}
        self.on_result = on_result
        self.budget = int(budget)
        self.work_cap = work_cap
        self.readback_bands = int(readback_bands)
        self.host_staging = host_staging
        self._arena = None
        self.plans: Dict[str, object] = {}
        self.models: Dict[str, object] = {}
        self.freqs: Dict[str, object] = {}
        self.state: Dict[tuple, _SlotState] = {}
        self.slots = []
        self.sched: Optional[Scheduler] = None

    @staticmethod
    def default_work_cap() -> float:
        import inspect
        return inspect.signature(Server.__init__).parameters["work_cap"].default

    # ---- set-up -----------------------------------------------------------
    def warm(self, models: Optional[Dict[str, np.ndarray]] = None, prewarm: bool = True):
        """Build every setup's plan (tables) and upload models and channels;
        allocate the slots' staging buffers; with ``prewarm``, create each
        slot's clone and graphs for every setup while the budget allows (the
        rest are created, and evicted, on demand)."""
        torch = self.torch
        resident = 0
        max_rows = 1
        max_grid = 0
        max_vis_el = 1
        for name, s in self.setups.items():
            p = self.Plan(**s.plan_kwargs, max_vis_per_call=1 << 16, device=self.device)
            if name in self.tuning:
                p.set_tuning(**self.tuning[name])
            self.plans[name] = p
            resident += p.info.table_bytes + p.info.scratch_bytes
            self.freqs[name] = torch.from_numpy(s.freq_hz).to(self.device)
            g = torch.zeros((s.npol, s.grid_n, s.grid_n), dtype=torch.complex64,
                            device=self.device)
            if models and name in models:
                m = models[name]
                g.copy_(m if isinstance(m, torch.Tensor) else torch.from_numpy(m))
            self.models[name] = g
            resident += s.grid_bytes()
            rows = -(-self.max_vis // s.nchan)
            max_rows = max(max_rows, rows)
            max_grid = max(max_grid, s.grid_bytes())
            max_vis_el = max(max_vis_el, rows * s.nchan * s.npol)
        n_host = max(max_grid // 8, max_vis_el)
        if self.host_staging is None:
            # the slots' result staging: one page-locked arena on huge pages
            from . import hostmem
            self._arena = hostmem.PinnedArena(
                hostmem.arena_bytes([(n_host, torch.complex64)] * self.n_slots))
        else:
            if len(self.host_staging) < self.n_slots or any(
                    h.numel() < n_host or not h.is_pinned() or h.dtype != torch.complex64
                    for h in self.host_staging[:self.n_slots]):
                raise ValueError(f"host_staging needs {self.n_slots} pinned complex64 tensors "
                                 f"of at least {n_host} elements")
        for k in range(self.n_slots):
            st = torch.cuda.Stream(self.device)
            slot = {
                "stream": st,
                "uvw": torch.empty((max_rows, 3), dtype=torch.float64, device=self.device),
                "vis": torch.empty(max_vis_el, dtype=torch.complex64, device=self.device),
                "grid": torch.empty(max_grid // 8, dtype=torch.complex64, device=self.device),
                "host": (self.host_staging[k] if self.host_staging is not None else
                         self._arena.take(n_host, torch.complex64)),
                "event": torch.cuda.Event(),
            }
            resident += (max_rows * 24 + max_vis_el * 8 + max_grid)
            self.slots.append(slot)
        torch.cuda.synchronize(self.device)
        self.resident = resident
        self.sched = Scheduler(self.n_slots, self.budget, resident, work_cap=self.work_cap)
        if prewarm:
            for slot in range(self.n_slots):
                for name in self.setups:
                    need = self._state_bytes(name)
                    if self.sched.used + need > self.budget:
                        continue
                    if self.use_graphs:
                        for kind in ("grid", "degrid"):
                            self._graph(slot, name, kind)
                    else:
                        self._ensure_state(slot, name)
                    self.sched.state[(slot, name)] = need
                    self.sched.lru[(slot, name)] = True
                    self.sched.used += need
            torch.cuda.synchronize(self.device)

    def close(self):
        for st in self.state.values():
            st.close()
        self.state.clear()
        for p in self.plans.values():
            p.close()
        self.plans.clear()
        if self._arena is not None:
            self.torch.cuda.synchronize(self.device)
            self.slots = []
            self._arena.release()
            self._arena = None

    # ---- slot state -------------------------------------------------------
    def _state_bytes(self, setup: str) -> int:
        """Device bytes of a slot's clone for ``setup``: the master's scratch
        plus the per-visibility parts (record, bin entries, work items) for
        the extra chunk length."""
        s = self.setups[setup]
        p = self.plans[setup]
        sm1 = s.plan_kwargs["support_max"] - 1
        mt = (sm1 // p.info.grid_tile_u + 2) * (sm1 // p.info.grid_tile_v + 2)
        per_vis = 16 + 4 * mt + 16 * mt / 64.0
        return int(p.info.scratch_bytes + (self.max_vis - p.info.chunk_vis) * per_vis)

    def _cost(self, slot: int, setup: str) -> int:
        return 0 if (slot, setup) in self.state else self._state_bytes(setup)

    def _ensure_state(self, slot: int, setup: str) -> _SlotState:
        key = (slot, setup)
        st = self.state.get(key)
        if st is None:
            torch = self.torch
            clone = self.plans[setup].clone(max_vis_per_call=self.max_vis,
                                            stream=self.slots[slot]["stream"])
            d_nrow = torch.zeros(1, dtype=torch.int64, device=self.device)
            st = _SlotState(clone, d_nrow)
            self.state[key] = st
        return st

    def _views(self, slot: int, setup: str, nrow_max: int):
        s = self.setups[setup]
        b = self.slots[slot]
        uvw = b["uvw"][:nrow_max]
        vis = b["vis"][:nrow_max * s.nchan * s.npol].view(nrow_max, s.nchan, s.npol)
        grid = b["grid"][:s.npol * s.grid_n * s.grid_n].view(s.npol, s.grid_n, s.grid_n)
        return uvw, vis, grid

    def _graph(self, slot: int, setup: str, kind: str):
        """The (slot, setup, kind) graph, captured on first use."""
        torch = self.torch
        st = self._ensure_state(slot, setup)
        g = st.graphs.get(kind)
        if g is not None:
            return g
        s = self.setups[setup]
        rows = -(-self.max_vis // s.nchan)
        uvw, vis, grid = self._views(slot, setup, rows)
        freq = self.freqs[setup]
        stream = self.slots[slot]["stream"]
        model = self.models[setup]

        host = self.slots[slot]["host"]
        host_grid = host[:grid.numel()].view(grid.shape)

        def body():
            if kind == "grid":
                grid.zero_()
                if self.readback_bands > 0:
                    st.plan.grid_devcount_readback(uvw, freq, st.d_nrow, vis, grid, host_grid,
                                                   n_bands=self.readback_bands)
                else:
                    st.plan.grid_devcount(uvw, freq, st.d_nrow, vis, grid)
            else:
                st.plan.degrid_devcount(uvw, freq, st.d_nrow, model, vis)

        with torch.cuda.stream(stream):
            st.d_nrow.zero_()
            body()                               # warm-up outside capture
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            body()
        # one replay with no rows: the graph's first launch (upload to the
        # device) happens here instead of in the first job that uses it
        with torch.cuda.stream(stream):
            st.d_nrow.zero_()
            g.replay()
        stream.synchronize()
        st.graphs[kind] = g
        return g

    def _drop_state(self, key):
        st = self.state.pop(key, None)
        if st is not None:
            self.slots[key[0]]["stream"].synchronize()
            st.close()

    # ---- job execution ------------------------------------------------------
    def _launch(self, job: Job, slot: int):
        # an NVTX range per launch and per completion: profiler timelines show
        # which job each slot's stream work belongs to
        self.torch.cuda.nvtx.range_push(f"gw launch job {job.id} {job.kind} {job.setup} slot {slot}")
        try:
            self._launch_job(job, slot)
        finally:
            self.torch.cuda.nvtx.range_pop()

    def _launch_job(self, job: Job, slot: int):
        torch = self.torch
        s = self.setups[job.setup]
        b = self.slots[slot]
        stream = b["stream"]
        nvis = job.nrow * s.nchan
        if self.use_graphs:
            g = self._graph(slot, job.setup, job.kind)
            st = self.state[(slot, job.setup)]
        else:
            st = self._ensure_state(slot, job.setup)
        uvw, vis, grid = self._views(slot, job.setup, job.nrow)
        with torch.cuda.stream(stream):
            uvw.copy_(job.uvw, non_blocking=True)
            if job.kind == "grid":
                vis.copy_(job.vis, non_blocking=True)
            if self.use_graphs:
                st.d_nrow.fill_(job.nrow)
                g.replay()
            else:
                freq = self.freqs[job.setup]
                if job.kind == "grid":
                    grid.zero_()
                    st.plan.grid(uvw, freq, vis, out=grid, stream=stream)
                else:
                    st.plan.degrid(uvw, freq, self.models[job.setup], out=vis, stream=stream)
            host = b["host"]
            if job.kind == "grid":
                if not (self.use_graphs and self.readback_bands > 0):   # else copied by the graph
                    n = grid.numel()
                    host[:n].view(grid.shape).copy_(grid, non_blocking=True)
            else:
                n = nvis * s.npol
                host[:n].view(vis.shape).copy_(vis, non_blocking=True)
            b["event"].record(stream)

    def _finish(self, slot: int, now: float):
        self.torch.cuda.nvtx.range_push(f"gw finish slot {slot}")
        try:
            return self._finish_job(slot, now)
        finally:
            self.torch.cuda.nvtx.range_pop()

    def _finish_job(self, slot: int, now: float):
        job = self.sched.complete(slot)
        job.t_done = now
        if self.on_result is not None:
            s = self.setups[job.setup]
            host = self.slots[slot]["host"]
            if job.kind == "grid":
                out = host[:s.npol * s.grid_n * s.grid_n].view(s.npol, s.grid_n, s.grid_n)
            else:
                out = host[:job.nrow * s.nchan * s.npol].view(job.nrow, s.nchan, s.npol)
            self.on_result(job, out)
        return job

    def run(self, jobs: List[Job], clock=time.perf_counter) -> List[Job]:
        """Serve ``jobs`` (sorted by arrival, seconds from now); returns them
        with admission and completion times filled in."""
        jobs = sorted(jobs, key=lambda j: j.arrival)
        for j in jobs:
            j.work = self._job_work(j) if j.setup in self.setups else 0.0
        t0 = clock()
        i = 0
        done = []

        def finish_unrun(job):
            job.t_admit = job.t_done = clock() - t0
            done.append(job)
            if self.on_result is not None:
                self.on_result(job, None)

        while len(done) < len(jobs):
            now = clock() - t0
            while i < len(jobs) and jobs[i].arrival <= now:
                j = jobs[i]
                i += 1
                why = self._check(j)
                if why:
                    j.error = why
                    finish_unrun(j)
                else:
                    self.sched.arrive(j)
            for job, slot, evicted, _ in self.sched.admit(self._cost):
                for key in evicted:
                    self._drop_state(key)
                job.t_admit = clock() - t0
                self._launch(job, slot)
            for job in self.sched.take_rejected():
                finish_unrun(job)
            progressed = False
            for slot in list(self.sched.busy):
                if self.slots[slot]["event"].query():
                    done.append(self._finish(slot, clock() - t0))
                    progressed = True
            if not progressed and not self.sched.pending and i < len(jobs):
                wait = jobs[i].arrival - (clock() - t0)
                if wait > 2e-4 and not self.sched.busy:
                    time.sleep(wait - 1e-4)
        return done

    def _check(self, job: Job) -> Optional[str]:
        """Why a job cannot run on this server (checked on arrival, before
        any GPU work), or None."""
        s = self.setups.get(job.setup)
        if s is None:
            return f"unknown setup {job.setup!r}"
        if job.kind not in ("grid", "degrid"):
            return f"unknown job kind {job.kind!r}"
        if job.nrow < 0 or job.nrow * s.nchan > self.max_vis:
            return (f"{job.nrow} rows x {s.nchan} channels exceed the server's max_vis "
                    f"({self.max_vis})")
        return None

    def _job_work(self, job: Job) -> float:
        """Nominal grid-point pol-updates of a job: visibilities x npol x the
        mean S_p^2 over the setup's planes (the per-record planes are not
        known on the host; the same nominal figure is used for the
        sequential baseline, so throughputs compare like with like)."""
        s = self.setups[job.setup]
        return float(job.nrow * s.nchan * s.npol * _mean_s2(s))


def _mean_s2(s: Setup) -> float:
    kw = s.plan_kwargs
    P, smin, smax = kw["n_wplanes"], kw["support_min"], kw["support_max"]
    if P <= 1:
        return float(smin * smin)
    sup = [2 * ((smin * (P - 1) + (smax - smin) * p) // (2 * (P - 1))) + 1 for p in range(P)]
    return float(np.mean(np.square(sup)))


# --------------------------------------------------------------------------
# baseline: one job at a time, plain launches
# --------------------------------------------------------------------------

def run_sequential(setups: List[Setup], plans: dict, models: dict, freqs: dict, jobs: List[Job],
                   device, on_result: Optional[Callable] = None, clock=time.perf_counter,
                   host_buf=None):
    """Jobs in arrival order on one stream: wait for arrival, copy in, grid or
    degrid with the setup's plan (default tuning, no graphs), copy out into a
    preallocated pinned buffer (as the server's slots do; ``host_buf`` if
    given and large enough), synchronise."""
    import torch
    setups = {s.name: s for s in setups}
    jobs = sorted(jobs, key=lambda j: j.arrival)
    stream = torch.cuda.current_stream(device)
    n_host = max(max(setups[j.setup].npol * setups[j.setup].grid_n ** 2,
                     j.nrow * setups[j.setup].nchan * setups[j.setup].npol) for j in jobs) \
        if jobs else 1
    from . import hostmem
    owned = host_buf is None or host_buf.numel() < n_host
    if owned:
        host_buf = hostmem.pinned_empty(n_host, torch.complex64)
    try:
        return _run_sequential(setups, plans, models, freqs, jobs, device, on_result, clock,
                               host_buf, stream)
    finally:
        if owned:
            stream.synchronize()
            hostmem.release(host_buf)


def _run_sequential(setups, plans, models, freqs, jobs, device, on_result, clock, host_buf,
                    stream):
    t0 = clock()
    for j in jobs:
        s = setups[j.setup]
        j.work = float(j.nrow * s.nchan * s.npol * _mean_s2(s))
        now = clock() - t0
        if j.arrival > now:
            time.sleep(j.arrival - now)
        j.t_admit = clock() - t0
        uvw = j.uvw.to(device, non_blocking=True)
        p = plans[j.setup]
        if j.kind == "grid":
            vis = j.vis.to(device, non_blocking=True)
            out = p.grid(uvw, freqs[j.setup], vis)
        else:
            out = p.degrid(uvw, freqs[j.setup], models[j.setup])
        host = host_buf[:out.numel()].view(out.shape)
        host.copy_(out, non_blocking=True)
        stream.synchronize()
        j.t_done = clock() - t0
        if on_result is not None:
            on_result(j, host)
    return jobs


# --------------------------------------------------------------------------
# wiring of generated specs into setups and jobs (host buffers pinned)
# --------------------------------------------------------------------------

def build_stream(setup_specs: List[dict], job_specs: List[dict], arrivals, max_vis: int,
                 vis_seed: int = 0):
    """Setups and Jobs from plain specs: per setup, pinned pools of sorted
    and shuffled uvw rows and of visibilities (CN(0, 1), max_vis x npol),
    all in one page-locked arena on huge pages; every job is a view into its
    setup's pools."""
    import torch
    from . import hostmem
    gen = torch.Generator().manual_seed(vis_seed)
    setups, host = [], {}
    for d in setup_specs:
        st = Setup(d["name"], dict(d["plan_kwargs"]), np.asarray(d["freq_hz"]))
        setups.append(st)
        npol, nchan = st.npol, st.nchan
        rows = -(-max_vis // nchan)
        v = torch.randn((rows, nchan, npol, 2), generator=gen, dtype=torch.float32)
        v.mul_(float(np.sqrt(0.5)))
        host[st.name] = {
            "sorted": torch.from_numpy(np.ascontiguousarray(d["uvw_sorted"])),
            "shuffled": torch.from_numpy(np.ascontiguousarray(d["uvw_shuffled"])),
            "vis": torch.view_as_complex(v),
        }
    arena = hostmem.PinnedArena(hostmem.arena_bytes(
        [(t.shape, t.dtype) for h in host.values() for t in h.values()]))
    pools = {}
    for name, h in host.items():
        pools[name] = {}
        for k, t in h.items():
            pools[name][k] = arena.take(t.shape, t.dtype)
            pools[name][k].copy_(t)
    jobs = []
    for spec, t in zip(job_specs, arrivals):
        pool = pools[spec["setup"]]
        o, n = spec["offset"], spec["nrow"]
        uvw = pool["shuffled" if spec["shuffled"] else "sorted"][o:o + n]
        vis = pool["vis"][:n] if spec["kind"] == "grid" else None
        jobs.append(Job(id=spec["id"], kind=spec["kind"], setup=spec["setup"], nrow=n,
                        arrival=float(t), uvw=uvw, vis=vis))
    return setups, jobs
