"""Host logic of the serving loop (no GPU): admission, HBM budget, eviction,
slot affinity, latency statistics, and the serving-stream generator."""
import math

import numpy as np

import synthetic as syn
from paper_2111_04141_gb300.serve import Job, Scheduler, latency_stats


def job(i, setup="a", arrival=0.0):
    return Job(id=i, kind="grid", setup=setup, nrow=10, arrival=arrival)


def test_fifo_admission_fills_free_slots_then_waits():
    s = Scheduler(n_slots=2, budget=10**12)
    for i in range(5):
        s.arrive(job(i))
    got = s.admit(lambda slot, setup: 0)
    assert [j.id for j, *_ in got] == [0, 1]
    assert sorted(slot for _, slot, *_ in got) == [0, 1]
    assert s.admit(lambda slot, setup: 0) == []          # no free slot
    s.complete(got[0][1])
    nxt = s.admit(lambda slot, setup: 0)
    assert [j.id for j, *_ in nxt] == [2]                # strict arrival order
    assert nxt[0][1] == got[0][1]


def test_budget_blocks_until_memory_is_released():
    s = Scheduler(n_slots=3, budget=100, resident=40)
    s.arrive(job(0, "a"))
    s.arrive(job(1, "b"))
    s.arrive(job(2, "c"))
    cost = lambda slot, setup: 0 if (slot, setup) in s.state else 30
    first = s.admit(cost)
    # 40 + 30 = 70 fits; a second state would need 100 -> also fits; a third would not
    assert [j.id for j, *_ in first] == [0, 1]
    assert s.used == 100
    assert s.admit(cost) == []                          # c waits: a and b are busy
    s.complete(first[0][1])                             # a finishes: its state is idle now
    got = s.admit(cost)
    assert [j.id for j, *_ in got] == [2]
    _, slot, evicted, need = got[0]
    assert evicted == [(first[0][1], "a")] and need == 30
    assert s.used == 100
    assert (first[1][1], "b") in s.state                # busy state never evicted


def test_head_of_line_is_not_overtaken():
    s = Scheduler(n_slots=3, budget=100, resident=0)
    s.arrive(job(0, "a"))
    cost = lambda slot, setup: 0 if (slot, setup) in s.state else {"a": 60, "big": 70,
                                                                    "small": 1}[setup]
    first = s.admit(cost)                               # a runs and holds 60
    assert [j.id for j, *_ in first] == [0]
    s.arrive(job(1, "big"))
    s.arrive(job(2, "small"))
    assert s.admit(cost) == []          # big fits only once a's state is idle; small waits too
    assert [j.id for j in s.pending] == [1, 2]
    s.complete(first[0][1])
    got = s.admit(cost)
    assert [j.id for j, *_ in got] == [1, 2]


def test_job_that_can_never_fit_is_rejected_not_waited_for():
    # resident 40 + a state of 70 > budget 100 even with no other state: the
    # job would wait forever (and block the queue behind it), so it leaves
    # the queue with an error and the next job runs
    s = Scheduler(n_slots=2, budget=100, resident=40)
    s.arrive(job(0, "huge"))
    s.arrive(job(1, "small"))
    cost = lambda slot, setup: {"huge": 70, "small": 10}[setup]
    got = s.admit(cost)
    assert [j.id for j, *_ in got] == [1]
    rej = s.take_rejected()
    assert [j.id for j in rej] == [0] and "budget" in rej[0].error
    assert s.used == 50 and not s.pending
    assert s.take_rejected() == []


def test_cancelled_job_leaves_the_queue_without_running():
    s = Scheduler(n_slots=1, budget=10**9)
    for i in range(3):
        s.arrive(job(i))
    first = s.admit(lambda slot, setup: 0)
    assert [j.id for j, *_ in first] == [0]
    assert s.cancel(1) is True
    assert s.cancel(0) is False                         # running: cannot be cancelled
    assert s.cancel(99) is False
    assert s.admit(lambda slot, setup: 0) == []         # no free slot yet
    s.complete(first[0][1])
    got = s.admit(lambda slot, setup: 0)
    assert [j.id for j, *_ in got] == [2]
    rej = s.take_rejected()
    assert [j.id for j in rej] == [1] and rej[0].error == "cancelled before admission"


def test_server_rejects_invalid_jobs_before_any_gpu_work():
    # a Server whose jobs are all invalid never touches the device: the
    # checks run on arrival and the jobs finish with an error and no result
    import torch
    from paper_2111_04141_gb300.serve import Server, Setup
    st = Setup("s", dict(grid_n=64, cell_rad=1e-3, support_min=7, support_max=7, oversample=8,
                         n_wplanes=1, w_max_lambda=0.0, npol=1), np.array([1.4e8, 1.5e8]))
    results = []
    srv = Server([st], "cpu", budget=1 << 30, n_slots=2, max_vis=1000,
                 on_result=lambda j, out: results.append((j.id, out)))
    srv.sched = Scheduler(2, 1 << 30)
    jobs = [Job(id=0, kind="grid", setup="s", nrow=501, arrival=0.0),      # 1002 > max_vis
            Job(id=1, kind="grid", setup="nope", nrow=1, arrival=0.0),
            Job(id=2, kind="transpose", setup="s", nrow=1, arrival=0.0)]
    done = srv.run(jobs)
    assert sorted(j.id for j in done) == [0, 1, 2]
    assert all(j.error for j in done)
    assert "max_vis" in jobs[0].error and "unknown setup" in jobs[1].error
    assert "kind" in jobs[2].error
    assert sorted(results) == [(0, None), (1, None), (2, None)]
    assert not srv.sched.busy and not srv.sched.pending


def test_slot_affinity_reuses_a_slot_holding_the_setup():
    s = Scheduler(n_slots=4, budget=10**9)
    s.state[(2, "x")] = 5
    s.lru[(2, "x")] = True
    s.arrive(job(0, "x"))
    got = s.admit(lambda slot, setup: 0 if (slot, setup) in s.state else 5)
    assert got[0][1] == 2 and got[0][3] == 0


def test_lru_evicts_oldest_idle_state_first():
    s = Scheduler(n_slots=2, budget=100, resident=0)
    for k, setup in enumerate(["p", "q", "r"]):
        s.state[(1, setup)] = 30
        s.lru[(1, setup)] = True
    s.used = 90
    s.arrive(job(0, "z"))
    got = s.admit(lambda slot, setup: 0 if (slot, setup) in s.state else 30)
    # slot 0 is free and empty: evict only the least recently used idle state
    assert got[0][2] == [(1, "p")]
    assert s.used == 90


def test_latency_stats():
    jobs = []
    for i in range(100):
        j = job(i, arrival=i * 0.01)
        j.t_done = j.arrival + 0.001 * (i + 1)
        j.work = 1e6
        jobs.append(j)
    st = latency_stats(jobs)
    assert math.isclose(st["p50_ms"], np.percentile(np.arange(1, 101), 50), rel_tol=1e-9)
    assert math.isclose(st["p99_ms"], np.percentile(np.arange(1, 101), 99), rel_tol=1e-9)
    assert math.isclose(st["makespan_s"], 0.99 + 0.1, rel_tol=1e-9)
    assert math.isclose(st["updates_per_s"], 1e8 / 1.09, rel_tol=1e-9)


def test_serving_stream_generator():
    setups = syn.serving_setups(n_setups=4, max_vis=20_000)
    for s in setups:
        kw = s["plan_kwargs"]
        field = kw["cell_rad"] * kw["grid_n"]
        assert 0.19 <= field <= 0.81
        assert 2 * (field / 2) ** 2 < 1.0
        assert kw["support_max"] % 2 == 1 and 7 <= kw["support_max"] <= 63
        assert s["uvw_sorted"].shape == s["uvw_shuffled"].shape
        assert np.allclose(np.sort(s["uvw_sorted"][:, 0]), np.sort(s["uvw_shuffled"][:, 0]))
    jobs = syn.serving_jobs(setups, n_jobs=400, min_vis=100, max_vis=20_000)
    nv = np.array([j["nrow"] for j in jobs])
    assert nv.min() >= 1
    kinds = [j["kind"] for j in jobs]
    assert 120 <= kinds.count("grid") <= 280
    names = {s["name"]: s for s in setups}
    for j in jobs:
        assert j["offset"] + j["nrow"] <= names[j["setup"]]["uvw_sorted"].shape[0]
    # log-uniform sizes: about half below the geometric mean
    nvis = np.array([j["nrow"] * names[j["setup"]]["freq_hz"].shape[0] for j in jobs])
    frac = np.mean(nvis < np.sqrt(100 * 20_000))
    assert 0.35 <= frac <= 0.65
    t = syn.poisson_arrivals(5000, 200.0)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 200.0) < 0.1 / 200.0


def test_work_cap_keeps_large_jobs_apart_but_lets_small_ones_overlap():
    s = Scheduler(n_slots=4, budget=10**12, work_cap=100.0, work_slack=0.5)
    big1, big2 = job(0), job(1)
    small = [job(2 + i) for i in range(3)]
    big1.work, big2.work = 500.0, 100.0            # both fill the GPU (load 1)
    for j in small:
        j.work = 20.0                               # load 0.2 each
    s.arrive(big1)
    got = s.admit(lambda slot, setup: 0)
    assert [j.id for j, *_ in got] == [0]           # the first job always runs
    for j in small[:2]:
        s.arrive(j)
    got = s.admit(lambda slot, setup: 0)
    assert [j.id for j, *_ in got] == [2, 3]        # 1 + 0.2 + 0.2 <= 1.5
    s.arrive(big2)
    s.arrive(small[2])
    assert s.admit(lambda slot, setup: 0) == []     # big2 at the head would reach 2.4
    s.complete(got[0][1])
    s.complete(got[1][1])
    assert s.admit(lambda slot, setup: 0) == []     # still 1 + 1 > 1.5 while big1 runs
    s.complete(0)
    got = s.admit(lambda slot, setup: 0)
    assert [j.id for j, *_ in got] == [1, 4]        # big2 alone, then the small one


def test_without_work_cap_only_slots_and_memory_limit_admission():
    s = Scheduler(n_slots=3, budget=10**12)
    for i in range(3):
        j = job(i)
        j.work = 1e15
        s.arrive(j)
    assert [j.id for j, *_ in s.admit(lambda slot, setup: 0)] == [0, 1, 2]


def test_slow_job_holds_one_slot_while_the_others_keep_serving():
    """A job that does not finish (a fake slow job: its slot is never
    completed) keeps only its own slot; every later job is served by the
    other slots in arrival order."""
    s = Scheduler(n_slots=3, budget=10**12)
    for i in range(12):
        s.arrive(job(i))
    first = s.admit(lambda slot, setup: 0)
    slow_slot = first[0][1]                               # job 0 never completes
    served = [j.id for j, *_ in first]
    running = {slot: j for j, slot, *_ in first}
    while s.pending:
        for slot in [sl for sl in list(running) if sl != slow_slot]:
            s.complete(slot)
            del running[slot]
        got = s.admit(lambda slot, setup: 0)
        assert got, "the other slots must keep admitting"
        assert all(slot != slow_slot for _, slot, *_ in got)
        for j, slot, *_ in got:
            running[slot] = j
            served.append(j.id)
    assert served == list(range(12))
    assert s.busy[slow_slot].id == 0


def test_tuning_cache_keys_by_plan_parameters_and_persists(tmp_path):
    """The autotuner cache key names the plan parameters the timings depend
    on and the SM count; the cache survives a reload from its JSON file."""
    from types import SimpleNamespace
    from paper_2111_04141_gb300.tune import TuningCache, plan_key
    desc = SimpleNamespace(grid_n=4096, support_min=7, support_max=63, oversample=8,
                           n_wplanes=32, npol=4, vis_dtype=0, table_dtype=1)
    plan = SimpleNamespace(desc=desc, device=None)
    k = plan_key(plan, num_sms=152)
    assert k == "N4096-S7-63-b8-P32-pol4-vis0-tab1-sm152"
    assert plan_key(plan, num_sms=148) != k
    desc.table_dtype = 0
    assert plan_key(plan, num_sms=152) != k
    path = str(tmp_path / "tune.json")
    c = TuningCache(path)
    c.put(k, {"item_max": 2048, "degrid_kernel": 1, "grid_kernel": 0, "compress_min_gain": 0})
    assert TuningCache(path).get(k)["item_max"] == 2048
    assert TuningCache(path).get("other") is None
