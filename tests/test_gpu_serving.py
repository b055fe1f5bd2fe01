"""Serving engine (continuous batching of reservoir jobs): each job's result is
the one the same reservoir gives stepped alone -- identical integer counters
and particle counts, energies equal up to the summation order of the moment
reduction -- whatever else was resident, however many engine iterations it
took, and whether it waited in the queue for memory.  FP64 jobs reproduce the
oracle's counters."""
import time

import numpy as np
import pytest

import oracle
from paper_2606_31548_b300 import hcao
from paper_2606_31548_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _jobs(n_res=9, seed=0x5E12):
    bw = W.batched_reservoirs(n_res=n_res, n_min=800, n_max=30000, T_min=5000.0, T_max=30000.0,
                              steps=1, seed=seed)
    rng = np.random.default_rng(seed)
    steps = [int(x) for x in rng.integers(0, 14, size=n_res)]
    steps[0] = 0  # a job with nothing to do
    return bw, steps


def _alone(bw, w, n_steps, precision):
    a = hcao.Context(precision=precision)
    a.set_species(bw.species)
    a.set_reactions(bw.reactions)
    rid = a.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    a.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
    a.init_vibration(rid, w.T_vib0)
    a.step(n_steps)
    out = (a.read_counters(rid), a.count(rid), a.read_moments(rid))
    a.close()
    return out


def _wait(ctx, ids, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(ids):
        for j in ids:
            if j not in res:
                r = ctx.serve_poll(j)
                if r is not None:
                    res[j] = r
        assert time.time() - t0 < timeout, "served jobs did not finish"
        time.sleep(0.002)
    return res


def _same(r, alone):
    cnt, n, m = alone
    assert r.status == 0
    assert np.array_equal(np.array(r.counters[: len(cnt)], np.uint64), cnt), (list(r.counters), cnt)
    assert r.n_particles == n
    assert list(r.moments.n) == list(m.n)
    for a, b in [(r.moments.E_tr, m.E_tr)] + [(r.moments.E_vib[i], m.E_vib[i]) for i in range(2)]:
        assert abs(a - b) <= 1e-12 * abs(b), (a, b)
    assert r.t_submit <= r.t_admit <= r.t_done


@pytest.mark.parametrize("precision", [hcao.FP64, hcao.FP32])
def test_served_jobs_equal_alone(precision):
    bw, steps = _jobs()
    ctx = hcao.Context(precision=precision)
    ctx.set_species(bw.species)
    # a budget of about three mid-size jobs: later jobs queue for memory and
    # are admitted while others are resident; K <= 4 steps per iteration
    ctx.serve_start(hbm_budget_bytes=24 << 20, max_active=4, max_batch_steps=4)
    ids = []
    for i, w in enumerate(bw.reservoirs):
        ids.append(ctx.serve_submit(w, steps[i]))
        if i == 3:
            time.sleep(0.05)  # the first wave is already running
    res = _wait(ctx, ids)
    q, a, used, iters = ctx.serve_stats()
    t = ctx.serve_timing()
    ctx.serve_stop()
    assert q == 0 and a == 0 and used == 0
    assert iters >= max(steps) // 4
    # the engine's time by activity: every job was admitted, stepped and retired
    assert t["admit_s"] > 0 and t["step_s"] > 0 and t["retire_s"] > 0 and t["wait_s"] >= 0
    for i, w in enumerate(bw.reservoirs):
        _same(res[ids[i]], _alone(bw, w, steps[i], precision))
        assert res[ids[i]].steps == steps[i]
    ctx.close()


def test_served_fp64_counters_match_oracle():
    bw, steps = _jobs(n_res=4, seed=0x5E13)
    ctx = hcao.Context(precision=hcao.FP64)
    ctx.set_species(bw.species)
    ctx.serve_start()
    ids = [ctx.serve_submit(w, steps[i]) for i, w in enumerate(bw.reservoirs)]
    res = _wait(ctx, ids)
    ctx.serve_stop()
    for i, w in enumerate(bw.reservoirs):
        o = oracle.from_workload(w)
        o.step(steps[i])
        co = o.read_counters(0)
        got = np.array(res[ids[i]].counters[:8], np.uint64)
        assert np.array_equal(got, co[:8]), (got, co[:8])


def test_serving_rejects_direct_calls_and_reports_failed_jobs():
    bw, steps = _jobs(n_res=3, seed=0x5E14)
    ctx = hcao.Context(precision=hcao.FP32)
    ctx.set_species(bw.species)
    ctx.serve_start(max_batch_steps=2)
    with pytest.raises(hcao.HcaoError) as e:
        ctx.step(1)  # only the engine thread steps a serving context
    assert e.value.code == -6
    bad = bw.reservoirs[1]
    bad.cell = bad.cell.copy()
    bad.cell[0] = 5  # a cell index outside the job's single cell
    ids = [ctx.serve_submit(w, 3) for w in bw.reservoirs]
    done = {}
    t0 = time.time()
    while len(done) < 3:
        for k, j in enumerate(ids):
            if j in done:
                continue
            try:
                r = ctx.serve_poll(j)
                if r is not None:
                    done[j] = r.status
            except hcao.HcaoError as err:
                done[j] = err.code
        assert time.time() - t0 < 60
        time.sleep(0.002)
    assert done[ids[0]] == 0 and done[ids[2]] == 0
    assert done[ids[1]] == -1  # EINVAL from the load
    with pytest.raises(hcao.HcaoError):
        ctx.serve_poll(ids[0])  # released by the first successful poll
    ctx.serve_stop()
    ctx.step(1)  # usable again once the engine has stopped
    ctx.close()


def _alone_w(sw, w, n_steps, precision, max_rounds):
    a = hcao.Context(precision=precision, max_rounds=max_rounds)
    a.set_species(sw.species)
    a.set_reactions(sw.reactions)
    rid = a.add_reservoir(w.n_cells, w.cell_volume, w.weight, w.dt, w.seed, w.T_tr0)
    a.load_particles(rid, w.v, w.qn0(), w.species_idx, w.cell)
    a.init_vibration(rid, w.T_vib0)
    a.step(n_steps)
    out = (a.read_counters(rid), a.count(rid), a.read_moments(rid))
    a.close()
    return out


@pytest.mark.parametrize("precision", [hcao.FP64, hcao.FP32])
def test_served_jobs_with_chemistry_equal_alone(precision):
    """The served mix of the benchmark's kinds -- triatomic relaxation, CH4
    heat bath with dissociation, CH4 <-> CH3 + H with recombination --
    at small sizes: each job's counters (reaction events included), particle
    count and moments equal the same job stepped alone."""
    sw = W.served_jobs(n_jobs=9, rate=1000.0, n_min=1500, n_max=12000, steps_min=2, steps_max=9,
                       recombination=True, seed=0x5E15)
    kinds = {j.kind for j in sw.jobs}
    assert kinds == {"relax", "bath", "equil"}
    ctx = hcao.Context(precision=precision, max_rounds=4)
    ctx.set_species(sw.species)
    ctx.set_reactions(sw.reactions)
    ctx.serve_start(hbm_budget_bytes=12 << 20, max_active=4, max_batch_steps=3)
    ids = [ctx.serve_submit(j.workload, j.steps) for j in sw.jobs]
    res = _wait(ctx, ids)
    ctx.serve_stop()
    rx_events = 0
    for jid, j in zip(ids, sw.jobs):
        r = res[jid]
        cnt, n, m = _alone_w(sw, j.workload, j.steps, precision, 4)
        assert r.status == 0 and r.steps == j.steps
        assert np.array_equal(np.array(r.counters[: len(cnt)], np.uint64), cnt), (j.kind, list(r.counters), cnt)
        assert r.n_particles == n
        assert list(r.moments.n) == list(m.n)
        for a, b in [(r.moments.E_tr, m.E_tr), (r.moments.E_form, m.E_form)] + \
                [(r.moments.E_vib[i], m.E_vib[i]) for i in range(4)]:
            assert abs(a - b) <= 1e-12 * max(abs(b), 1e-30), (j.kind, a, b)
        rx_events += int(sum(cnt[8:]))
    assert rx_events > 0
    ctx.close()


def _poll_status(ctx, jid, timeout=60.0):
    """The final status of a job: 0, or the error code its poll raises."""
    t0 = time.time()
    while True:
        try:
            r = ctx.serve_poll(jid)
        except hcao.HcaoError as e:
            return e.code
        if r is not None:
            return r.status
        assert time.time() - t0 < timeout, "served job did not finish"
        time.sleep(0.002)


def test_serving_cancel_queued_and_resident_jobs():
    """A resident job cancelled mid-run is retired at the end of the engine's
    iteration and reports HCAO_ECANCELLED; a queued job is dropped at once;
    the job that runs beside them is unaffected (equal to itself alone);
    cancelling a finished job is HCAO_ENOTFOUND."""
    bw, _ = _jobs(n_res=3)
    ctx = hcao.Context(precision=hcao.FP32)
    ctx.set_species(bw.species)
    # one resident job at a time; 4 steps per iteration
    ctx.serve_start(max_active=1, max_batch_steps=4)
    w_long, w_queued, w_short = bw.reservoirs
    long_id = ctx.serve_submit(w_long, 200000)
    queued_id = ctx.serve_submit(w_queued, 5)
    time.sleep(0.2)  # the long job is resident and stepping, the other queued
    ctx.serve_cancel(queued_id)
    ctx.serve_cancel(long_id)
    assert _poll_status(ctx, queued_id) == -11
    assert _poll_status(ctx, long_id) == -11
    short_id = ctx.serve_submit(w_short, 6)
    res = _wait(ctx, [short_id])
    with pytest.raises(hcao.HcaoError) as e:
        ctx.serve_cancel(short_id)  # finished and released
    assert e.value.code == -9
    q, a, used, _ = ctx.serve_stats()
    ctx.serve_stop()
    assert q == 0 and a == 0 and used == 0
    _same(res[short_id], _alone(bw, w_short, 6, hcao.FP32))
    ctx.close()


def test_serving_admission_allocation_failure():
    """A device allocation that fails while a job is admitted (injected on
    the host) fails that job with HCAO_ENOMEM; the engine goes on, and the
    next job's result equals its run alone."""
    bw, _ = _jobs(n_res=2)
    ctx = hcao.Context(precision=hcao.FP64)
    ctx.set_species(bw.species)
    ctx.serve_start(max_active=4, max_batch_steps=4)
    ctx.debug_fail_allocs(1)
    bad = ctx.serve_submit(bw.reservoirs[0], 5)
    assert _poll_status(ctx, bad) == -2
    ctx.debug_fail_allocs(0)
    good = ctx.serve_submit(bw.reservoirs[1], 7)
    res = _wait(ctx, [good])
    q, a, used, _ = ctx.serve_stats()
    ctx.serve_stop()
    assert q == 0 and a == 0 and used == 0
    _same(res[good], _alone(bw, bw.reservoirs[1], 7, hcao.FP64))
    ctx.close()
