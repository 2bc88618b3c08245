"""Host logic of the serving form (no GPU): the request stream, HBM admission
and the continuous-batching scheduler, driven by a stand-in executor."""
import random
import threading
import time

import numpy as np
import pytest

from paper_2511_18233_gb300 import serve, synth


def test_trajectory_pool_properties():
    specs = serve.make_trajectories(200, seed=3)
    again = serve.make_trajectories(200, seed=3)
    assert specs == again
    kinds = {s.kind for s in specs}
    assert kinds == {"chain", "flake"}
    for s in specs:
        assert 5 <= s.nstates <= 10
        assert 0 <= s.active <= s.nstates - 2          # S_1 .. S_{n-1}
        if s.kind == "chain":
            assert s.size in range(4, 41, 4)
        else:
            assert 4.0 <= s.size <= 7.0
        for (i, j) in s.pairs:                          # neighbours of the active state
            assert j == i + 1 and s.active in (i, j) and 0 <= i and j < s.nstates
        assert (s.active, s.active + 1) in s.pairs
        assert ((s.active - 1, s.active) in s.pairs) == (s.active >= 1)


def test_step_geometry_displacements():
    el, xyz = synth.chain_geometry(40)
    spec = serve.TrajectorySpec(0, "chain", 40, 5, 1, 123)
    a = serve.step_coords(xyz, spec, 4)
    b = serve.step_coords(xyz, spec, 4)
    c = serve.step_coords(xyz, spec, 5)
    np.testing.assert_array_equal(a, b)
    assert not np.allclose(a, c)
    d = np.concatenate([serve.step_coords(xyz, spec, s) - xyz for s in range(40)]).ravel()
    sigma = 0.05 * synth.ANGSTROM
    assert abs(d.mean()) < 4 * sigma / np.sqrt(d.size)
    assert abs(d.std() / sigma - 1.0) < 0.05


def test_poisson_arrivals():
    t = serve.poisson_arrivals(20000, 200.0, seed=1)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.03
    # exponential gaps: coefficient of variation 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05


def test_percentile_nearest_rank():
    x = list(range(1, 101))
    random.Random(0).shuffle(x)
    assert serve.percentile(x, 50) == 50
    assert serve.percentile(x, 99) == 99
    assert serve.percentile(x, 100) == 100
    assert serve.percentile([7.0], 99) == 7.0


def test_footprint_estimate_grows_with_size():
    base = serve.footprint_bytes(512, 81, 102, 42, 102, 10, 3, True)
    assert serve.footprint_bytes(1024, 162, 204, 84, 204, 10, 3, True) > 8 * base * 0.9
    assert serve.footprint_bytes(512, 81, 102, 42, 102, 10, 3, True) >= \
        serve.footprint_bytes(512, 81, 102, 42, 102, 5, 3, True)
    # the derivative integrals alone (3 nao^2 nU, FP32 in mixed precision) are a lower bound
    assert base > 3 * 512 * 512 * 102 * 4
    assert serve.footprint_bytes(512, 81, 102, 42, 102, 10, 3, False) > 3 * 512 * 512 * 102 * 8


def test_molecule_dims_union_aux():
    mol = synth.chain_molecule(8, 1, p_aux=True, with_mo=False)
    dm = serve.molecule_dims(mol)
    natm = mol.natm
    assert dm["nK"] == natm and dm["nJ"] == natm + 3 * 8 and dm["nU"] == dm["nJ"]


def test_admission_accounting():
    a = serve.Admission(100)
    a.reside(30)
    assert a.fits(70) and not a.fits(71)
    a.take(50)
    assert a.fits(20) and not a.fits(21)
    a.give(50)
    assert a.fits(70)
    assert a.peak == 80


class _Traj:
    def __init__(self, tid):
        self.spec = serve.TrajectorySpec(tid, "chain", 4, 5, 1, tid)
        self.measured = 0
        self.busy = False
        self.next_step = 0
        self.ref = np.zeros((3, 3))

    def footprint(self, mixed):
        return 10 + self.spec.tid % 3 * 20 if not self.measured else self.measured


def _fake_executor(log, lock, budget_seen, adm):
    def run(slot, req):
        with lock:
            log.append(("start", slot, req.traj.spec.tid, req.step, time.perf_counter()))
            budget_seen.append(adm.resident + adm.running)
        time.sleep(0.002 + 0.003 * ((req.traj.spec.tid * 7 + req.step) % 5))
        with lock:
            log.append(("end", slot, req.traj.spec.tid, req.step, time.perf_counter()))
        return {"tid": req.traj.spec.tid, "step": req.step}, req.footprint
    return run


def test_scheduler_slots_and_budget():
    adm = serve.Admission(60)
    log, lock, seen = [], threading.Lock(), []
    sch = serve.Scheduler(4, adm, _fake_executor(log, lock, seen, adm))
    trajs = [_Traj(t) for t in range(12)]
    try:
        for k in range(60):
            tr = trajs[k % 12]
            r = serve.Request(tr, k // 12, None)
            r.footprint = tr.footprint(True)
            sch.submit(r)
        assert sch.wait_idle(30)
    finally:
        sch.close()
    assert len(sch.done) == 60 and all(r.error is None for r in sch.done)
    assert max(seen) <= 60                        # budget never exceeded
    assert 1 <= sch.max_inflight <= 4             # never more than the slots
    # per slot, runs never overlap
    for s in range(4):
        ev = [e for e in log if e[1] == s]
        for a, b in zip(ev[::2], ev[1::2]):
            assert a[0] == "start" and b[0] == "end" and a[2:4] == b[2:4]
    assert sch.max_inflight >= 2                  # several requests did run together


def test_scheduler_oversized_request_runs_alone():
    adm = serve.Admission(50)
    log, lock, seen = [], threading.Lock(), []
    sch = serve.Scheduler(3, adm, _fake_executor(log, lock, seen, adm))
    big = _Traj(0)
    big.measured = 80                             # larger than the whole budget
    small = [_Traj(t) for t in range(1, 5)]
    try:
        for k, tr in enumerate([small[0], big] + small[1:]):
            r = serve.Request(tr, 0, None)
            r.footprint = tr.footprint(True)
            sch.submit(r)
        assert sch.wait_idle(30)
    finally:
        sch.close()
    assert len(sch.done) == 5
    # while the oversized request ran, nothing else did
    t_big = [e for e in log if e[2] == 0]
    s0, e0 = t_big[0][4], t_big[1][4]
    for e in log:
        if e[2] != 0 and e[0] == "start":
            end = [f for f in log if f[0] == "end" and f[2:4] == e[2:4]][0][4]
            assert end <= s0 or e[4] >= e0


def test_scheduler_executor_error_is_reported():
    adm = serve.Admission(1000)

    def boom(slot, req):
        if req.step == 1:
            raise RuntimeError("planted failure")
        return {}, 0

    sch = serve.Scheduler(2, adm, boom)
    trajs = [_Traj(t) for t in range(3)]
    try:
        for s in range(3):
            for tr in trajs:
                r = serve.Request(tr, s, None)
                r.footprint = 1
                sch.submit(r)
        assert sch.wait_idle(30)
    finally:
        sch.close()
    errs = [r for r in sch.done if r.error]
    assert len(errs) == 3 and all("planted failure" in r.error for r in errs)
    assert adm.running == 0


def test_run_stream_keeps_trajectory_steps_sequential():
    adm = serve.Admission(10 ** 6)
    log, lock, seen = [], threading.Lock(), []
    sch = serve.Scheduler(4, adm, _fake_executor(log, lock, seen, adm))
    trajs = [_Traj(t) for t in range(6)]
    try:
        res = serve.run_stream(trajs, sch, n_requests=40, n_warmup=5, rate=2000.0, seed=2,
                               mixed=True, timeout=60)
    finally:
        sch.close()
    assert res["requests"] == 40 and res["errors"] == 0
    assert res["p50_ms"] <= res["p99_ms"]
    assert res["throughput_per_s"] > 0
    for tr in trajs:
        mine = sorted((r for r in res["done"] if r.traj is tr), key=lambda r: r.step)
        assert [r.step for r in mine] == list(range(len(mine)))
        for a, b in zip(mine, mine[1:]):          # step k+1 arrives after step k is done
            assert b.t_arrive >= a.t_done
