"""Host logic of the serving engine (admission by free slot and HBM budget,
arrival order per shape), with the C library replaced by a fake server that
finishes jobs after a fixed number of polls.  No GPU."""
import types

import numpy as np
import pytest

from paper_2309_14584_gb300 import serving


class _FakePlan:
    count = 0

    def __init__(self, support, sizes, nodes=None, **opts):
        _FakePlan.count += 1
        self.handle = 1000 + _FakePlan.count
        n = int(np.asarray(support).shape[0])
        self.info = {"N": n, "M": 10 * n, "R": 3 * n}
        # tables and one workspace, as the library reports them
        self.info["device_bytes"] = 8.0 * (2 * 10 * n + 3 * 3 * n + 2 * n) + 4.0 * (3 * n + 3 * n)

    def clone(self):
        c = _FakePlan.__new__(_FakePlan)
        _FakePlan.count += 1
        c.handle = 1000 + _FakePlan.count
        c.info = dict(self.info)
        return c

    def close(self):
        pass


class _FakeServer:
    def __init__(self, work_polls):
        self.jobs = {}
        self.next = 0
        self.work_polls = work_polls
        self.in_flight_handles = []
        self.max_same_handle = 0
        self.log = []

    def submit(self, plan, x, c):
        assert plan not in self.in_flight_handles, "a plan handle was reused while its job ran"
        self.in_flight_handles.append(plan)
        t = self.next
        self.next += 1
        self.jobs[t] = [self.work_polls, plan]
        self.log.append((t, plan, c))
        return t

    def poll(self, t):
        j = self.jobs[t]
        j[0] -= 1
        if j[0] <= 0:
            if j[1] in self.in_flight_handles:
                self.in_flight_handles.remove(j[1])
            return {"status": 0, "iterations": 1, "refinements": 1, "rel_normal_residual": 0.0, "gamma0": 1.0}
        return None


def _engine(monkeypatch, shapes, budget, max_slots, work_polls=3):
    srv = _FakeServer(work_polls)
    fake = types.SimpleNamespace(
        Plan=_FakePlan,
        fct_server_create=lambda *a: srv,
        fct_server_submit=lambda s, plan, x, c: s.submit(plan, x, c),
        fct_server_poll=lambda s, t: s.poll(t),
        fct_server_destroy=lambda s: None,
    )
    monkeypatch.setattr(serving, "F", fake)
    return serving.ServingEngine(shapes, hbm_budget_bytes=budget, max_slots_per_shape=max_slots), srv


def _shape(n):
    return types.SimpleNamespace(support=np.zeros((n, 2), dtype=np.uint16), sizes=np.ones((1, 2), np.int32),
                                 nodes=np.zeros((1, 2)))


def test_all_requests_finish_in_arrival_order_per_shape(monkeypatch):
    shapes = [_shape(100), _shape(300)]
    eng, srv = _engine(monkeypatch, shapes, budget=1e9, max_slots=2)
    reqs = [(0.0, i % 2, ("in", i % 2)) for i in range(12)]
    outs = [f"out{i}" for i in range(12)]
    res = eng.run(reqs, {("in", 0): "x0", ("in", 1): "x1"}, outs, timeout_s=30)
    assert all(r is not None and r["report"]["status"] == 0 for r in res)
    # submissions of each shape follow arrival order
    order = [outs.index(c) for _, _, c in srv.log]
    for s in (0, 1):
        mine = [i for i in order if reqs[i][1] == s]
        assert mine == sorted(mine)
    s = serving.latency_summary(res, [100 if r[1] == 0 else 300 for r in reqs])
    assert s["requests"] == 12 and s["all_converged"] and s["p99_ms"] >= s["p50_ms"] >= 0


def test_slots_and_budget_bound_the_work_in_flight(monkeypatch):
    shapes = [_shape(1000)]
    one_slot = 8.0 * (2 * 10000 + 3 * 3000 + 2 * 1000) + 4.0 * (3000 + 3 * 1000)
    # budget for two slots only, although four are allowed per shape
    eng, srv = _engine(monkeypatch, shapes, budget=2.5 * one_slot, max_slots=4, work_polls=5)
    assert len(eng.slots[0]) == 2
    peak = {"n": 0}
    orig = srv.submit

    def submit(plan, x, c):
        t = orig(plan, x, c)
        peak["n"] = max(peak["n"], len(srv.in_flight_handles))
        assert eng.in_flight_bytes <= eng.budget
        return t

    srv.submit = submit
    reqs = [(0.0, 0, "in") for _ in range(9)]
    res = eng.run(reqs, {"in": "x"}, [f"o{i}" for i in range(9)], timeout_s=30)
    assert all(r is not None for r in res)
    assert peak["n"] == 2


def test_run_times_out_when_nothing_finishes(monkeypatch):
    shapes = [_shape(10)]
    eng, srv = _engine(monkeypatch, shapes, budget=1e9, max_slots=1, work_polls=10**9)
    with pytest.raises(TimeoutError):
        eng.run([(0.0, 0, "in")], {"in": "x"}, ["o"], timeout_s=0.2)


class _FailingServer(_FakeServer):
    """The launch abandons its jobs after the `fail_after`-th poll: the job in
    progress is reported finished with FCT_ERR_TIMEOUT, and every later poll
    of an unfinished job raises the launch's error (as fct_server_poll does
    once the device has published an error in the ring)."""

    def __init__(self, work_polls, fail_after):
        super().__init__(work_polls)
        self.polls = 0
        self.fail_after = fail_after
        self.failed = False

    def poll(self, t):
        self.polls += 1
        if self.polls >= self.fail_after and not self.failed:
            self.failed = True
            self.jobs[t][0] = 0
            if self.jobs[t][1] in self.in_flight_handles:
                self.in_flight_handles.remove(self.jobs[t][1])
            return {"status": 4, "iterations": 0, "refinements": 0, "rel_normal_residual": 0.0, "gamma0": 0.0}
        if self.failed and self.jobs[t][0] > 0:
            raise RuntimeError("FCT_ERR_TIMEOUT: the serving launch abandoned its jobs after a device-side error")
        return super().poll(t)


def test_device_error_ends_the_run_promptly(monkeypatch):
    shapes = [_shape(50)]
    srv = _FailingServer(work_polls=4, fail_after=3)
    fake = types.SimpleNamespace(
        Plan=_FakePlan,
        fct_server_create=lambda *a: srv,
        fct_server_submit=lambda s, plan, x, c: s.submit(plan, x, c),
        fct_server_poll=lambda s, t: s.poll(t),
        fct_server_destroy=lambda s: None,
    )
    monkeypatch.setattr(serving, "F", fake)
    eng = serving.ServingEngine(shapes, hbm_budget_bytes=1e9, max_slots_per_shape=3)
    import time
    t0 = time.perf_counter()
    with pytest.raises(RuntimeError, match="device-side error"):
        eng.run([(0.0, 0, "in") for _ in range(6)], {"in": "x"}, [f"o{i}" for i in range(6)], timeout_s=30)
    assert time.perf_counter() - t0 < 5.0   # the error ends the run, not the run's own time limit


def test_failed_job_report_reaches_the_summary(monkeypatch):
    """A job the device reports finished with an error status is counted as
    not converged by the latency summary."""
    shapes = [_shape(50)]
    srv = _FailingServer(work_polls=2, fail_after=10**9)
    orig = srv.poll

    def poll(t):
        rep = orig(t)
        if rep is not None and t == 1:
            rep = dict(rep, status=4)
        return rep

    srv.poll = poll
    fake = types.SimpleNamespace(
        Plan=_FakePlan,
        fct_server_create=lambda *a: srv,
        fct_server_submit=lambda s, plan, x, c: s.submit(plan, x, c),
        fct_server_poll=lambda s, t: s.poll(t),
        fct_server_destroy=lambda s: None,
    )
    monkeypatch.setattr(serving, "F", fake)
    eng = serving.ServingEngine(shapes, hbm_budget_bytes=1e9, max_slots_per_shape=2)
    res = eng.run([(0.0, 0, "in") for _ in range(3)], {"in": "x"}, ["a", "b", "c"], timeout_s=30)
    summ = serving.latency_summary(res, [50] * 3)
    assert not summ["all_converged"]
    assert sorted(r["report"]["status"] for r in res) == [0, 0, 4]


def test_lazy_plans_are_built_on_first_request_and_counted_cold(monkeypatch):
    """lazy_plans: no plan exists before its shape's first request; that
    request is reported cold, later ones of the shape are not, and clones are
    made on demand within the budget."""
    shapes = [_shape(100), _shape(200)]
    srv = _FakeServer(2)
    fake = types.SimpleNamespace(
        Plan=_FakePlan,
        fct_server_create=lambda *a: srv,
        fct_server_submit=lambda s, plan, x, c: s.submit(plan, x, c),
        fct_server_poll=lambda s, t: s.poll(t),
        fct_server_destroy=lambda s: None,
    )
    monkeypatch.setattr(serving, "F", fake)
    eng = serving.ServingEngine(shapes, hbm_budget_bytes=1e9, max_slots_per_shape=3, lazy_plans=True)
    assert eng.plans == [None, None]
    reqs = [(0.0, 1, "b"), (0.0, 1, "b"), (0.0, 1, "b"), (0.05, 0, "a")]
    res = eng.run(reqs, {"a": "xa", "b": "xb"}, ["o0", "o1", "o2", "o3"], timeout_s=30)
    assert res[0]["cold"] and res[3]["cold"]
    assert not res[1]["cold"] and not res[2]["cold"]
    assert eng.plans[0] is not None and eng.plans[1] is not None
    assert len(eng.slots[1]) == 3          # base plan + two clones made on demand
    assert set(eng.plan_build_s) == {0, 1}
    assert eng.used_bytes <= eng.budget
