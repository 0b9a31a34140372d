"""Serving with continuous batching: results in the mix equal results alone,
and work submitted while other work runs joins it on the device."""
import time

import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O
from paper_2309_14584_gb300.serving import ServingEngine, latency_summary

pytestmark = pytest.mark.gpu


def _shapes():
    # small shapes of several dimensions (N ~ 1e3) so the test stays short
    return [W.make_workload(f"s{D}", 70 + D, D, d, 3 * D, 1, d + 1, W.FAMILY_GAUSSCOS, tol=1e-12, precision="mixed")
            for D, d in ((2, 40), (3, 15), (4, 9), (6, 6))]


def test_served_results_equal_results_alone():
    shapes = _shapes()
    eng = ServingEngine(shapes, max_slots_per_shape=3, team_blocks=8, precision=F.FCT_MIXED, tol=1e-12,
                        inner_tol=1e-5)
    rng = np.random.default_rng(0)
    inputs = {}
    for s, w in enumerate(shapes):
        for v in range(3):
            x = torch.empty(eng.plans[s].M, dtype=torch.float64, device="cuda")
            eng.plans[s].sample(W.FAMILY_GAUSSCOS, W.gausscos_params(1000 * s + v, w.D), x)
            inputs[(s, v)] = x
    torch.cuda.synchronize()
    # a burst: everything arrives at once and is admitted as slots free up
    reqs = [(0.0, int(rng.integers(0, len(shapes))), None) for _ in range(30)]
    reqs = [(t, s, (s, i % 3)) for i, (t, s, _) in enumerate(reqs)]
    outs = [torch.full((eng.plans[s].N,), float("nan"), dtype=torch.float64, device="cuda") for _, s, _ in reqs]
    res = eng.run(reqs, inputs, outs, timeout_s=120)
    summ = latency_summary(res, [eng.plans[s].N for _, s, _ in reqs])
    assert summ["all_converged"]
    F.fct_server_destroy(eng.server)
    eng.server = None
    for (t, s, key), o in zip(reqs, outs):
        alone = torch.empty_like(o)
        assert eng.plans[s].execute(inputs[key], alone)["status"] == 0
        assert torch.equal(alone, o)
    eng.close()


def test_jobs_submitted_while_others_run_join_them():
    """A long transform is submitted first; short ones submitted while it runs
    finish before it (they run on other teams of the same launch)."""
    long_w = W.config_d10_rational()
    short = _shapes()[:2]
    pl = F.Plan(long_w.support, long_w.sizes, long_w.nodes, precision=F.FCT_FP64, tol=1e-13)
    ps = [F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5) for w in short]
    xl = torch.empty(pl.M, dtype=torch.float64, device="cuda")
    pl.sample(long_w.family, long_w.params, xl)
    xs = []
    for p, w in zip(ps, short):
        x = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(W.FAMILY_GAUSSCOS, W.gausscos_params(7, w.D), x)
        xs.append(x)
    ol = torch.empty(pl.N, dtype=torch.float64, device="cuda")
    osh = [torch.empty(p.N, dtype=torch.float64, device="cuda") for p in ps]
    torch.cuda.synchronize()
    srv = F.fct_server_create(0, 16, 0, 0.2)
    tl = F.fct_server_submit(srv, pl.handle, xl, ol)
    time.sleep(0.002)
    ts = [F.fct_server_submit(srv, p.handle, x, o) for p, x, o in zip(ps, xs, osh)]
    order = []
    pending = {tl: "long", ts[0]: "short0", ts[1]: "short1"}
    t0 = time.time()
    while pending and time.time() - t0 < 60:
        for t in list(pending):
            r = F.fct_server_poll(srv, t)
            if r is not None:
                assert r["status"] == 0
                order.append(pending.pop(t))
    assert not pending
    assert order[-1] == "long", order
    F.fct_server_destroy(srv)
    for p in ps + [pl]:
        p.close()


def test_plans_built_while_the_server_runs_are_served():
    """Plans are built on a stream of their own, so a plan created while a
    serving launch holds part of the device is served at once (a plan-cache
    miss), with the coefficients of the same transform alone.  Plans and
    servers of one block size use one shared-memory limit, so a plan built
    later cannot lower the running server's launch limit."""
    long_w = W.config_d10_rational()
    pl = F.Plan(long_w.support, long_w.sizes, long_w.nodes, precision=F.FCT_FP64, tol=1e-13)
    xl = torch.empty(pl.M, dtype=torch.float64, device="cuda")
    pl.sample(long_w.family, long_w.params, xl)
    ol = torch.empty(pl.N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    srv = F.fct_server_create(0, 16, 4, 0.2)  # 4 teams of 16 blocks: most SMs stay free
    tl = F.fct_server_submit(srv, pl.handle, xl, ol)
    jobs = []
    for i, w in enumerate(_shapes()):
        p = F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)
        x = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(W.FAMILY_GAUSSCOS, W.gausscos_params(40 + i, w.D), x)
        o = torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        jobs.append((p, x, o, F.fct_server_submit(srv, p.handle, x, o)))
    for _, _, _, t in jobs:
        assert F.fct_server_wait(srv, t, 60.0)["status"] == 0
    assert F.fct_server_wait(srv, tl, 120.0)["status"] == 0
    F.fct_server_destroy(srv)
    for p, x, o, _ in jobs:
        alone = torch.empty_like(o)
        assert p.execute(x, alone)["status"] == 0
        assert torch.equal(alone, o)
        p.close()
    alone = torch.empty_like(ol)
    assert pl.execute(xl, alone)["status"] == 0
    assert torch.equal(alone, ol)
    pl.close()


def test_teams_stay_while_a_long_job_runs():
    """The server is left idle longer than its idle timeout while one long
    transform runs on one team; short jobs submitted afterwards still run on
    the other teams and finish first (no team left the launch)."""
    long_w = W.config_d10_rational()
    short = _shapes()
    pl = F.Plan(long_w.support, long_w.sizes, long_w.nodes, precision=F.FCT_FP64, tol=1e-13)
    ps = [F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5) for w in short]
    xl = torch.empty(pl.M, dtype=torch.float64, device="cuda")
    pl.sample(long_w.family, long_w.params, xl)
    xs = []
    for p, w in zip(ps, short):
        x = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(W.FAMILY_GAUSSCOS, W.gausscos_params(11, w.D), x)
        xs.append(x)
    ol = torch.empty(pl.N, dtype=torch.float64, device="cuda")
    osh = [torch.empty(p.N, dtype=torch.float64, device="cuda") for p in ps]
    torch.cuda.synchronize()
    srv = F.fct_server_create(0, 8, 0, 0.01)
    tl = F.fct_server_submit(srv, pl.handle, xl, ol)
    time.sleep(0.05)  # five idle timeouts with only the long job on the device
    ts = [F.fct_server_submit(srv, p.handle, x, o) for p, x, o in zip(ps, xs, osh)]
    order = []
    pending = {tl: "long", **{t: f"short{i}" for i, t in enumerate(ts)}}
    t0 = time.time()
    while pending and time.time() - t0 < 60:
        for t in list(pending):
            r = F.fct_server_poll(srv, t)
            if r is not None:
                assert r["status"] == 0
                order.append(pending.pop(t))
    assert not pending
    assert order[-1] == "long", order
    F.fct_server_destroy(srv)
    for p in ps + [pl]:
        p.close()


def test_served_results_match_the_oracle():
    """Gaussian-cosine requests over shapes of D = 2 .. 20, served in one
    burst (several teams at once), each result against the oracle's
    least-squares solution of the same seeded problem at the mixed-path bar."""
    shapes = [W.make_workload(f"s{D}", 70 + D, D, d, 3 * D, 1, d + 1, W.FAMILY_GAUSSCOS, tol=1e-12, precision="mixed")
              for D, d in ((2, 40), (3, 15), (4, 9), (6, 6), (12, 3), (20, 2))]
    eng = ServingEngine(shapes, max_slots_per_shape=2, team_blocks=8, precision=F.FCT_MIXED, tol=1e-12,
                        inner_tol=1e-4)
    inputs = {}
    for s, w in enumerate(shapes):
        for v in range(2):
            x = torch.empty(eng.plans[s].M, dtype=torch.float64, device="cuda")
            eng.plans[s].sample(W.FAMILY_GAUSSCOS, W.gausscos_params(500 + 10 * s + v, w.D), x)
            inputs[(s, v)] = x
    torch.cuda.synchronize()
    reqs = [(0.0, s, (s, v)) for v in range(2) for s in range(len(shapes))]
    outs = [torch.empty(eng.plans[s].N, dtype=torch.float64, device="cuda") for _, s, _ in reqs]
    res = eng.run(reqs, inputs, outs, timeout_s=120)
    eng.close()
    assert all(r["report"]["status"] == 0 for r in res)
    for (t, s, (_, v)), o in zip(reqs, outs):
        w = shapes[s]
        params = W.gausscos_params(500 + 10 * s + v, w.D)
        f = O.sample_lgrid(W.FAMILY_GAUSSCOS, params, w.support, w.sizes, w.nodes)
        ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
        err = float(np.linalg.norm(o.cpu().numpy() - ref) / np.linalg.norm(ref))
        assert err <= 1e-10, (w.name, v, err)
