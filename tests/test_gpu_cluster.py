"""The cluster solver of the mixed path (fct_options.cluster_solve = 1): one
thread-block cluster holds the FP32 tables and the Krylov vectors in
distributed shared memory.  Compared with the FP64 oracle and with the team
solver; bit-reproducible run to run."""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-10
MIXED = dict(precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5, cluster_solve=1)

CASES = [
    ("D2_gc", 41, 2, 9, 5, 3, 12, W.FAMILY_GAUSSCOS),
    ("D3_rat", 42, 3, 6, 9, 1, 7, W.FAMILY_RATIONAL),
    ("D4_gc", 43, 4, 5, 12, 1, 6, W.FAMILY_GAUSSCOS),
    ("D4_polygc", 44, 4, 4, 12, 1, 5, W.FAMILY_POLY_GAUSSCOS),
    ("D5_rat", 45, 5, 4, 15, 1, 5, W.FAMILY_RATIONAL),
]


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _run(w, f, **opts):
    plan = F.Plan(w.support, w.sizes, w.nodes, **opts)
    x = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    c = torch.full((plan.N,), float("nan"), dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    c2 = torch.full_like(c, float("nan"))
    rep2 = plan.execute(x, c2)
    info = plan.info
    plan.close()
    return c.cpu().numpy(), c2.cpu().numpy(), rep, rep2, info


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_cluster_solver_matches_oracle(case):
    name, seed, D, d, K, lo, hi, fam = case
    w = W.make_workload(name, seed, D, d, K, lo, hi, fam)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    got, again, rep, rep2, info = _run(w, f, **MIXED)
    assert info["cluster_blocks"] in (8, 16)
    assert rep["status"] == 0, rep
    assert rel(got, ref) <= TOL_MIXED, (rel(got, ref), rep)
    assert np.array_equal(got, again) and rep == rep2


def test_cluster_solver_d6_matches_oracle_and_team_solver():
    w = W.config_d6_gausscos()
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "csne")
    got, again, rep, _, info = _run(w, f, **MIXED)
    assert info["cluster_blocks"] == 16, info
    assert rep["status"] == 0, rep
    assert rel(got, ref) <= TOL_MIXED, (rel(got, ref), rep)
    assert np.array_equal(got, again)
    team, _, rep_t, _, info_t = _run(w, f, **dict(MIXED, cluster_solve=0))
    assert info_t["cluster_blocks"] == 0
    assert rel(got, team) <= TOL_MIXED


def test_cluster_solver_d6_poly_exact_recovery():
    w = W.config_d6_gausscos(family=W.FAMILY_POLY)
    plan = F.Plan(w.support, w.sizes, w.nodes, **MIXED)
    x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, x)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    assert rep["status"] == 0
    assert rel(c.cpu().numpy(), w.coeffs_true) <= TOL_MIXED


def test_cluster_solver_fp64_continuation():
    """One refinement sweep allowed: the cluster solver finishes in FP64 CG
    from the current x and still meets the oracle."""
    name, seed, D, d, K, lo, hi, fam = CASES[2]
    w = W.make_workload(name, seed, D, d, K, lo, hi, fam)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    got, _, rep, _, _ = _run(w, f, **dict(MIXED, max_refine=1, tol=1e-13))
    assert rep["status"] == 0 and rep["refinements"] == 1, rep
    assert rel(got, ref) <= TOL_MIXED


def test_cluster_solver_reports_nonfinite_samples():
    name, seed, D, d, K, lo, hi, fam = CASES[0]
    w = W.make_workload(name, seed, D, d, K, lo, hi, fam)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    f[3] = np.nan
    plan = F.Plan(w.support, w.sizes, w.nodes, **MIXED)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FctError) as e:
        plan.execute(torch.from_numpy(f).cuda(), c)
    assert "NONFINITE" in str(e.value)
    plan.close()
