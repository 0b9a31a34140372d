"""Algorithm 2 on the device: the Lanczos condition estimate of
fct_plan_condition and the grid-count selection built on it, against the
oracle's exact kappa (singular values) and its Algorithm 2 loop."""
import math

import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O
from paper_2309_14584_gb300 import lgrid

pytestmark = pytest.mark.gpu

D3 = (3, 4)  # D, d: N = 35


def _cands(seed=14, K=24):
    D, d = D3
    sup = W.total_degree_support(D, d)
    sizes, nodes = W.l_grid(seed, sup.shape[0], D, K, 2, d + 1)
    return sup, sizes, nodes


def _start(N, seed=0):
    z = W.stream(seed, "probe").standard_normal(N)
    return torch.from_numpy(z).cuda()


@pytest.mark.parametrize("L", [6, 9, 16, 24])
def test_condition_estimate_matches_singular_values(L):
    sup, sizes, nodes = _cands()
    A = O.AliasSystem(sup, sizes[:L], nodes[:L]).A.toarray()
    sv = np.linalg.svd(A, compute_uv=False)
    p = F.Plan(sup, sizes[:L], nodes[:L])
    z = _start(p.N)
    r = F.fct_plan_condition(p.handle, z, torch.empty_like(z), p.N)
    p.close()
    assert r["iterations"] >= 2
    assert r["lambda_max"] == pytest.approx(sv[0] ** 2, rel=1e-5)
    assert r["lambda_min"] == pytest.approx(sv[-1] ** 2, rel=1e-4)
    assert r["kappa"] == pytest.approx(sv[0] / sv[-1], rel=1e-4)


def test_condition_estimate_larger_case_is_a_tight_lower_bound():
    """D2 d16 (N = 153), 4 grids of 9..33 points per axis: 150 Lanczos steps
    bound kappa from below and within 2 %."""
    w = W.config_small_poly()
    A = O.AliasSystem(w.support, w.sizes, w.nodes).A.toarray()
    sv = np.linalg.svd(A, compute_uv=False)
    kappa = sv[0] / sv[-1]
    p = F.Plan(w.support, w.sizes, w.nodes)
    z = _start(p.N, 1)
    r = F.fct_plan_condition(p.handle, z, torch.empty_like(z), 150)
    p.close()
    assert r["kappa"] <= kappa * (1 + 1e-4)
    assert r["kappa"] >= kappa * 0.98


def test_condition_estimate_sees_a_null_space():
    """All grids share one single-point node at x = 1 on axis 0: A has more
    rows than columns but loses rank, and the random start vector exposes the
    zero singular value."""
    D, d = 2, 3
    sup = W.total_degree_support(D, d)
    sizes = np.array([[1, 5], [1, 4], [1, 6]], dtype=np.int32)
    nodes = np.ones((3, D))
    assert O.AliasSystem(sup, sizes, nodes).R >= sup.shape[0]
    assert O.condition_number(O.AliasSystem(sup, sizes, nodes).A) == math.inf
    r = lgrid.probe_condition(sup, sizes, nodes, iterations=sup.shape[0] + 1)
    assert r["kappa"] > 1e4


def test_condition_of_a_collision_free_grid_is_one():
    d = 9
    sup = np.arange(d + 1, dtype=np.uint16).reshape(-1, 1)
    r = lgrid.probe_condition(sup, np.array([[d + 1]], dtype=np.int32), np.ones((1, 1)), iterations=8)
    assert r["kappa"] == pytest.approx(1.0, abs=1e-5)


@pytest.mark.parametrize("kappa0", [1e3, 6.0, 4.6])
@pytest.mark.parametrize("step", [1, 4])
def test_select_grids_matches_oracle_algorithm2(kappa0, step):
    sup, sizes, nodes = _cands()
    L_ref, k_ref = O.construct_alias_system(sup, sizes, nodes, kappa0)
    r = lgrid.select_grids(sup, sizes, nodes, kappa0=kappa0, step=step, probe_iterations=sup.shape[0] + 1)
    assert r["L"] == L_ref
    assert r["kappa"] == pytest.approx(k_ref, rel=1e-3)


def test_select_grids_reports_exhaustion():
    sup, sizes, nodes = _cands(K=8)
    r = lgrid.select_grids(sup, sizes, nodes, kappa0=2.0, step=3, probe_iterations=36)
    assert r["L"] is None and r["kappa"] > 2.0


def test_condition_estimate_past_convergence_stays_exact():
    """More probe iterations than CG needs to converge (D=4, degree 8, 12
    grids: converged in well under 100): the estimate must not drift once the
    residual is tiny (it stops at a 1e12 reduction)."""
    sup = W.total_degree_support(4, 8)
    sizes, nodes = W.l_grid(21, sup.shape[0], 4, 12, 1, 9)
    A = O.AliasSystem(sup, sizes, nodes).A.toarray()
    sv = np.linalg.svd(A, compute_uv=False)
    r = lgrid.probe_condition(sup, sizes, nodes, iterations=400)
    assert r["iterations"] < 400
    assert r["kappa"] == pytest.approx(sv[0] / sv[-1], rel=1e-3)


def test_rank_check_refuses_a_rank_deficient_plan():
    """fct_options.kappa_max: the plan of the rank-deficient L-grid above (all
    grids share the single-point node x = 1) is refused with FCT_ERR_RANK; the
    same support on grids that separate it is accepted, with an estimate that
    agrees with the oracle's exact kappa."""
    D, d = 2, 3
    sup = W.total_degree_support(D, d)
    sizes = np.array([[1, 5], [1, 4], [1, 6]], dtype=np.int32)
    with pytest.raises(F.FctError) as e:
        F.Plan(sup, sizes, np.ones((3, D)), kappa_max=1e4)
    assert e.value.status == F.fct.FCT_ERR_RANK
    sup, sizes, nodes = _cands()
    p = F.Plan(sup, sizes[:16], nodes[:16], kappa_max=1e4)
    k = p.info["kappa_estimate"]
    p.close()
    exact = O.condition_number(O.AliasSystem(sup, sizes[:16], nodes[:16]).A)
    assert 1.0 <= k <= exact * (1 + 1e-6) and k >= 0.9 * exact
    p = F.Plan(sup, sizes[:16], nodes[:16])            # no check: no estimate
    assert p.info["kappa_estimate"] == 0.0
    p.close()
    with pytest.raises(F.FctError) as e:                 # every kappa is >= 1
        F.Plan(sup, sizes[:16], nodes[:16], kappa_max=0.5)
    assert e.value.status == F.fct.FCT_ERR_RANK


def test_rank_check_option_is_validated():
    sup, sizes, nodes = _cands()
    with pytest.raises(F.FctError) as e:
        F.Plan(sup, sizes[:16], nodes[:16], kappa_max=-1.0)
    assert e.value.status == F.fct.FCT_ERR_INVALID_ARG
