"""Evaluation of the expansion at arbitrary points on the device
(fct_evaluate) against the oracle's term-by-term definition."""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu

CASES = [(1, 40, 300), (2, 253, 30), (6, 10, 200), (20, 3, 100), (3, 6, 1000)]


@pytest.mark.parametrize("D,d,P", CASES, ids=[f"D{c[0]}_d{c[1]}" for c in CASES])
def test_evaluate_matches_oracle(D, d, P):
    sup = W.total_degree_support(D, d)
    sizes, nodes = W.l_grid(80 + D, sup.shape[0], D, 2, 1, d + 1)
    plan = F.Plan(sup, sizes, nodes)
    g = W.stream(90 + D, "probe")
    c = W.poly_coefficients(90 + D, sup)
    pts = g.uniform(-1.0, 1.0, (P, D))
    vals = torch.full((P,), float("nan"), dtype=torch.float64, device="cuda")
    plan.evaluate(torch.from_numpy(c).cuda(), torch.from_numpy(pts).cuda(), vals)
    torch.cuda.synchronize()
    plan.close()
    ref = O.evaluate_expansion(c, sup, pts)
    assert np.max(np.abs(vals.cpu().numpy() - ref)) <= 1e-12 * np.abs(c).sum()


def test_evaluate_zero_points_is_a_noop():
    sup = W.total_degree_support(2, 3)
    plan = F.Plan(sup, np.array([[4, 4]], dtype=np.int32))
    F.fct_evaluate(plan.handle, torch.zeros(sup.shape[0], dtype=torch.float64, device="cuda"),
                   torch.zeros((0, 2), dtype=torch.float64, device="cuda"),
                   torch.zeros(1, dtype=torch.float64, device="cuda"))
    plan.close()


def test_solve_then_evaluate_reproduces_the_polynomial():
    """A seeded polynomial sampled on the D=6, degree-10 L-grid, solved (mixed)
    and evaluated at 500 random points equals the polynomial there."""
    w = W.config_d6_gausscos(family=W.FAMILY_POLY)
    plan = F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)
    x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, x)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    assert plan.execute(x, c)["status"] == 0
    pts = W.stream(5, "probe").uniform(-1.0, 1.0, (500, w.D))
    vals = torch.empty(500, dtype=torch.float64, device="cuda")
    plan.evaluate(c, torch.from_numpy(pts).cuda(), vals)
    torch.cuda.synchronize()
    plan.close()
    ref = O.evaluate_expansion(w.coeffs_true, w.support, pts)
    assert np.max(np.abs(vals.cpu().numpy() - ref)) <= 1e-10 * np.abs(w.coeffs_true).sum()
