"""The paper's own grid on the device (fct_options.grid_kind =
FCT_GRID_FIRST_KIND): first-kind points, 1/n DCT-II quadrature and signed
half-weight alias entries, against the oracle's first-kind form."""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11
TOL_MIXED = 1e-10
FK = F.FCT_GRID_FIRST_KIND

CASES = [
    # name, seed, D, d, K, lo, hi, family -- all full rank on first-kind grids
    ("D1_poly", 61, 1, 14, 6, 4, 11, W.FAMILY_POLY),
    ("D2_gc", 62, 2, 9, 5, 2, 8, W.FAMILY_GAUSSCOS),
    ("D3_rat", 63, 3, 5, 9, 1, 6, W.FAMILY_RATIONAL),
    ("D4_polygc", 64, 4, 4, 12, 1, 5, W.FAMILY_POLY_GAUSSCOS),
]


def _w(case):
    name, seed, D, d, K, lo, hi, fam = case
    return W.make_workload(name, seed, D, d, K, lo, hi, fam)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_first_kind_sampler_matches_oracle(case):
    w = _w(case)
    plan = F.Plan(w.support, w.sizes, w.nodes, grid_kind=FK)
    s = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, s)
    ref = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes, kind="first")
    got = s.cpu().numpy()
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(got - ref)) <= 1e-13 * scale
    if w.family in (W.FAMILY_POLY, W.FAMILY_POLY_GAUSSCOS):
        sf = torch.empty_like(s)
        plan.sample(w.family | F.fct.FCT_SAMPLE_FOLDED, w.params, sf)
        assert np.max(np.abs(sf.cpu().numpy() - ref)) <= 1e-12 * scale
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_first_kind_solve_matches_oracle(case, precision):
    w = _w(case)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes, kind="first")
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr", kind="first")
    opts = (dict(precision=F.FCT_FP64, tol=1e-14) if precision == "fp64"
            else dict(precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5))
    plan = F.Plan(w.support, w.sizes, w.nodes, grid_kind=FK, **opts)
    x = torch.from_numpy(f).cuda()
    c = torch.full((plan.N,), float("nan"), dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    got = c.cpu().numpy()
    tol = TOL_FP64 if precision == "fp64" else TOL_MIXED
    assert rep["status"] == 0, rep
    assert rel(got, ref) <= tol, (rel(got, ref), rep)
    if w.coeffs_true is not None:
        assert rel(got, w.coeffs_true) <= tol


def test_first_kind_d6_matches_oracle_and_differs_from_extrema():
    """Full-size D=6, degree 10 Gaussian-cosine on the first-kind form of the
    same L-grid: FP64 and mixed within tolerance of the oracle's weighted
    least squares (which is not the extrema-grid answer: the targets are not
    polynomials, so grid and weighting change c*)."""
    w = W.config_d6_gausscos()
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes, kind="first")
    ref = O.fct(w.support, w.sizes, w.nodes, f, "csne", kind="first")
    x = torch.from_numpy(f).cuda()
    # kappa(A) is ~160 on this form (~10 on the extrema grid): the normal
    # residual tolerances are tightened accordingly
    for opts, tol in ((dict(precision=F.FCT_FP64, tol=1e-15), TOL_FP64),
                      (dict(precision=F.FCT_MIXED, tol=1e-14, inner_tol=1e-5), TOL_MIXED)):
        plan = F.Plan(w.support, w.sizes, w.nodes, grid_kind=FK, **opts)
        c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
        rep = plan.execute(x, c)
        plan.close()
        assert rep["status"] == 0, rep
        assert rel(c.cpu().numpy(), ref) <= tol
    f_ext = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref_ext = O.fct(w.support, w.sizes, w.nodes, f_ext, "csne")
    assert rel(ref, ref_ext) > 1e-8


def test_first_kind_d6_poly_exact_recovery_with_device_samples():
    w = W.config_d6_gausscos(family=W.FAMILY_POLY)
    plan = F.Plan(w.support, w.sizes, w.nodes, grid_kind=FK, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)
    x = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family | F.fct.FCT_SAMPLE_FOLDED, w.params, x)
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    assert rep["status"] == 0
    assert rel(c.cpu().numpy(), w.coeffs_true) <= TOL_MIXED
