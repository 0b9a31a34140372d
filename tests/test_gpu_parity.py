"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: the FP64 path must match the oracle's least-squares solution to
1e-11 relative l2 error, the mixed path (FP32 inner solves, FP64 refinement)
to 1e-10; integer alias tables bit-exactly (test_capi_host.py); samples to
1e-13 absolute (O(1) values, device vs host transcendental functions).
"""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-11
TOL_MIXED = 1e-10


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_run(w, samples_np=None, **opts):
    plan = F.Plan(w.support, w.sizes, w.nodes, **opts)
    samples = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    if samples_np is None:
        plan.sample(w.family, w.params, samples)
    else:
        samples.copy_(torch.from_numpy(np.ascontiguousarray(samples_np)))
    coeffs = torch.full((plan.N,), float("nan"), dtype=torch.float64, device="cuda")
    rep = plan.execute(samples, coeffs)
    torch.cuda.synchronize()
    out = coeffs.cpu().numpy()
    s = samples.cpu().numpy()
    plan.close()
    return out, s, rep


SMALL = [
    # name, seed, D, d, K, lo, hi, family
    ("D1_poly", 21, 1, 12, 5, 2, 9, W.FAMILY_POLY),
    ("D2_gc", 41, 2, 9, 5, 3, 12, W.FAMILY_GAUSSCOS),
    ("D3_rat", 42, 3, 6, 9, 1, 7, W.FAMILY_RATIONAL),
    ("D4_gc", 43, 4, 5, 12, 1, 6, W.FAMILY_GAUSSCOS),
    ("D4_polygc", 44, 4, 4, 12, 1, 5, W.FAMILY_POLY_GAUSSCOS),
    ("D5_rat", 45, 5, 4, 15, 1, 5, W.FAMILY_RATIONAL),
]


def _small(case):
    name, seed, D, d, K, lo, hi, fam = case
    return W.make_workload(name, seed, D, d, K, lo, hi, fam)


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_sampler_matches_oracle(case):
    w = _small(case)
    _, s_gpu, _ = gpu_run(w)
    s_ref = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    assert s_gpu.shape == s_ref.shape
    assert np.max(np.abs(s_gpu - s_ref)) <= 1e-13 * max(1.0, np.max(np.abs(s_ref)))


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_fp64_small_matches_oracle(case):
    """Same samples on both sides (the oracle's own); the solve is compared."""
    w = _small(case)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    got, _, rep = gpu_run(w, samples_np=f, tol=1e-14)
    assert rep["status"] == 0
    assert rel(got, ref) <= TOL_FP64, (rel(got, ref), rep)
    if w.coeffs_true is not None:
        assert rel(got, w.coeffs_true) <= TOL_FP64


def test_config_small_poly_recovers_and_matches_oracle():
    w = W.config_small_poly()
    got, s_gpu, rep = gpu_run(w, tol=1e-13)
    ref = O.fct(w.support, w.sizes, w.nodes, O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes), "qr")
    assert rep["status"] == 0
    assert rel(got, ref) <= TOL_FP64
    assert rel(got, w.coeffs_true) <= TOL_FP64


@pytest.fixture(scope="module")
def d6_gausscos():
    w = W.config_d6_gausscos()
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "csne")
    return w, f, ref


def test_d6_fp64_matches_oracle(d6_gausscos):
    w, f, ref = d6_gausscos
    got, s_gpu, rep = gpu_run(w, tol=1e-13)
    assert rep["status"] == 0, rep
    assert np.max(np.abs(s_gpu - f)) <= 1e-13
    assert rel(got, ref) <= TOL_FP64, (rel(got, ref), rep)


def test_d6_mixed_matches_oracle(d6_gausscos):
    w, f, ref = d6_gausscos
    got, _, rep = gpu_run(w, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)
    assert rep["status"] == 0, rep
    assert rel(got, ref) <= TOL_MIXED, (rel(got, ref), rep)


def test_d6_poly_exact_recovery():
    """Seeded polynomial on the D=6, d=10 support sampled on the GPU: the
    solve returns the true coefficients (consistent system)."""
    w = W.config_d6_gausscos(family=W.FAMILY_POLY)
    got, _, rep = gpu_run(w, tol=1e-13)
    assert rep["status"] == 0
    assert rel(got, w.coeffs_true) <= TOL_FP64, rel(got, w.coeffs_true)


def test_execute_host_equals_device():
    w = _small(SMALL[3])
    plan = F.Plan(w.support, w.sizes, w.nodes)
    samples = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, samples)
    c_dev = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    plan.execute(samples, c_dev)
    s_host = samples.cpu().pin_memory()
    c_host = torch.empty(plan.N, dtype=torch.float64).pin_memory()
    rep = plan.execute_host(s_host, c_host)
    assert rep["status"] == 0
    assert torch.equal(c_host, c_dev.cpu())
    plan.close()


def test_batch_bitwise_equals_alone():
    ws = [_small(c) for c in SMALL[1:]] + [W.config_small_poly()]
    plans, samples, alone = [], [], []
    for w in ws:
        p = F.Plan(w.support, w.sizes, w.nodes, tol=1e-13)
        s = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(w.family, w.params, s)
        c = torch.empty(p.N, dtype=torch.float64, device="cuda")
        p.execute(s, c)
        plans.append(p)
        samples.append(s)
        alone.append(c.clone())
    outs = [torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda") for p in plans]
    for team_blocks in (1, 3, 0):
        reps = F.fct_execute_batch([p.handle for p in plans], samples, outs, team_blocks=team_blocks)
        assert all(r["status"] == 0 for r in reps)
        for a, o in zip(alone, outs):
            assert torch.equal(a, o)
    for p in plans:
        p.close()


@pytest.mark.parametrize("bt,lanes,blocks", [(128, 1, 0), (256, 4, 7), (512, 16, 0), (256, 2, 1)])
def test_launch_shapes_agree(bt, lanes, blocks):
    w = _small(SMALL[3])
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    got, _, rep = gpu_run(w, samples_np=f, tol=1e-14, block_threads=bt, coef_lanes=lanes, max_blocks=blocks)
    assert rep["status"] == 0
    assert rel(got, ref) <= TOL_FP64


@pytest.mark.parametrize("epl", [2, 4, 8])
def test_entries_per_lane_agree(epl):
    """Fixed gather granularity (fewer, longer row units) gives the same
    answer as the automatic choice, within tolerance of the oracle."""
    w = _small(SMALL[4])
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    for prec in (F.FCT_FP64, F.FCT_MIXED):
        got, _, rep = gpu_run(w, samples_np=f, tol=1e-14 if prec == F.FCT_FP64 else 1e-12, inner_tol=1e-5,
                              precision=prec, entries_per_lane=epl, coef_lanes=1)
        assert rep["status"] == 0
        assert rel(got, ref) <= (TOL_FP64 if prec == F.FCT_FP64 else TOL_MIXED)


def test_edge_single_coefficient_and_single_point_grid():
    """N = 1 (support {0}) on grids that are single points: c* = mean-free LS
    of the constant, i.e. the average of the samples weighted as one row per grid."""
    support = np.zeros((1, 3), dtype=np.uint16)
    sizes = np.ones((3, 3), dtype=np.int32)
    nodes = np.array([[0.1, 0.2, 0.3], [-0.5, 0.5, 0.0], [0.9, -0.9, 0.4]])
    plan = F.Plan(support, sizes, nodes)
    assert plan.M == 3
    samples = torch.tensor([1.0, 2.0, 4.0], dtype=torch.float64, device="cuda")
    c = torch.empty(1, dtype=torch.float64, device="cuda")
    rep = plan.execute(samples, c)
    assert rep["status"] == 0
    assert abs(c.item() - 7.0 / 3.0) <= 1e-15
    plan.close()


def test_edge_ragged_and_one_dimensional():
    """D = 1 with ragged grid sizes; compared with the oracle."""
    support = np.arange(40, dtype=np.uint16)[:, None]
    sizes = np.array([[7], [12], [5], [33], [2], [1]], dtype=np.int32)
    nodes = np.full((6, 1), 0.37)
    f = np.random.default_rng(3).standard_normal(int(sizes.sum()))
    ref = O.fct(support, sizes, nodes, f, "qr")
    plan = F.Plan(support, sizes, nodes, tol=1e-14)
    s = torch.from_numpy(f).cuda()
    c = torch.empty(40, dtype=torch.float64, device="cuda")
    rep = plan.execute(s, c)
    assert rep["status"] == 0
    assert rel(c.cpu().numpy(), ref) <= TOL_FP64
    plan.close()


def test_invalid_arguments_are_rejected():
    sup = np.zeros((4, 2), dtype=np.uint16)
    with pytest.raises(F.FctError) as e:
        F.Plan(sup, np.array([[0, 3]], dtype=np.int32))
    assert e.value.status == 1
    with pytest.raises(F.FctError):
        F.Plan(sup, np.array([[1, 3]], dtype=np.int32), np.array([[2.0, 0.0]]))
    with pytest.raises(F.FctError):
        F.Plan(sup, np.array([[2, 3]], dtype=np.int32), block_threads=100)


def test_nonfinite_samples_reported():
    w = _small(SMALL[2])
    plan = F.Plan(w.support, w.sizes, w.nodes)
    s = torch.zeros(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, s)
    s[5] = float("nan")
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FctError) as e:
        plan.execute(s, c)
    assert e.value.status == F.fct.FCT_ERR_NONFINITE
    # the plan stays usable
    plan.sample(w.family, w.params, s)
    assert plan.execute(s, c)["status"] == 0
    plan.close()


@pytest.mark.slow
def test_d10_rational_full_size_fp64_and_mixed_match_oracle():
    """D=10, total degree 8 (N=43758), 30 grids, rational target, at full
    size: the FP64 path within 1e-11 and the mixed path within 1e-10 of the
    oracle's FP64 CGLS solution (tolerance 1e-15 on |A^T r| / |A^T b|)."""
    w = W.config_d10_rational()
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    system = O.AliasSystem(w.support, w.sizes, w.nodes)
    ref, it, relres = O.cgls(system.A, system.rhs(f), tol=1e-15)
    got64, s_gpu, rep64 = gpu_run(w, samples_np=f, precision=F.FCT_FP64, tol=1e-13)
    assert rep64["status"] == 0
    assert rel(got64, ref) <= TOL_FP64, (rel(got64, ref), rep64)
    gotmx, _, repmx = gpu_run(w, samples_np=f, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)
    assert repmx["status"] == 0
    assert rel(gotmx, ref) <= TOL_MIXED, (rel(gotmx, ref), repmx)


FOLDED_CASES = [
    ("D2_poly", 51, 2, 16, 4, 9, 33, W.FAMILY_POLY),
    ("D4_poly", 52, 4, 6, 12, 1, 7, W.FAMILY_POLY),
    ("D4_polygc", 53, 4, 6, 12, 1, 7, W.FAMILY_POLY_GAUSSCOS),
    ("D6_poly", 54, 6, 5, 18, 1, 6, W.FAMILY_POLY),
]


@pytest.mark.parametrize("case", FOLDED_CASES, ids=[c[0] for c in FOLDED_CASES])
def test_folded_polynomial_sampler_matches_term_by_term_and_oracle(case):
    """The fast sampler (coefficients folded into bins, grid interpolant
    evaluated at the nodes) equals term-by-term evaluation on the device and
    the oracle's brute-force samples."""
    w = _small(case)
    plan = F.Plan(w.support, w.sizes, w.nodes)
    s_term = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    s_fold = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, s_term)
    plan.sample(w.family | F.fct.FCT_SAMPLE_FOLDED, w.params, s_fold)
    torch.cuda.synchronize()
    a, b = s_term.cpu().numpy(), s_fold.cpu().numpy()
    scale = max(1.0, np.max(np.abs(a)))
    assert np.max(np.abs(a - b)) <= 1e-12 * scale
    ref = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    assert np.max(np.abs(b - ref)) <= 1e-12 * scale
    plan.close()


@pytest.mark.slow
def test_batch_of_512_mixed_transforms_equals_alone_and_oracle():
    """The 512-transform batch (D in 3..8, degree 6..14, polynomial plus
    Gaussian-cosine targets, mixed precision) in one persistent launch: every
    result is bit-identical to the same transform solved alone, all converge,
    and the smallest transforms match the oracle within 1e-10."""
    ws = W.config_batch()
    plans, samples, outs = [], [], []
    for w in ws:
        p = F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)
        s = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(w.family, w.params, s)
        plans.append(p)
        samples.append(s)
        outs.append(torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda"))
    reps = F.fct_execute_batch([p.handle for p in plans], samples, outs)
    assert all(r["status"] == 0 for r in reps), [r for r in reps if r["status"] != 0][:3]
    alone = torch.empty(max(p.N for p in plans), dtype=torch.float64, device="cuda")
    for p, s, o in zip(plans, samples, outs):
        a = alone[:p.N]
        assert p.execute(s, a)["status"] == 0
        assert torch.equal(a, o)
    small = sorted(range(len(ws)), key=lambda i: ws[i].N)[:4]
    for i in small:
        w = ws[i]
        f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
        ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
        assert rel(outs[i].cpu().numpy(), ref) <= TOL_MIXED, (w.name, rel(outs[i].cpu().numpy(), ref))
    for p in plans:
        p.close()


def test_bounded_wait_times_out_and_context_survives():
    """A barrier that nothing completes ends by its time limit with
    FCT_ERR_TIMEOUT; the device stays usable afterwards."""
    st, el = F.fct.fct_selftest_wait_timeout(0.2)
    assert st == F.fct.FCT_ERR_TIMEOUT
    assert 0.15 <= el <= 5.0
    w = W.config_small_poly()
    got, _, rep = gpu_run(w, tol=1e-13)
    assert rep["status"] == 0 and rel(got, w.coeffs_true) <= TOL_FP64


RHS_CASES = SMALL[:4] + [("D6_d10", None, None, None, None, None, None, None)]


@pytest.mark.parametrize("case", RHS_CASES, ids=[c[0] for c in RHS_CASES])
@pytest.mark.parametrize("kind", ["extrema", "first"])
def test_rhs_dct_stage_matches_oracle(case, kind):
    """The DCT stage alone (fct_plan_rhs): b = F f at the nonempty bins equals
    the oracle's per-grid DCT (direct matrix products) row by row, and the
    rows are exactly the oracle's nonempty bins."""
    w = W.config_d6_gausscos() if case[1] is None else _small(case)
    gk = F.FCT_GRID_EXTREMA if kind == "extrema" else F.FCT_GRID_FIRST_KIND
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes, kind=kind)
    s = O.AliasSystem(w.support, w.sizes, w.nodes, kind=kind)
    ref = s.rhs(f)
    plan = F.Plan(w.support, w.sizes, w.nodes, grid_kind=gk)
    b = torch.empty(plan.info["R"], dtype=torch.float64, device="cuda")
    bins = F.fct_plan_rhs(plan.handle, torch.from_numpy(f).cuda(), b)
    plan.close()
    order = np.argsort(bins, kind="stable")
    want_bins = np.concatenate([s.offsets[l] + s.rows[l] for l in range(len(s.rows))])
    assert np.array_equal(bins[order], want_bins)
    got = b.cpu().numpy()[order]
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(f)))


@pytest.mark.parametrize("case", RHS_CASES, ids=[c[0] for c in RHS_CASES])
@pytest.mark.parametrize("kind", ["extrema", "first"])
def test_alias_operator_matches_oracle(case, kind):
    """A x and A^T y from the plan's device tables (fct_plan_apply) equal the
    oracle's fold-built sparse matrix products, row by row."""
    w = W.config_d6_gausscos() if case[1] is None else _small(case)
    gk = F.FCT_GRID_EXTREMA if kind == "extrema" else F.FCT_GRID_FIRST_KIND
    s = O.AliasSystem(w.support, w.sizes, w.nodes, kind=kind)
    g = W.stream(31, "probe")
    x = g.standard_normal(w.N)
    y = g.standard_normal(s.R)
    plan = F.Plan(w.support, w.sizes, w.nodes, grid_kind=gk)
    ax = torch.empty(s.R, dtype=torch.float64, device="cuda")
    bins = F.fct_plan_apply(plan.handle, torch.from_numpy(x).cuda(), ax)
    order = np.argsort(bins, kind="stable")          # internal row order -> oracle order
    y_int = np.empty(s.R)
    y_int[order] = y                                  # y in the plan's internal row order
    aty = torch.empty(w.N, dtype=torch.float64, device="cuda")
    F.fct_plan_apply(plan.handle, torch.from_numpy(y_int).cuda(), aty, transpose=True)
    torch.cuda.synchronize()
    plan.close()
    ref_ax = s.A @ x
    ref_aty = s.A.T @ y
    assert np.max(np.abs(ax.cpu().numpy()[order] - ref_ax)) <= 1e-13 * max(1.0, np.abs(ref_ax).max())
    assert np.max(np.abs(aty.cpu().numpy() - ref_aty)) <= 1e-13 * max(1.0, np.abs(ref_aty).max())


@pytest.mark.parametrize("kind", ["extrema", "first"])
def test_rhs_by_fibre_matches_oracle(kind):
    """DCT passes with enough fibres run one thread per fibre with the even/odd
    split of the DCT matrix rows: axes of 2..16 points (odd and even n), 2^18
    or more fibres per pass; b must equal the oracle's direct DCT row by row."""
    D, d, K = 4, 6, 400
    sup = W.total_degree_support(D, d)
    g = W.stream(77, "sizes")
    sizes = g.integers(2, 17, size=(K, D)).astype(np.int32)
    nodes = np.cos(np.pi * W.stream(77, "nodes").random((K, D)))
    T = np.prod(sizes.astype(np.int64), axis=1)
    for p in range(D - 1):   # every pass but the last runs by fibre
        assert int(np.sum(T // sizes[:, p])) >= 1 << 18
    params = W.gausscos_params(78, D)
    f = O.sample_lgrid(W.FAMILY_GAUSSCOS, params, sup, sizes, nodes, kind=kind)
    s = O.AliasSystem(sup, sizes, nodes, kind=kind)
    ref = s.rhs(f)
    gk = F.FCT_GRID_EXTREMA if kind == "extrema" else F.FCT_GRID_FIRST_KIND
    plan = F.Plan(sup, sizes, nodes, grid_kind=gk, tensor_dct=-1)
    b = torch.empty(plan.info["R"], dtype=torch.float64, device="cuda")
    bins = F.fct_plan_rhs(plan.handle, torch.from_numpy(f).cuda(), b)
    plan.close()
    order = np.argsort(bins, kind="stable")
    want_bins = np.concatenate([s.offsets[l] + s.rows[l] for l in range(len(s.rows))])
    assert np.array_equal(bins[order], want_bins)
    got = b.cpu().numpy()[order]
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(f)))
