"""The allocation-free execute (fct_execute_noalloc) against fct_execute.

fct_execute_noalloc serves callers that cannot allocate device memory when
they solve (memory policies that forbid cudaMalloc after start-up, fixed
pools, runtimes that own the device memory): it runs a plan built earlier with
its workspace in the library's fixed 32 MiB device array.  Its results must
match fct_execute's within the FP64 parity tolerance, on consecutive calls
(the array keeps the previous call's contents), and plans that need more
workspace than the array holds must be refused cleanly.  This file is named so
that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11  # relative l2, the FP64 parity tolerance of the GPU tests


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mk,prec", [(W.config_small_poly, F.FCT_FP64),
                                     (W.config_d6_gausscos, F.FCT_FP64),
                                     (W.config_d6_gausscos, F.FCT_MIXED)],
                         ids=["small_fp64", "d6_fp64", "d6_mixed"])
def test_noalloc_matches_execute_on_consecutive_calls(mk, prec):
    w = mk()
    opts = dict(precision=prec, tol=1e-13) if prec == F.FCT_FP64 else dict(precision=prec, tol=1e-12, inner_tol=1e-5)
    plan = F.Plan(w.support, w.sizes, w.nodes, **opts)
    samples = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, samples)
    ref = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep_ref = plan.execute(samples, ref)
    assert rep_ref["status"] == 0
    ref_np = ref.cpu().numpy()
    for call in range(2):
        out = torch.full((plan.N,), float("nan"), dtype=torch.float64, device="cuda")
        rep = F.fct_execute_noalloc(plan.handle, samples, out)
        assert rep["status"] == 0, rep
        assert rep["iterations"] == rep_ref["iterations"]
        assert _rel(out.cpu().numpy(), ref_np) <= TOL, call
    plan.close()


def test_noalloc_calls_take_no_device_memory():
    """After one warm call (which may load kernels), further calls leave the
    device's free memory unchanged: the workspace is the fixed array, and the
    samples, outputs and plan exist beforehand."""
    w = W.config_d6_gausscos()
    plan = F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-5)
    samples = torch.empty(plan.M, dtype=torch.float64, device="cuda")
    plan.sample(w.family, w.params, samples)
    out = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    F.fct_execute_noalloc(plan.handle, samples, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rep = F.fct_execute_noalloc(plan.handle, samples, out)
        assert rep["status"] == 0
        F.fct_execute_noalloc(plan.handle, samples, out, report=False)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    plan.close()


def test_noalloc_refuses_plans_beyond_its_array():
    """A 200 x 200 x 130 grid (5.2 million samples) needs more than 32 MiB of workspace."""
    support = np.zeros((8, 3), dtype=np.uint16)
    support[:, 2] = np.arange(8)
    sizes = np.array([[200, 200, 130]], dtype=np.int32)
    plan = F.Plan(support, sizes)
    samples = torch.zeros(plan.M, dtype=torch.float64, device="cuda")
    out = torch.zeros(plan.N, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FctError) as e:
        F.fct_execute_noalloc(plan.handle, samples, out)
    assert e.value.status == F.fct.FCT_ERR_INVALID_ARG
    assert "32" in str(e.value) or "bytes" in str(e.value)
    plan.close()
