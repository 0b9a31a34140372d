"""Prepared batches (fct_batch_*): the job table stays on the device, so one
launch needs nothing from the host, is recorded by stream capture into a
CUDA graph, and every replay solves the batch again from the samples as they
are at that moment.  Results equal fct_execute_batch and each transform alone
bit for bit."""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O

pytestmark = pytest.mark.gpu


def _batch(n=6):
    ws = [W.make_workload(f"g{i}", 80 + i, 2 + i % 3, 8, 3 * (2 + i % 3), 1, 9, W.FAMILY_GAUSSCOS) for i in range(n)]
    plans = [F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-4) for w in ws]
    xs, cs = [], []
    for i, (p, w) in enumerate(zip(plans, ws)):
        x = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(W.FAMILY_GAUSSCOS, W.gausscos_params(300 + i, w.D), x)
        xs.append(x)
        cs.append(torch.full((p.N,), float("nan"), dtype=torch.float64, device="cuda"))
    return ws, plans, xs, cs


def test_prepared_batch_equals_execute_batch_and_alone():
    ws, plans, xs, cs = _batch()
    hs = [p.handle for p in plans]
    b = F.fct_batch_create(hs, xs, cs, team_blocks=8)
    F.fct_batch_launch(b)
    reps = F.fct_batch_reports(b, len(plans))
    assert all(r["status"] == 0 for r in reps)
    ref = [torch.empty_like(c) for c in cs]
    F.fct_execute_batch(hs, xs, ref, team_blocks=16)
    for p, x, c, r in zip(plans, xs, cs, ref):
        assert torch.equal(c, r)
        alone = torch.empty_like(c)
        assert p.execute(x, alone)["status"] == 0
        assert torch.equal(alone, c)
    F.fct_batch_destroy(b)
    for p in plans:
        p.close()


def test_graph_captured_batch_replays_on_new_samples():
    ws, plans, xs, cs = _batch()
    hs = [p.handle for p in plans]
    b = F.fct_batch_create(hs, xs, cs, team_blocks=8)
    F.fct_batch_launch(b)          # one launch outside the graph first
    torch.cuda.synchronize()
    first = [c.clone() for c in cs]
    for c in cs:
        c.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.fct_batch_launch(b)
    g.replay()
    torch.cuda.synchronize()
    assert all(r["status"] == 0 for r in F.fct_batch_reports(b, len(plans)))
    for c, f in zip(cs, first):
        assert torch.equal(c, f)
    # new targets written into the same sample buffers: the replay solves them
    for i, (p, w) in enumerate(zip(plans, ws)):
        p.sample(W.FAMILY_GAUSSCOS, W.gausscos_params(900 + i, w.D), xs[i])
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert all(r["status"] == 0 for r in F.fct_batch_reports(b, len(plans)))
    for p, w, x, c in zip(plans, ws, xs, cs):
        alone = torch.empty_like(c)
        assert p.execute(x, alone)["status"] == 0
        assert torch.equal(alone, c)
    # the smallest transform against the oracle's least-squares solution
    i = min(range(len(plans)), key=lambda k: plans[k].N)
    f = O.sample_lgrid(W.FAMILY_GAUSSCOS, W.gausscos_params(900 + i, ws[i].D), ws[i].support, ws[i].sizes,
                       ws[i].nodes)
    ref = O.fct(ws[i].support, ws[i].sizes, ws[i].nodes, f, "qr")
    got = cs[i].cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
    del g
    F.fct_batch_destroy(b)
    for p in plans:
        p.close()


def test_batch_create_rejects_bad_arguments():
    ws, plans, xs, cs = _batch(2)
    hs = [p.handle for p in plans]
    with pytest.raises(F.FctError):
        F.fct_batch_create([hs[0], hs[0]], xs, cs)      # a plan twice
    with pytest.raises(F.FctError):
        F.fct_batch_create(hs, [xs[0], 0], cs)           # a NULL buffer
    for p in plans:
        p.close()


def test_graph_batch_of_grid_split_and_fp64_plans():
    """A prepared batch mixing a grid-split plan (90 grids, wide rows) with FP64
    and mixed plans of other shapes, replayed from a CUDA graph: each result
    equals the transform alone bit for bit."""
    sup = W.sparse_infinity_support(12, 30, 9, 2000, 3)
    N, D = sup.shape
    sizes, nodes = W.l_grid(130, N, D, 3 * D, 1, 10)
    big = F.Plan(sup, sizes, nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-4, entries_per_lane=2)
    assert big.info["coef_split"] == 1 and big.info["wide_rows"] > 0
    ws, plans, xs, cs = _batch(3)
    plans = list(plans)
    fp = F.Plan(ws[0].support, ws[0].sizes, ws[0].nodes, precision=F.FCT_FP64, tol=1e-13)
    xb = torch.empty(big.M, dtype=torch.float64, device="cuda")
    big.sample(W.FAMILY_GAUSSCOS, W.gausscos_params(5, D), xb)
    plans += [big, fp]
    xs += [xb, xs[0]]
    cs += [torch.full((big.N,), float("nan"), dtype=torch.float64, device="cuda"),
           torch.full((fp.N,), float("nan"), dtype=torch.float64, device="cuda")]
    b = F.fct_batch_create([p.handle for p in plans], xs, cs, team_blocks=16)
    F.fct_batch_launch(b)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.fct_batch_launch(b)
    for c in cs:
        c.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert all(r["status"] == 0 for r in F.fct_batch_reports(b, len(plans)))
    for p, x, c in zip(plans, xs, cs):
        alone = torch.empty_like(c)
        assert p.execute(x, alone)["status"] == 0
        assert torch.equal(alone, c)
    del g
    F.fct_batch_destroy(b)
    for p in plans:
        p.close()
