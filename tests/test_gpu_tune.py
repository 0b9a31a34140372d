"""The launch-shape autotuner picks one of its candidates, and the plan built
with the chosen shape still meets the oracle."""
import numpy as np
import pytest
import torch

import paper_2309_14584_gb300 as F
import workloads as W
from oracle import fct_oracle as O
from paper_2309_14584_gb300.tune import CANDIDATES, autotune

pytestmark = pytest.mark.gpu


def test_autotune_choice_solves_to_tolerance():
    w = W.make_workload("tune", 43, 4, 5, 12, 1, 6, W.FAMILY_GAUSSCOS)
    f = O.sample_lgrid(w.family, w.params, w.support, w.sizes, w.nodes)
    ref = O.fct(w.support, w.sizes, w.nodes, f, "qr")
    x = torch.from_numpy(f).cuda()
    opts = dict(precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-4)
    r = autotune(w.support, w.sizes, w.nodes, x, opts, reps=3)
    assert len(r["timings"]) >= len(CANDIDATES) and r["ms"] > 0
    chosen = {k: v for k, v in r["options"].items() if k not in opts}
    shape = {k: v for k, v in chosen.items() if k not in ("coef_split", "normal_matrix", "tensor_dct")}
    assert shape in [dict(c) for c in CANDIDATES]
    tried = [t for t, _ in r["timings"]]
    assert any("coef_split" in t for t in tried)
    assert r["ms"] == min(ms for _, ms in r["timings"])
    plan = F.Plan(w.support, w.sizes, w.nodes, **r["options"])
    c = torch.empty(plan.N, dtype=torch.float64, device="cuda")
    rep = plan.execute(x, c)
    plan.close()
    assert rep["status"] == 0
    assert np.linalg.norm(c.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("blocks,bt", [(1, 256), (8, 256), (152, 512), (304, 256)])
def test_team_barrier_floor_is_measured(blocks, bt):
    us = F.fct_measure_team_barrier(blocks, bt, 500)
    assert 0.0 < us < 100.0


def test_team_barrier_probe_rejects_bad_arguments():
    with pytest.raises(F.FctError):
        F.fct_measure_team_barrier(0, 256, 10)
    with pytest.raises(F.FctError):
        F.fct_measure_team_barrier(100000, 256, 10)
    with pytest.raises(F.FctError):
        F.fct_measure_team_barrier(4, 96, 10)


def test_team_size_autotune_keeps_batch_results_bit_identical():
    """The team-size tuner picks one of its candidates; every team size gives
    the same coefficients bit for bit (reductions follow a fixed order that
    does not depend on the team), equal to each transform alone."""
    from paper_2309_14584_gb300.tune import TEAM_BLOCKS, autotune_team_blocks
    ws = [W.make_workload(f"b{i}", 60 + i, 3, 8, 9, 1, 9, W.FAMILY_GAUSSCOS) for i in range(6)]
    plans = [F.Plan(w.support, w.sizes, w.nodes, precision=F.FCT_MIXED, tol=1e-12, inner_tol=1e-4) for w in ws]
    xs, cs = [], []
    for p, w in zip(plans, ws):
        x = torch.empty(p.M, dtype=torch.float64, device="cuda")
        p.sample(w.family, w.params, x)
        xs.append(x)
        cs.append(torch.empty(p.N, dtype=torch.float64, device="cuda"))
    hs = [p.handle for p in plans]
    r = autotune_team_blocks(hs, xs, cs, reps=1)
    assert r["team_blocks"] in TEAM_BLOCKS and len(r["timings"]) == len(TEAM_BLOCKS)
    F.fct_execute_batch(hs, xs, cs, team_blocks=r["team_blocks"])
    tuned = [c.clone() for c in cs]
    F.fct_execute_batch(hs, xs, cs, team_blocks=8)
    for a, b in zip(tuned, cs):
        assert torch.equal(a, b)
    for p, x, a in zip(plans, xs, tuned):
        alone = torch.empty_like(a)
        assert p.execute(x, alone)["status"] == 0
        assert torch.equal(alone, a)
    for p in plans:
        p.close()
