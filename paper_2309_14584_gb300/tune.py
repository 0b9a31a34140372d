"""Autotuner: time a few launch configurations of one plan (or one batch) on
the caller's device-resident inputs and keep the fastest.

Every candidate solves the same system to the same tolerance; the results
differ only by the order of floating-point additions (or not at all: team
sizes never change a transform's result).  Timing uses CUDA events on the
current stream; all arithmetic runs in libfct_gb300.so.

Dimensions:
  * single transforms (autotune): block size, threads per coefficient in the
    A^T q gather, entries per lane of the A p gather; then the A^T q gather
    layout, the inner solve on the stored normal matrix (one team barrier per
    iteration) and whether the grids with long axes take their DCT passes on
    the tensor cores;
  * batches and serving (autotune_team_blocks): blocks per team.
"""
from __future__ import annotations

from . import fct as F

CANDIDATES = (
    dict(block_threads=256),
    dict(block_threads=512),
    dict(block_threads=512, coef_lanes=8),
    dict(block_threads=256, coef_lanes=8),
    dict(block_threads=128),
    dict(block_threads=256, entries_per_lane=8),
    dict(block_threads=512, entries_per_lane=8),
)
TEAM_BLOCKS = (8, 16, 19, 38, 76)


def _time(fn, reps: int) -> float:
    import torch
    fn()
    for _ in range(2):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(support, sizes, nodes, samples, options: dict, candidates=CANDIDATES, reps: int = 10) -> dict:
    """Returns {"options": fastest options (options updated with a candidate
    and the toggles that won), "ms": its mean time, "timings": [(options
    tried beyond `options`, ms) for each trial that converged]}.  samples:
    device double[M] of this L-grid.

    First the launch shapes of `candidates`; then, on the fastest shape, each
    algorithmic choice the caller left open, flipped one at a time and kept
    when faster: the A^T q gather layout (coef_split), for mixed-path plans
    that store W = A^T A the inner solve without it (normal_matrix = -1), and
    for plans with tensor-core grids their DCT on the FP64 units
    (tensor_dct = -1)."""
    import torch

    timings = []

    def measure(extra):
        try:
            plan = F.Plan(support, sizes, nodes, **dict(options, **extra))
        except F.FctError:
            return None, None
        try:
            c = torch.empty(plan.N, dtype=torch.float64, device=samples.device)
            if plan.execute(samples, c)["status"] != 0:
                return None, None
            ms = _time(lambda: plan.execute(samples, c, report=False), reps)
            info = dict(plan.info)
        except F.FctError:
            return None, None
        finally:
            plan.close()
        timings.append((dict(extra), ms))
        return ms, info

    best, best_ms, best_info = None, None, None
    for cand in candidates:
        ms, info = measure(dict(cand))
        if ms is not None and (best_ms is None or ms < best_ms):
            best, best_ms, best_info = dict(cand), ms, info
    if best is None:
        raise RuntimeError("no launch shape converged")
    toggles = []
    if "coef_split" not in options:
        toggles.append(dict(coef_split=-1 if best_info.get("coef_split") else 1))
    if options.get("precision") == F.FCT_MIXED and "normal_matrix" not in options and best_info.get("normal_nnz"):
        # the automatic rule stores W only where it has no more entries than A and
        # A^T together, the only case it can win (forcing it on elsewhere was
        # measured up to 30x slower), so the tuner only tries it off
        toggles.append(dict(normal_matrix=-1))
    if "tensor_dct" not in options and best_info.get("tensor_dct_grids", 0) > 0:
        toggles.append(dict(tensor_dct=-1))
    for t in toggles:
        ms, _ = measure(dict(best, **t))
        if ms is not None and ms < best_ms:
            best, best_ms = dict(best, **t), ms
    return {"options": dict(options, **best), "ms": best_ms, "timings": timings}


def autotune_team_blocks(handles, samples, coeffs, candidates=TEAM_BLOCKS, reps: int = 3) -> dict:
    """Blocks per team for one batch (fct_execute_batch of the given plan
    handles and device buffers): {"team_blocks": fastest, "ms": its time per
    launch, "timings": [(team_blocks, ms)]}.  Candidates larger than the
    batch can use are skipped by the library's own clamp, so the times of
    those candidates repeat."""
    timings = []
    for tb in candidates:
        reps_ = F.fct_execute_batch(handles, samples, coeffs, team_blocks=tb)
        if not all(r["status"] == 0 for r in reps_):
            continue
        ms = _time(lambda: F.fct_execute_batch(handles, samples, coeffs, team_blocks=tb, report=False), reps)
        timings.append((tb, ms))
    if not timings:
        raise RuntimeError("no team size converged")
    tb, ms = min(timings, key=lambda t: t[1])
    return {"team_blocks": tb, "ms": ms, "timings": timings}
