"""Launch-shape autotuner: time fct_execute for a few launch shapes of one
plan on the caller's device-resident samples and keep the fastest.

The shapes change only how the work is split over threads (block size,
threads per coefficient in the A^T q gather, entries per lane in the A p
gather); every shape solves the same system to the same tolerance, and the
results differ only by the order of floating-point additions.  Timing uses
CUDA events on the current stream; all arithmetic runs in libfct_gb300.so.
"""
from __future__ import annotations

from . import fct as F

CANDIDATES = (
    dict(block_threads=256),
    dict(block_threads=512),
    dict(block_threads=512, coef_lanes=8),
    dict(block_threads=256, coef_lanes=8),
    dict(block_threads=128),
)


def autotune(support, sizes, nodes, samples, options: dict, candidates=CANDIDATES, reps: int = 10) -> dict:
    """Returns {"options": fastest options (options updated with a candidate),
    "ms": its mean time, "timings": [(candidate, ms) for each candidate that
    converged]}.  samples: device double[M] of this L-grid."""
    import torch

    timings = []
    for cand in candidates:
        opts = dict(options, **cand)
        plan = F.Plan(support, sizes, nodes, **opts)
        try:
            c = torch.empty(plan.N, dtype=torch.float64, device=samples.device)
            if plan.execute(samples, c)["status"] != 0:
                continue
            for _ in range(2):
                plan.execute(samples, c, report=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                plan.execute(samples, c, report=False)
            e1.record()
            torch.cuda.synchronize()
            timings.append((cand, e0.elapsed_time(e1) / reps))
        finally:
            plan.close()
    if not timings:
        raise RuntimeError("no launch shape converged")
    cand, ms = min(timings, key=lambda t: t[1])
    return {"options": dict(options, **cand), "ms": ms, "timings": timings}
