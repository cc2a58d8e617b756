"""Schedule autotuner: pick solve parameters for a workload by measurement.

The paper fixes none of the schedule (check points, refinement step, the
penalty rho); the defaults were measured on the walking workload.  For
another workload (another model, horizon or contact set) `autotune` times
trial solves of a representative batch on the device for each candidate
configuration and returns the fastest of those that certify the most
instances.
Host logic only: every trial runs the library's kernels through the C ABI.
"""
from __future__ import annotations

import itertools
from typing import Dict, Iterable, List, Optional

import numpy as np

from . import pinmpc

# the parameters the schedule exposes, and values worth trying for each
DEFAULT_GRID = {
    "check_start": (8, 12, 16, 24),
    "check_every": (10, 20, 40),
    "refine_alpha": (0.005, 0.01, 0.02),
    "rho": (30.0, 100.0, 300.0),
}
LIBRARY_DEFAULTS = {"check_start": 12, "check_every": 20, "refine_alpha": 0.01, "rho": 100.0}


def candidates(grid: Optional[Dict[str, Iterable]] = None, limit: Optional[int] = None) -> List[dict]:
    """The grid's configurations, the defaults' neighbourhood first: ordered by
    how many parameters differ from the library defaults, then by grid order."""
    grid = grid or DEFAULT_GRID
    names = list(grid)
    combos = [dict(zip(names, vals)) for vals in itertools.product(*(grid[n] for n in names))]
    combos.sort(key=lambda c: sum(1 for n in names if n in LIBRARY_DEFAULTS and c[n] != LIBRARY_DEFAULTS[n]))
    return combos[:limit] if limit else combos


def select_best(table: List[dict]) -> Optional[dict]:
    """The fastest entry (lowest ms) among those that certified the most
    instances; ties go to the earlier entry.  None for an empty table."""
    if not table:
        return None
    most = max(t["certified"] for t in table)
    return min((t for t in table if t["certified"] == most), key=lambda t: t["ms"])


def time_config(batch, trials: int = 3, **overrides) -> dict:
    """Median device time (ms) of `trials` solves of `batch` with `overrides`,
    after one warm-up solve, and how many instances were certified."""
    import torch

    s = pinmpc.solver_for(batch, **overrides)
    try:
        t = pinmpc.device_inputs(batch, "cuda")
        s.set_stages(batch.B, batch.N, **t)
        s.solve(batch.B)
        torch.cuda.synchronize()
        ms = []
        for _ in range(trials):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.solve(batch.B)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = torch.empty(batch.B, dtype=torch.int32, device="cuda")
        s.get_traj(None, None, st, None, None, None)
        torch.cuda.synchronize()
        certified = int((st.cpu().numpy() == pinmpc.CONVERGED).sum())
    finally:
        s.close()
    return {"config": overrides, "ms": float(np.median(ms)), "certified": certified, "instances": batch.B}


def autotune(batch, grid: Optional[Dict[str, Iterable]] = None, limit: Optional[int] = 24, trials: int = 3) -> dict:
    """Time the candidate configurations on `batch`; returns {"best": entry or
    None, "default": the first candidate's entry (the library defaults when the
    grid holds them), "table": all entries}."""
    cands = candidates(grid, limit)
    table = [time_config(batch, trials=trials, **c) for c in cands]
    return {"best": select_best(table), "default": table[0] if table else None, "table": table}
