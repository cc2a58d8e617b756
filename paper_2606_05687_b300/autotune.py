"""Schedule autotuner: pick solve parameters for a workload by measurement.

The paper fixes none of the schedule (check points, refinement steps and
step, the penalty rho) and none of the launch shapes; the library's
defaults were measured per shape on the walking and small centroidal
workloads.  Besides the schedule, a grid may hold "horizon_classes": the
round kernel's CTA shapes for batches with ragged horizons.  For
another workload (another model, horizon or contact set) `autotune` times
trial solves of a representative batch on the device for each candidate
configuration and returns the fastest of those that certify the most
instances.
Host logic only: every trial runs the library's kernels through the C ABI.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, Iterable, List, Optional

import numpy as np

from . import pinmpc

# the parameters the schedule exposes, and values worth trying for each
DEFAULT_GRID = {
    "check_start": (8, 12, 16, 24, 32),
    "check_every": (10, 20, 40),
    "refine_alpha": (0.001, 0.005, 0.01, 0.02),
    "rho": (30.0, 100.0, 300.0),
    "refine_steps": (2, 3, 4),
}
# the library defaults of the walking shape (nx 13, eight 3-D contacts);
# `library_defaults` reads those of any shape from the C library
LIBRARY_DEFAULTS = {"check_start": 12, "check_every": 20, "refine_alpha": 0.01, "rho": 100.0, "refine_steps": 3}


def library_defaults(nx: int, n_contacts: int, contact_dim: int, names: Iterable[str] = tuple(DEFAULT_GRID)) -> dict:
    """The C library's defaults of the given shape for the named parameters
    (floats rounded to the nearest grid-style decimal of their FP32 value)."""
    cfg = pinmpc.default_config(nx, n_contacts, contact_dim, 1, 1)
    out = {}
    for n in names:
        if not hasattr(cfg, n):  # a launch-shape key, not a configuration field
            continue
        v = getattr(cfg, n)
        out[n] = float(f"{v:.6g}") if isinstance(v, float) else v
    return out


def _differs(a, b) -> bool:
    return not math.isclose(float(a), float(b), rel_tol=1e-6)


def candidates(grid: Optional[Dict[str, Iterable]] = None, limit: Optional[int] = None,
               defaults: Optional[dict] = None) -> List[dict]:
    """The grid's configurations, the defaults' neighbourhood first: ordered by
    how many parameters differ from `defaults` (the walking shape's library
    defaults when None), then by grid order."""
    grid = grid or DEFAULT_GRID
    defaults = LIBRARY_DEFAULTS if defaults is None else defaults
    names = list(grid)
    combos = [dict(zip(names, vals)) for vals in itertools.product(*(grid[n] for n in names))]
    combos.sort(key=lambda c: sum(1 for n in names if n in defaults and _differs(c[n], defaults[n])))
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
    after one warm-up solve, and how many instances were certified.  The
    key "horizon_classes" (a tuple of stage counts) sets the handle's
    round-kernel CTA shapes (mpc_set_horizon_classes); the others are
    solver configuration fields."""
    import torch

    cfg = {k: v for k, v in overrides.items() if k != "horizon_classes"}
    s = pinmpc.solver_for(batch, **cfg)
    try:
        if "horizon_classes" in overrides:
            s.set_horizon_classes(list(overrides["horizon_classes"]))
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
    """Time the candidate configurations on `batch`, nearest to the library
    defaults of the batch's shape first; returns {"best": entry or None,
    "default": the first candidate's entry (the library defaults when the grid
    holds them), "table": all entries}."""
    grid = grid or DEFAULT_GRID
    cands = candidates(grid, limit, library_defaults(batch.nx, batch.nc, batch.contact_dim, grid))
    table = [time_config(batch, trials=trials, **c) for c in cands]
    return {"best": select_best(table), "default": table[0] if table else None, "table": table}
