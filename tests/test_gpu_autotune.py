"""Schedule autotuner on the device: the chosen configuration certifies every
instance and is no slower than the defaults on the batch it was tuned on."""
import pytest

from paper_2606_05687_b300 import workload as W

pytestmark = pytest.mark.gpu


def test_autotune_small_grid():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import autotune as A
    batch = W.generate(W.rl_scale_walking(B=256, N=20, seed=62))
    grid = {"check_start": (12, 8), "check_every": (20, 10), "refine_alpha": (0.01,), "rho": (100.0,)}
    res = A.autotune(batch, grid=grid, limit=None, trials=3)
    assert len(res["table"]) == 4
    assert res["default"]["config"] == {"check_start": 12, "check_every": 20, "refine_alpha": 0.01, "rho": 100.0}
    best = res["best"]
    assert best is not None and best["certified"] == batch.B
    assert best["ms"] <= res["default"]["ms"]


def test_autotune_horizon_classes():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import autotune as A
    batch = W.generate(W.rl_scale_walking(B=512, N=30, seed=63, horizon_min=5))
    grid = {"rho": (100.0,), "horizon_classes": ((), (10, 20))}
    res = A.autotune(batch, grid=grid, limit=None, trials=3)
    assert [t["config"]["horizon_classes"] for t in res["table"]] == [(), (10, 20)]
    # the classes change the launch shapes, never which instances certify
    assert res["table"][0]["certified"] == res["table"][1]["certified"] == batch.B
    print("ms without / with classes", res["table"][0]["ms"], res["table"][1]["ms"])
