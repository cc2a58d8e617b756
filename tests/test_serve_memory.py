"""Admission by a device-memory budget (serve.py): the plan on the CPU, with a
fake per-handle size, and the warm-state rows' reclaiming; on the GPU, a
server under a budget allocates within it and still answers every request."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W
from paper_2606_05687_b300.serve import WarmRows, plan_memory


def per_handle(b):
    return 1000 + 100 * b


def test_plan_fits_everything_requested_when_the_budget_allows():
    p = plan_memory(10 ** 9, n_env=1000, n_handles=4, B_max=64, per_handle=per_handle, state_row_bytes=50,
                    warm=True)
    assert (p["handles"], p["B_max"], p["warm_rows"]) == (4, 64, 1000) and p["bytes"] <= 10 ** 9


def test_plan_trades_warm_rows_then_handles_then_batch_size():
    budget = 4 * per_handle(64) + 400 * 50 + 512
    p = plan_memory(budget, n_env=1000, n_handles=4, B_max=64, per_handle=per_handle, state_row_bytes=50, warm=True)
    assert p["handles"] == 4 and p["B_max"] == 64 and 4 * 64 <= p["warm_rows"] < 1000 and p["bytes"] <= budget
    # not enough rows for every slot in flight: fewer handles
    budget = 4 * per_handle(64) + 100 * 50
    p = plan_memory(budget, n_env=1000, n_handles=4, B_max=64, per_handle=per_handle, state_row_bytes=50, warm=True)
    assert p["handles"] < 4 and p["warm_rows"] >= p["handles"] * p["B_max"] and p["bytes"] <= budget
    # one handle of the full batch does not fit: smaller batches
    budget = per_handle(16) + 16 * 50 + 1024
    p = plan_memory(budget, n_env=1000, n_handles=4, B_max=64, per_handle=per_handle, state_row_bytes=50, warm=True)
    assert p["handles"] == 1 and p["B_max"] == 16 and p["bytes"] <= budget
    # without warm starts no rows are planned
    p = plan_memory(2 * per_handle(64), n_env=1000, n_handles=4, B_max=64, per_handle=per_handle,
                    state_row_bytes=50, warm=False)
    assert (p["handles"], p["warm_rows"]) == (2, 0)
    with pytest.raises(MemoryError):
        plan_memory(per_handle(1) - 1, n_env=10, n_handles=1, B_max=1, per_handle=per_handle,
                    state_row_bytes=50, warm=False)


def test_warm_rows_reclaim_least_recently_used_and_never_pinned():
    wr = WarmRows(n_env=10, rows=4)
    has = np.zeros(10, bool)
    r1 = wr.acquire(np.array([0, 1]), has)
    has[[0, 1]] = True
    r2 = wr.acquire(np.array([2, 3]), has)
    has[[2, 3]] = True
    assert len(set(r1) | set(r2)) == 4
    wr.release(r1)
    # rows of 0 and 1 are free to reclaim (least recently used); 2 and 3 are pinned
    r3 = wr.acquire(np.array([4, 5]), has)
    assert set(r3) == set(r1) and not has[0] and not has[1] and has[2] and has[3]
    with pytest.raises(RuntimeError):
        wr.acquire(np.array([6]), has)  # every row pinned
    wr.release(r2)
    wr.release(r3)
    # an environment keeps its row while it has one; repeats share it
    r4 = wr.acquire(np.array([2, 2, 7]), has)
    assert r4[0] == r4[1] == r2[0] and wr.row_of[7] == r4[2]
    assert wr.evicted == 3


@pytest.fixture(scope="module")
def pinmpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc as P
    return P


@pytest.mark.gpu
def test_server_under_a_budget_stays_within_it(pinmpc):
    import torch
    from paper_2606_05687_b300.serve import BatchServer, poisson_arrivals, serve_load
    batch = W.generate(W.rl_scale_walking(B=512, N=20, seed=26))
    pool = pinmpc.device_inputs(batch)
    from paper_2606_05687_b300.serve import STAGE_KEYS, handle_bytes
    cfg = pinmpc.default_config(13, 8, 3, 128, 20)
    env_bytes = {k: int(pool[k][0].numel() * pool[k].element_size()) for k in STAGE_KEYS}
    ph = handle_bytes(pinmpc.workspace_estimate(cfg), 128, 20, 13, 24, env_bytes)
    # two handles of 128 and 300 warm-state rows for 512 environments
    budget = 2 * ph + 300 * 4 * pinmpc.state_floats_estimate(cfg, 20)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    srv = BatchServer(pool, 13, 8, 3, B_max=128, N=20, n_handles=4, warm_shift=0, mem_budget=budget)
    plan = srv.plan
    assert plan["handles"] == 2 and plan["B_max"] == 128 and 256 <= plan["warm_rows"] < 512
    assert plan["bytes"] <= budget
    torch.cuda.synchronize()
    used = torch.cuda.memory_allocated() - before + sum(h["solver"].workspace_bytes for h in srv.handles)
    assert used <= budget, (used, budget, plan)
    assert sum(h["solver"].workspace_bytes for h in srv.handles) == len(srv.handles) * pinmpc.workspace_estimate(
        pinmpc.default_config(13, 8, 3, plan["B_max"], 20))
    rep = serve_load(srv, poisson_arrivals(40000.0, 0.1, 512, seed=2))
    assert rep["certified"] == rep["requests"] > 0
    assert srv.rows.evicted > 0 and srv.warm_loads > 0
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() - before + sum(h["solver"].workspace_bytes for h in srv.handles) <= budget
    srv.close()
