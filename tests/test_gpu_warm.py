"""Receding-horizon warm start (mpc_warm_start) against the oracle: a warm
start changes the starting iterate, never the certified solution."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

from parity_util import compare, oracle_refs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pinmpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc as P
    return P


def test_warm_restart_same_batch(pinmpc):
    """Shift 0: re-solving from the final iterate certifies at the first check."""
    batch = W.generate(W.rl_scale_walking(B=96, N=20, seed=1002))
    s = pinmpc.solver_for(batch)
    cold = pinmpc.solve_workload(batch, solver=s)
    s.warm_start(0)
    warm = pinmpc.solve_workload(batch, solver=s)
    assert np.all(cold["status"] == 0) and np.all(warm["status"] == 0)
    assert warm["iters"].max() <= s.cfg.check_start
    ids = list(range(0, 96, 12))
    refs = oracle_refs(batch, ids)
    compare(batch, cold, ids, refs)
    compare(batch, warm, ids, refs)
    # one solve consumes the warm start: the next one is cold again
    again = pinmpc.solve_workload(batch, solver=s)
    assert np.array_equal(again["iters"], cold["iters"]) and np.array_equal(again["u"], cold["u"])


def test_receding_horizon_shift(pinmpc):
    """Shift 1 with the next MPC step's stage data: oracle parity, and on average
    no more ADMM iterations or polishes than a cold solve of the same batch."""
    batch = W.generate(W.rl_scale_walking(B=128, N=20, seed=1002))
    s = pinmpc.solver_for(batch)
    first = pinmpc.solve_workload(batch, solver=s)
    nxt = batch.receding(first["xi"][:, 0], first["u"][:, 0])
    s.warm_start(1)
    warm = pinmpc.solve_workload(nxt, solver=s)
    cold = pinmpc.solve_workload(nxt)
    assert np.all(warm["status"] == 0)
    ids = list(range(0, 128, 16)) + [1, 127]
    refs = oracle_refs(nxt, ids)
    compare(nxt, warm, ids, refs)
    compare(nxt, cold, ids, refs)
    print("iters warm/cold", warm["iters"].mean(), cold["iters"].mean(),
          "polishes warm/cold", warm["polishes"].mean(), cold["polishes"].mean())
    assert warm["iters"].mean() <= cold["iters"].mean()
    assert warm["polishes"].mean() <= cold["polishes"].mean() + 0.05


def test_warm_start_argument_checks(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=8, N=20, seed=1002))
    s = pinmpc.solver_for(batch)
    with pytest.raises(pinmpc.MpcError) as ei:
        s.warm_start(1)  # no solve yet
    assert ei.value.code == pinmpc.MPC_ERR_STATE
    pinmpc.solve_workload(batch, solver=s)
    with pytest.raises(pinmpc.MpcError) as ei:
        s.warm_start(20)
    assert ei.value.code == pinmpc.MPC_ERR_INVALID_ARG


def test_state_calls_reject_host_buffers(pinmpc):
    """mpc_save_state / mpc_load_state check that the store and the row indices
    are device memory of the handle's device before launching anything: a
    host index array (natural from C or numpy) is an argument error, not a
    kernel reading a host address."""
    import torch
    batch = W.generate(W.rl_scale_walking(B=8, N=10, seed=3))
    s = pinmpc.solver_for(batch)
    pinmpc.solve_workload(batch, solver=s)
    F = s.state_floats(10)
    store = torch.zeros((8, F), device="cuda")
    host_idx = np.arange(8, dtype=np.int32)
    host_store = np.zeros((8, F), np.float32)
    for call in (lambda: s.save_state(store, host_idx, 8, shift=0),
                 lambda: s.save_state(host_store, None, 8, shift=0),
                 lambda: s.load_state(store, host_idx, 8),
                 lambda: s.load_state(host_store, None, 8)):
        with pytest.raises(pinmpc.MpcError) as ei:
            call()
        assert ei.value.code == pinmpc.MPC_ERR_INVALID_ARG
    # device buffers still work afterwards
    s.save_state(store, torch.arange(8, dtype=torch.int32, device="cuda"), 8, shift=0)
    s.load_state(store, None, 8)
    torch.cuda.synchronize()
    s.close()
