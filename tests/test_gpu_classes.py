"""Horizon classes (mpc_set_horizon_classes): each ADMM round runs once per
class on CTAs sized for the class's longest horizon.  The arithmetic per
instance is unchanged, so one-CTA classes give results identical to one
class bit for bit; CTA-pair batches match the oracle; bad horizons, warm
starts and graph replay keep working."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

from parity_util import REL_TRAJ, compare

pytestmark = pytest.mark.gpu

KEYS = ("xi", "u", "status", "iters", "kkt", "active_bits", "polishes")


@pytest.fixture(scope="module")
def pinmpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc as P
    return P


def _solve(P, batch, caps, graph=False, solver=None):
    s = solver or P.solver_for(batch)
    s.set_horizon_classes(caps)
    if graph:
        s.set_graph_mode(True)
        P.solve_workload(batch, solver=s)  # capture
    out = P.solve_workload(batch, solver=s)
    if solver is None:
        s.close()
    return out


@pytest.mark.parametrize("maker,N,caps", [(W.rl_scale_walking, 30, [10, 20]),
                                          (W.small_centroidal, 32, [10, 20]),
                                          (W.rl_scale_walking, 20, [10])])
def test_classes_equal_one_class_bit_for_bit(pinmpc, maker, N, caps):
    batch = W.generate(maker(B=384, N=N, seed=91, horizon_min=1))
    one = _solve(pinmpc, batch, [])
    cls = _solve(pinmpc, batch, caps)
    for k in KEYS:
        assert np.array_equal(one[k], cls[k]), k
    assert np.all(cls["status"] == 0)
    h = batch.horizon
    compare(batch, cls, [int(np.argmin(h)), int(np.argmax(h)), int(np.flatnonzero(h == caps[0])[0])])


def test_pair_form_with_classes(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=256, N=40, seed=92, horizon_min=5))
    one = _solve(pinmpc, batch, [])
    cls = _solve(pinmpc, batch, pinmpc.horizon_classes_for(40))
    assert np.all(cls["status"] == 0)
    h = batch.horizon
    long_ = h > 32
    # instances above 32 stages stay on CTA pairs in both runs: identical
    for k in ("xi", "u", "iters"):
        assert np.array_equal(one[k][long_], cls[k][long_]), k
    # shorter ones moved from CTA pairs to single CTAs: same optimum
    for b in np.flatnonzero(~long_)[:40]:
        n = int(h[b])
        su = np.abs(one["u"][b, :n]).max()
        assert np.abs(cls["u"][b, :n] - one["u"][b, :n]).max() <= 2 * REL_TRAJ * su
    compare(batch, cls, [int(np.argmin(h)), int(np.flatnonzero((h > 10) & (h <= 20))[0]),
                         int(np.flatnonzero((h > 20) & (h <= 32))[0]), int(np.flatnonzero(long_)[0])])


def test_bad_horizon_reported_in_a_classed_batch(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=64, N=30, seed=93, horizon_min=5))
    batch.horizon[3] = 0
    batch.horizon[7] = 31
    out = _solve(pinmpc, batch, [10, 20])
    assert out["status"][3] == 5 and out["status"][7] == 5  # bad horizon
    ok = np.ones(64, bool)
    ok[[3, 7]] = False
    assert np.all(out["status"][ok] == 0)


def test_warm_start_and_graph_replay_with_classes(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=256, N=30, seed=94, horizon_min=3))
    ref = _solve(pinmpc, batch, [])
    g = _solve(pinmpc, batch, [10, 20], graph=True)
    for k in KEYS:
        assert np.array_equal(ref[k], g[k]), k
    s = pinmpc.solver_for(batch)
    s.set_horizon_classes([10, 20])
    pinmpc.solve_workload(batch, solver=s)
    s.warm_start(0)
    warm = pinmpc.solve_workload(batch, solver=s)
    s2 = pinmpc.solver_for(batch)
    pinmpc.solve_workload(batch, solver=s2)
    s2.warm_start(0)
    warm1 = pinmpc.solve_workload(batch, solver=s2)
    s.close()
    s2.close()
    for k in KEYS:
        assert np.array_equal(warm[k], warm1[k]), k
    assert np.all(warm["status"] == 0) and warm["iters"].mean() < ref["iters"].mean()


def test_class_argument_errors(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=4, N=20, seed=95))
    s = pinmpc.solver_for(batch)
    for caps in ([20, 10], [0], [10, 10], [21], [4, 8, 12, 16]):
        with pytest.raises(pinmpc.MpcError) as ei:
            s.set_horizon_classes(caps)
        assert ei.value.code == pinmpc.MPC_ERR_INVALID_ARG
    s.set_horizon_classes([20])  # at the stride: one class
    out = pinmpc.solve_workload(batch, solver=s)
    s.close()
    assert np.all(out["status"] == 0)
