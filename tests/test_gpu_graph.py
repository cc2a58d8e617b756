"""CUDA-graph replay of the solve (mpc_set_graph_mode): bit-identical to the
direct launches for fresh and repeated solves, new batch sizes and warm
starts; per-kernel timing falls back to direct launches."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

pytestmark = pytest.mark.gpu

KEYS = ("xi", "u", "status", "iters", "kkt", "active_bits", "polishes", "pivots")


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc
    return pinmpc


def same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in KEYS)


def test_graph_replay_equals_direct(P):
    for spec in (W.rl_scale_walking(B=256, N=20, seed=51), W.small_centroidal(B=64, N=10, seed=52)):
        batch = W.generate(spec)
        direct = P.solve_workload(batch)
        s = P.solver_for(batch)
        s.set_graph_mode(True)
        first = P.solve_workload(batch, solver=s)   # captures
        second = P.solve_workload(batch, solver=s)  # replays
        assert s.graph_stats() == (1, 2)
        assert same(direct, first) and same(direct, second)
        # a smaller batch is a new graph; the old one stays cached
        sub = batch.subset(range(batch.B // 2))
        half = P.solve_workload(sub, solver=s)
        assert same(P.solve_workload(sub), half) and s.graph_stats() == (2, 3)
        s.close()


def test_graph_replay_with_warm_start_and_timing(P):
    batch = W.generate(W.rl_scale_walking(B=128, N=20, seed=53))
    ref = P.solver_for(batch)
    s = P.solver_for(batch)
    s.set_graph_mode(True)
    a, b = P.solve_workload(batch, solver=ref), P.solve_workload(batch, solver=s)
    assert same(a, b)
    nxt = batch.receding(a["xi"][:, 0], a["u"][:, 0])
    ref.warm_start(1)
    s.warm_start(1)
    assert same(P.solve_workload(nxt, solver=ref), P.solve_workload(nxt, solver=s))
    assert s.graph_stats() == (2, 2)  # the warm solve is its own graph
    s.set_kernel_timing(True)
    assert same(P.solve_workload(batch, solver=ref), P.solve_workload(batch, solver=s))
    assert s.graph_stats() == (2, 2)  # timed solves launch directly
    s.set_kernel_timing(False)
    s.set_graph_mode(False)
    assert same(P.solve_workload(batch, solver=ref), P.solve_workload(batch, solver=s))
    ref.close()
    s.close()


def test_round_events_expose_finished_instances(P):
    # after round r's event, an instance reads its final status exactly when its
    # certified iteration count is at most the round's end, else MPC_RUNNING
    import torch
    batch = W.generate(W.rl_scale_walking(B=512, N=20, seed=55))
    s = P.solver_for(batch)
    ends = P.round_schedule(s.cfg)
    side = torch.cuda.Stream()
    events = [torch.cuda.Event() for _ in ends]
    for ev in events:
        ev.record(side)
    s.set_round_events(events)
    main = torch.cuda.current_stream()
    s.set_stages(batch.B, batch.N, **P.device_inputs(batch), stream=main)
    s.solve(batch.B, stream=main)
    per_round = [torch.empty(batch.B, dtype=torch.int32, device="cuda") for _ in ends]
    for ev, st in zip(events, per_round):
        side.wait_event(ev)
        s.get_traj(status=st, stream=side)
    final = torch.empty(batch.B, dtype=torch.int32, device="cuda")
    iters = torch.empty(batch.B, dtype=torch.int32, device="cuda")
    s.get_traj(status=final, iters=iters, stream=main)
    torch.cuda.synchronize()
    final, iters = final.cpu().numpy(), iters.cpu().numpy()
    assert np.all(final == P.CONVERGED) and iters.max() > ends[0]  # some instances need a later round
    for end, st in zip(ends, per_round):
        st = st.cpu().numpy()
        done = iters <= end
        assert np.array_equal(st[done], final[done]) and np.all(st[~done] == P.RUNNING), end
    assert np.array_equal(P.solve_workload(batch)["status"], final)
    s.set_round_events([])
    s.close()
