"""GPU path (C ABI, CUDA) against the FP64 oracle on the same seeded inputs."""
import dataclasses

import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

from parity_util import KKT_TOL, compare, cone_violation, dynamics_residual

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


def test_small_centroidal_full_batch(pinmpc):
    """64 instances, N=10, two 6-D foot wrenches: every instance vs the oracle."""
    batch = W.generate(W.small_centroidal(B=64, N=10, seed=1001))
    out = pinmpc.solve_workload(batch)
    worst = compare(batch, out, list(range(batch.B)))
    print("small centroidal worst", worst, "iters mean", out["iters"].mean())


def test_rl_scale_subset(pinmpc):
    """256 instances of the walking workload (N=20, 8 point contacts); 48 sampled."""
    batch = W.generate(W.rl_scale_walking(B=256, N=20, seed=1002))
    out = pinmpc.solve_workload(batch)
    assert np.all(out["status"] == 0)
    ids = sorted(set(range(0, 256, 16)) | set(range(1, 256, 8)))
    worst = compare(batch, out, ids)
    print("rl scale worst", worst, "iters mean", out["iters"].mean())


def test_rl_scale_full_size_launch(pinmpc):
    """B=4096, N=20 in the benchmark's launch configuration: sampled instances
    against the oracle, and properties that hold for every instance."""
    batch = W.generate(W.rl_scale_walking(B=4096, N=20, seed=1002))
    out = pinmpc.solve_workload(batch)
    dyn = dynamics_residual(batch, out)
    viol, swing = cone_violation(batch, out)
    print("full size: status", np.unique(out["status"], return_counts=True), "kkt max", out["kkt"].max(),
          "iters mean", out["iters"].mean(), "max", out["iters"].max(), "polishes mean", out["polishes"].mean(),
          "dyn", dyn, "cone", viol, "swing", swing)
    assert np.all(out["status"] == 0), np.flatnonzero(out["status"])[:20]
    assert out["kkt"].max() <= KKT_TOL
    assert dyn <= 1e-6
    # face violations are part of the KKT residual (r_feas), so they share its bar
    assert viol <= KKT_TOL and swing == 0.0
    ids = [0, 1, 517, 1024, 2047, 2048, 3071, 4095]
    compare(batch, out, ids)


def test_edge_single_instance_and_single_stage(pinmpc):
    for spec in (W.rl_scale_walking(B=1, N=20, seed=5), W.rl_scale_walking(B=3, N=1, seed=6),
                 W.small_centroidal(B=2, N=1, seed=7)):
        batch = W.generate(spec)
        out = pinmpc.solve_workload(batch)
        compare(batch, out, list(range(batch.B)))


def test_ragged_horizons(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=24, N=20, seed=8))
    batch.horizon[:] = np.array([1 + (7 * b) % 20 for b in range(24)], dtype=np.int32)
    out = pinmpc.solve_workload(batch)
    compare(batch, out, list(range(24)))
    for b in range(24):
        h = batch.horizon[b]
        assert np.all(out["u"][b, h:] == 0) and np.all(out["xi"][b, h:] == 0)
        assert np.all(out["active_bits"][b, h:] == 0)


def test_all_swing_is_free_rollout(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=4, N=12, schedule="all_swing", seed=9, e_scale=0.02))
    out = pinmpc.solve_workload(batch)
    assert np.all(out["status"] == 0)
    assert np.all(out["u"] == 0)
    x = batch.xi0.astype(np.float64)
    for k in range(batch.N):
        x = np.einsum("bij,bj->bi", batch.A[:, k].astype(np.float64), x) + batch.e[:, k]
        assert np.allclose(out["xi"][:, k], x, rtol=1e-6, atol=1e-6)


def test_offsets_and_velocity_form_initial_input(pinmpc):
    """Non-zero e_k and r^u_k are honoured, and u_{-1} does not change the optimum."""
    spec = W.rl_scale_walking(B=16, N=20, seed=10, e_scale=0.02)
    batch = W.generate(spec)
    batch.ru[..., 2::3] = 50.0  # a normal-force reference
    out0 = pinmpc.solve_workload(batch)
    compare(batch, out0, list(range(16)))
    b2 = W.generate(dataclasses.replace(spec, u_prev_scale=80.0))
    b2.ru[..., 2::3] = 50.0
    out1 = pinmpc.solve_workload(b2)
    assert np.all(out1["status"] == 0)
    su = np.abs(out0["u"]).max()
    assert np.abs(out1["u"] - out0["u"]).max() <= 1e-4 * su


def test_bad_inputs_are_reported_per_instance(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=6, N=8, seed=11))
    batch.A[1, 3, 0, 0] = np.nan
    batch.fmax[2, 0, :] = -1.0
    batch.mask[2, 0] = 0xff
    batch.horizon[3] = 0
    batch.horizon[4] = 9
    out = pinmpc.solve_workload(batch)
    assert out["status"].tolist() == [0, 2, 3, 5, 5, 0]
    for b in (1, 2, 3, 4):
        assert np.all(out["u"][b] == 0) and np.all(out["xi"][b] == 0)
    compare(batch, out, [0, 5])


def test_host_buffers_match_device_buffers(pinmpc):
    import torch
    batch = W.generate(W.rl_scale_walking(B=32, N=20, seed=12))
    dev = pinmpc.solve_workload(batch)
    s = pinmpc.solver_for(batch)
    host = pinmpc.device_inputs(batch, pin_host=True)
    s.set_stages(batch.B, batch.N, **host)
    s.solve(batch.B)
    xi = np.empty((batch.B, batch.N, 13), np.float32)
    u = np.empty((batch.B, batch.N, batch.nu), np.float32)
    st = np.empty(batch.B, np.int32)
    s.get_traj(xi=xi, u=u, status=st)  # pageable memory: synchronous
    assert np.array_equal(xi, dev["xi"]) and np.array_equal(u, dev["u"])
    assert np.array_equal(st, dev["status"])
    # pinned memory: asynchronous, the results are there once the stream has passed the call
    pu = torch.empty((batch.B, batch.N, batch.nu), dtype=torch.float32).pin_memory()
    pst = torch.full((batch.B,), -7, dtype=torch.int32).pin_memory()
    s.set_stages(batch.B, batch.N, **host)
    s.solve(batch.B)
    s.get_traj(u=pu, status=pst)
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(pu.numpy(), dev["u"]) and np.array_equal(pst.numpy(), dev["status"])


def test_alone_equals_in_batch_and_repeatable(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=64, N=20, seed=13))
    full = pinmpc.solve_workload(batch)
    again = pinmpc.solve_workload(batch)
    assert np.array_equal(full["u"], again["u"])
    for b in (0, 17, 63):
        alone = pinmpc.solve_workload(batch.subset([b]))
        assert np.array_equal(alone["u"][0], full["u"][b])
        assert np.array_equal(alone["xi"][0], full["xi"][b])


def test_plain_admm_certificate_is_honest(pinmpc):
    """polish=0 certifies the ADMM iterate itself; its certificate agrees with
    the oracle's checker on the returned trajectory."""
    from oracle import kkt as okkt
    from oracle import qp
    batch = W.generate(W.small_centroidal(B=8, N=10, seed=14))
    out = pinmpc.solve_workload(batch, polish=0, max_iter=400, check_every=50, check_start=50)
    for b in range(batch.B):
        inst = qp.instance(batch, b)
        rep = okkt.kkt_residual(inst, out["xi"][b].astype(np.float64), out["u"][b].astype(np.float64))
        assert abs(out["kkt"][b] - rep.kkt) <= 0.2 * rep.kkt + 5e-7, (b, out["kkt"][b], rep.kkt)
        assert out["status"][b] in (0, 1)


def test_maximum_horizon_both_contact_models(pinmpc):
    """N = 32 (one warp per stage, the 1024-thread round kernel; records too
    large for the double-buffered TMA prefetch) for point contacts and wrenches."""
    assert pinmpc.load().mpc_max_horizon(13, 24) >= 32 and pinmpc.load().mpc_max_horizon(13, 12) >= 32
    for spec in (W.rl_scale_walking(B=24, N=32, seed=31), W.small_centroidal(B=24, N=32, seed=32)):
        batch = W.generate(spec)
        out = pinmpc.solve_workload(batch)
        assert np.all(out["status"] == 0), out["status"]
        compare(batch, out, [0, 5, 11, 23])


def test_large_batch_work_lists(pinmpc):
    """B = 16384: persistent round CTAs and list-indexed polish CTAs over four
    times the benchmark's batch; every instance certified, samples vs the oracle."""
    batch = W.generate(W.rl_scale_walking(B=16384, N=20, seed=33))
    out = pinmpc.solve_workload(batch)
    assert np.all(out["status"] == 0) and out["kkt"].max() <= KKT_TOL
    assert dynamics_residual(batch, out) <= 1e-6
    compare(batch, out, [0, 4095, 4096, 9999, 16383])


@pytest.mark.parametrize("spec", [W.centroidal9_walking(B=64, N=20, seed=41), W.centroidal9_small(B=64, N=10, seed=42)],
                         ids=["cd9-points", "cd9-wrenches"])
def test_nine_state_centroidal_model(pinmpc, spec):
    # the paper's own 9-state model (Sec. II-A), linearised, both contact models
    batch = W.generate(spec)
    out = pinmpc.solve_workload(batch)
    assert np.all(out["status"] == 0) and out["kkt"].max() <= KKT_TOL, out["status"]
    compare(batch, out, [0, 13, 31, 63])
