"""Horizons above 32 stages: the ADMM round runs as a thread-block cluster
of two CTAs per instance, half of the stages in each.  Parity with the
oracle for ragged horizons U{5..40}, for the edge horizons 1, 2, 3, 33, 63
and 64 of a 64-stage batch (one CTA of the pair empty; the 640- and the
1024-thread forms), a warm restart at 40 stages, instances of 32 stages
or fewer, which a 32-stage handle solves with the one-CTA form, the
stall stop of an instance whose certificate sits at its FP32 floor, and an
instance whose refinement used to cycle through face sets."""
import dataclasses

import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

from oracle import kkt as okkt
from oracle import qp
from parity_util import KKT_TOL, OBJ_GAP, REL_TRAJ, compare, oracle_refs

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


def _first_stages(batch, n):
    """The batch cut to its first n stages (horizons must be n or fewer)."""
    assert int(batch.horizon.max()) <= n
    kw = {}
    for f in dataclasses.fields(batch):
        v = getattr(batch, f.name)
        kw[f.name] = v if f.name in ("spec", "xi0", "u_prev", "horizon", "nu_arr") else np.ascontiguousarray(v[:, :n])
    kw["spec"] = dataclasses.replace(batch.spec, N=n)
    return W.Batch(**kw)


def test_max_horizon_reports_pairs(pinmpc):
    lib = pinmpc.load()
    assert lib.mpc_max_horizon(13, 24) == 64 and lib.mpc_max_horizon(13, 12) == 64


def test_ragged_horizons_up_to_40(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=128, N=40, seed=81, horizon_min=5))
    out = pinmpc.solve_workload(batch)
    assert np.all(out["status"] == 0), np.flatnonzero(out["status"])
    h = batch.horizon
    ids = [int(np.argmin(h)), int(np.argmax(h))] + [int(i) for i in np.flatnonzero(h == 33)[:1]]
    ids += [int(i) for i in np.flatnonzero((h > 32) & (h < 40))[:3]] + [int(i) for i in np.flatnonzero(h <= 32)[:2]]
    compare(batch, out, ids)
    # instances of 32 stages or fewer: the same solution from a 32-stage
    # handle, which runs the one-CTA form
    short = [int(i) for i in np.flatnonzero(h <= 32)[:8]]
    sub = _first_stages(batch.subset(short), 32)
    one = pinmpc.solve_workload(sub)
    assert np.all(one["status"] == 0)
    for t, b in enumerate(short):
        n = int(h[b])
        su = np.abs(out["u"][b, :n]).max()
        assert np.abs(one["u"][t, :n] - out["u"][b, :n]).max() <= 2 * REL_TRAJ * su


def test_edge_horizons_64(pinmpc):
    batch = W.generate(W.small_centroidal(B=16, N=64, seed=83))
    batch.horizon[:6] = [1, 2, 3, 33, 63, 64]
    out = pinmpc.solve_workload(batch)
    ids = list(range(6))
    compare(batch, out, ids)
    # shorter horizons leave the outputs past them zero
    assert np.all(out["u"][0, 1:] == 0) and np.all(out["xi"][3, 33:] == 0)


def test_warm_restart_40(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=64, N=40, seed=85))
    s = pinmpc.solver_for(batch)
    cold = pinmpc.solve_workload(batch, solver=s)
    s.warm_start(0)
    warm = pinmpc.solve_workload(batch, solver=s)
    assert np.all(cold["status"] == 0) and np.all(warm["status"] == 0)
    assert warm["iters"].max() <= s.cfg.check_start
    ids = [0, 21, 63]
    refs = oracle_refs(batch, ids)
    compare(batch, cold, ids, refs)
    compare(batch, warm, ids, refs)


def test_stalled_instance_returns_its_polished_point(pinmpc):
    """Past ~40 stages the FP32 floor of the certificate can sit just above
    kkt_tol on the right faces: instance 54 of this 48-stage walking batch
    polishes to a point 1e-6 from the optimum whose certificate is 2.5e-6
    against the 2e-6 tolerance, and no later polish can do better (the
    faces of the iterate do not change).  It stops once its faces have held
    for two checks after that polish, with status STALLED and the polished
    point, which meets the oracle bars; it used to run to the iteration cap
    and return the ADMM iterate (KKT 0.57).  No instance of the batch ends
    at the cap."""
    batch = W.generate(W.rl_scale_walking(B=1024, N=48, seed=125))
    out = pinmpc.solve_workload(batch)
    st = out["status"]
    assert set(np.unique(st).tolist()) <= {pinmpc.CONVERGED, pinmpc.STALLED}, np.unique(st)
    sub = batch.subset([54])
    s = pinmpc.solver_for(sub)
    tol, cap = s.cfg.kkt_tol, s.cfg.max_iter
    one = pinmpc.solve_workload(sub, solver=s)
    s.close()
    assert st[54] == pinmpc.STALLED and one["status"][0] == pinmpc.STALLED
    assert one["iters"][0] < cap
    assert tol < one["kkt"][0] <= 4 * tol
    inst = qp.instance(sub, 0)
    sol = qp.solve_instance(inst)
    u = one["u"][0].astype(np.float64)
    xi = one["xi"][0].astype(np.float64)
    rep = okkt.kkt_residual(inst, xi, u)
    assert np.abs(u - sol.u).max() <= REL_TRAJ * np.abs(sol.u).max()
    assert np.abs(xi - sol.xi).max() <= REL_TRAJ * np.abs(sol.xi).max()
    assert rep.kkt <= KKT_TOL
    assert abs(qp.objective(inst, xi, u) - sol.objective) <= OBJ_GAP * abs(sol.objective)
    # the device certificate is the oracle checker's figure
    assert abs(one["kkt"][0] - rep.kkt) <= 0.2 * rep.kkt + 5e-7


def test_refinement_breaks_an_active_set_cycle(pinmpc):
    """Instance 2859 of this 64-stage walking batch cycled through face sets
    in the refinement (89 polishes) and certified only at the last check,
    iteration 1000.  A longer refinement step after two refinements in a row
    that do not improve the certificate, a face set already polished in the
    call retried with a longer step, and the longer step from round 4 on
    certify it at iteration 152 (12 polishes); the result matches the
    oracle."""
    batch = W.generate(W.rl_scale_walking(B=4096, N=64, seed=1077))
    sub = batch.subset([2859])
    out = pinmpc.solve_workload(sub)
    assert out["status"][0] == pinmpc.CONVERGED
    assert out["iters"][0] <= 312 and out["polishes"][0] <= 32, (out["iters"][0], out["polishes"][0])
    compare(sub, out, [0])


def test_stalled_points_meet_the_oracle_bars(pinmpc):
    """Every instance of the 64-stage walking batch that stalls (15 of 4096,
    each at the certificate's FP32 floor) returns a point within the oracle
    bars: u and xi within 1e-4, the checker's KKT within 1e-5, the objective
    within 1e-6 (measured worst: 1.3e-6, 3.7e-6, 6.8e-8)."""
    batch = W.generate(W.rl_scale_walking(B=4096, N=64, seed=1077))
    out = pinmpc.solve_workload(batch)
    ids = np.flatnonzero(out["status"] == pinmpc.STALLED)
    assert 0 < len(ids) <= 40, len(ids)
    assert np.all((out["status"] == pinmpc.CONVERGED) | (out["status"] == pinmpc.STALLED))
    for b in ids:
        inst = qp.instance(batch, int(b))
        sol = qp.solve_instance(inst)
        u = out["u"][b].astype(np.float64)
        xi = out["xi"][b].astype(np.float64)
        rep = okkt.kkt_residual(inst, xi, u)
        assert np.abs(u - sol.u).max() <= REL_TRAJ * np.abs(sol.u).max(), b
        assert np.abs(xi - sol.xi).max() <= REL_TRAJ * np.abs(sol.xi).max(), b
        assert rep.kkt <= KKT_TOL, (b, rep.kkt)
        assert abs(qp.objective(inst, xi, u) - sol.objective) <= OBJ_GAP * abs(sol.objective), b
