"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each pin checks the oracle against something other than itself:
  * the unconstrained case against the finite-horizon LQR tracking solution
    (backward Riccati recursion), a different algorithm on a different form;
  * tiny horizons against brute-force enumeration of active sets on the
    non-condensed KKT system;
  * a small case against scipy's SLSQP on the non-condensed problem;
  * invariants (cost scaling, all-swing instances, local optimality);
  * a planted mistake in the oracle (dropped e_k, transposed A_k) that the
    Riccati pin must catch.
"""
import dataclasses
import itertools

import numpy as np
import pytest
import scipy.optimize as so

from oracle import kkt, qp
from paper_2606_05687_b300 import workload as W


def lqr_tracking(inst: qp.Instance):
    """Finite-horizon LQR tracking solution by the backward Riccati recursion
    (no inequality constraints; every contact free)."""
    N = inst.N
    P = np.zeros((inst.nx, inst.nx))
    p = np.zeros(inst.nx)
    gains = [None] * N
    for k in range(N - 1, -1, -1):
        A, B, e = inst.A[k], inst.Bm[k], inst.e[k]
        R = np.diag(inst.R[k])
        Cm = np.diag(inst.cdiag()[k])
        S = Cm.T @ np.diag(inst.Q[k]) @ Cm + P
        s = Cm.T @ (inst.Q[k] * inst.ry[k]) + p
        M = R + B.T @ S @ B
        K = -np.linalg.solve(M, B.T @ S @ A)
        kap = np.linalg.solve(M, R @ inst.ru[k] + B.T @ (s - S @ e))
        P = A.T @ S @ (A + B @ K)
        p = A.T @ (s - S @ (B @ kap + e))
        gains[k] = (K, kap)
    x = inst.xi0.copy()
    xs, us = [], []
    for k in range(N):
        K, kap = gains[k]
        u = K @ x + kap
        x = inst.A[k] @ x + inst.Bm[k] @ u + inst.e[k]
        us.append(u)
        xs.append(x)
    return np.array(xs), np.array(us)


def standing_interior(inst: qp.Instance, r_weight=0.05):
    """Make the optimum interior: heavy input weight around an interior
    reference force (the body weight shared by the stance contacts)."""
    cd = inst.contact_dim
    inst.R = np.full_like(inst.R, r_weight)
    ru = np.zeros_like(inst.ru)
    for k in range(inst.N):
        n_st = max(int(inst.stance[k].sum()), 1)
        for i in range(inst.nc):
            if inst.stance[k, i]:
                ru[k, i * cd + 2] = W.MASS * W.GRAVITY / n_st
    inst.ru = ru
    return inst


def strictly_inside(inst, u, margin=1e-3):
    cd = inst.contact_dim
    for k in range(inst.N):
        for i in range(inst.nc):
            if not inst.stance[k, i]:
                continue
            G, h = qp.contact_faces(cd, inst.mu[k, i], inst.fmax[k, i])
            if np.any(G @ u[k, i * cd:(i + 1) * cd] - h > -margin):
                return False
    return True


@pytest.mark.parametrize("maker,e_scale", [(W.small_centroidal, 0.0), (W.small_centroidal, 0.05),
                                           (W.rl_scale_walking, 0.05)])
def test_unconstrained_equals_lqr(maker, e_scale):
    spec = maker(B=3, N=8, schedule="all_stance", e_scale=e_scale, seed=11)
    b = W.generate(spec)
    for i in range(b.B):
        inst = standing_interior(qp.instance(b, i))
        inst.ru[:, 0] += 3.0  # a non-zero tangential reference on the first contact
        xs, us = lqr_tracking(inst)
        assert strictly_inside(inst, us), "pin setup must leave every face inactive"
        sol = qp.solve_instance(inst)
        scale_u = np.abs(us).max()
        assert np.abs(sol.u - us).max() <= 1e-9 * scale_u
        assert np.abs(sol.xi - xs).max() <= 1e-9 * max(1.0, np.abs(xs).max())


def test_unconstrained_equals_lqr_with_output_map():
    """A diagonal output map C in the cost ||C xi - r^y||^2_Q (weights in
    [0.3, 2], some components dropped with C = 0) against the Riccati
    recursion with S = C'QC + P, s = C'Q r^y + p."""
    b = W.generate(W.rl_scale_walking(B=2, N=8, schedule="all_stance", e_scale=0.05, seed=13))
    rng = np.random.default_rng(13)
    for i in range(b.B):
        inst = standing_interior(qp.instance(b, i))
        inst.ru[:, 0] += 3.0
        inst.C = rng.uniform(0.3, 2.0, size=inst.Q.shape)
        inst.C[:, [5, 12]] = 0.0  # yaw and the gravity state out of the cost
        xs, us = lqr_tracking(inst)
        assert strictly_inside(inst, us)
        sol = qp.solve_instance(inst)
        assert np.abs(sol.u - us).max() <= 1e-9 * np.abs(us).max()
        # and C changes the answer (the pin is sensitive to it)
        plain = qp.solve_instance(dataclasses.replace(inst, C=None))
        assert np.abs(plain.u - us).max() > 1e-4 * np.abs(us).max()


@pytest.mark.parametrize("maker,N", [(W.small_centroidal, 40), (W.rl_scale_walking, 64)])
def test_unconstrained_equals_lqr_long_horizons(maker, N):
    """The same closed-form pin at the long horizons the two-CTA round serves."""
    b = W.generate(maker(B=1, N=N, schedule="all_stance", e_scale=0.05, seed=12))
    inst = standing_interior(qp.instance(b, 0))
    inst.ru[:, 0] += 3.0
    xs, us = lqr_tracking(inst)
    assert strictly_inside(inst, us), "pin setup must leave every face inactive"
    sol = qp.solve_instance(inst)
    assert np.abs(sol.u - us).max() <= 1e-8 * np.abs(us).max()
    assert np.abs(sol.xi - xs).max() <= 1e-8 * max(1.0, np.abs(xs).max())


def test_planted_mistakes_fail_lqr_pin(monkeypatch):
    """A dropped offset e_k or a transposed A_k in the oracle's condensing must
    make the LQR pin fail (the pin is sensitive to them)."""
    spec = W.rl_scale_walking(B=1, N=6, schedule="all_stance", e_scale=0.05, seed=12)
    inst = standing_interior(qp.instance(W.generate(spec), 0))
    xs, us = lqr_tracking(inst)
    orig = qp.condense

    def dropped_e(ins):
        saved = ins.e
        ins.e = np.zeros_like(saved)
        try:
            return orig(ins)
        finally:
            ins.e = saved

    def transposed_A(ins):
        saved = ins.A
        ins.A = np.swapaxes(saved, 1, 2).copy()
        try:
            return orig(ins)
        finally:
            ins.A = saved

    for bad in (dropped_e, transposed_A):
        monkeypatch.setattr(qp, "condense", bad)
        sol = qp.solve_instance(inst)
        assert np.abs(sol.u - us).max() > 1e-6 * np.abs(us).max()
    monkeypatch.setattr(qp, "condense", orig)


def full_kkt_bruteforce(inst: qp.Instance):
    """Enumerate every working set of the face inequalities on the
    non-condensed problem in z = (xi_1..xi_N, u_0..u_{N-1}); return the
    unique primal point that is feasible with non-negative multipliers."""
    N, nx, nu, cd = inst.N, inst.nx, inst.nu, inst.contact_dim
    nz = N * nx + N * nu
    xi_idx = lambda k: slice(k * nx, (k + 1) * nx)          # xi_{k+1}
    u_idx = lambda k: slice(N * nx + k * nu, N * nx + (k + 1) * nu)
    H = np.zeros((nz, nz))
    g = np.zeros(nz)
    for k in range(N):
        H[xi_idx(k), xi_idx(k)] = np.diag(inst.Q[k])
        g[xi_idx(k)] = -inst.Q[k] * inst.ry[k]
        H[u_idx(k), u_idx(k)] = np.diag(inst.R[k])
        g[u_idx(k)] = -inst.R[k] * inst.ru[k]
    Eq, eq = [], []
    for k in range(N):            # xi_{k+1} - A_k xi_k - B_k u_k = e_k (+ A_0 xi_0)
        for r in range(nx):
            row = np.zeros(nz)
            row[xi_idx(k).start + r] = 1.0
            if k > 0:
                row[xi_idx(k - 1)] -= inst.A[k][r]
            row[u_idx(k)] -= inst.Bm[k][r]
            Eq.append(row)
            eq.append(inst.e[k][r] + (inst.A[0][r] @ inst.xi0 if k == 0 else 0.0))
    Ineq, ih = [], []
    for k in range(N):
        for i in range(inst.nc):
            cols = np.arange(u_idx(k).start + i * cd, u_idx(k).start + (i + 1) * cd)
            if not inst.stance[k, i]:
                for c in cols:
                    row = np.zeros(nz)
                    row[c] = 1.0
                    Eq.append(row)
                    eq.append(0.0)
                continue
            G, h = qp.contact_faces(cd, inst.mu[k, i], inst.fmax[k, i])
            for r in range(G.shape[0]):
                row = np.zeros(nz)
                row[cols] = G[r]
                Ineq.append(row)
                ih.append(h[r])
    for lim, sgn in ((inst.xhi, 1.0), (inst.xlo, -1.0)):   # state boxes on xi_{k+1}
        if lim is None:
            continue
        for k in range(N):
            for r in range(nx):
                if np.isfinite(lim[k, r]):
                    row = np.zeros(nz)
                    row[xi_idx(k).start + r] = sgn
                    Ineq.append(row)
                    ih.append(sgn * lim[k, r])
    Eq, eq, Ineq, ih = map(np.array, (Eq, eq, Ineq, ih))
    found = []
    m = len(ih)
    for active in itertools.product([False, True], repeat=m):
        act = np.array(active)
        C = np.vstack([Eq, Ineq[act]])
        d = np.concatenate([eq, ih[act]])
        nc = C.shape[0]
        K = np.block([[H, C.T], [C, np.zeros((nc, nc))]])
        rhs = np.concatenate([-g, d])
        sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
        if np.abs(K @ sol - rhs).max() > 1e-9 * (1 + np.abs(rhs).max()):
            continue
        z = sol[:nz]
        mult = sol[nz + len(eq):]
        if np.any(Ineq @ z - ih > 1e-9 * (1 + np.abs(ih).max())):
            continue
        if np.any(mult < -1e-9):
            continue
        found.append(z)
    assert found, "no KKT point found"
    z = found[0]
    for other in found[1:]:
        assert np.abs(other - z).max() <= 1e-7 * (1 + np.abs(z).max())
    xi = z[:N * nx].reshape(N, nx)
    u = z[N * nx:].reshape(N, nu)
    return xi, u


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_bruteforce_active_sets_tiny(seed):
    # N=2 with a single stance 3-D contact (6 faces per stage: 2^12 working sets)
    spec = W.rl_scale_walking(B=1, N=2, schedule="all_stance", seed=seed, ref_noise=1.0)
    inst = qp.instance(W.generate(spec), 0)
    inst.stance[:] = False
    inst.stance[:, 0] = True
    inst.fmax[:] = 150.0
    xi_b, u_b = full_kkt_bruteforce(inst)
    sol = qp.solve_instance(inst)
    assert np.abs(sol.u - u_b).max() <= 1e-8 * (1 + np.abs(u_b).max())
    assert np.abs(sol.xi - xi_b).max() <= 1e-8 * (1 + np.abs(xi_b).max())


@pytest.mark.parametrize("seed", [21])
def test_bruteforce_with_state_bounds(seed):
    """State boxes X_k as condensed rows: N = 2, one 3-D contact, and two
    bounds placed inside the unbounded optimum (so they bind), against the
    enumeration of every working set of faces and bounds (2^14) on the
    non-condensed problem; the checker's joint multipliers certify it."""
    spec = W.rl_scale_walking(B=1, N=2, schedule="all_stance", seed=seed, ref_noise=1.0)
    inst = qp.instance(W.generate(spec), 0)
    inst.stance[:] = False
    inst.stance[:, 0] = True
    inst.fmax[:] = 150.0
    free = qp.solve_instance(inst)
    inst.xhi = np.full((2, inst.nx), np.inf)
    inst.xlo = np.full((2, inst.nx), -np.inf)
    # v_x of xi_1 capped below its free value, v_z of xi_2 held above its free value
    inst.xhi[0, 6] = free.xi[0, 6] - 0.02 * (1 + abs(free.xi[0, 6]))
    inst.xlo[1, 8] = free.xi[1, 8] + 0.02 * (1 + abs(free.xi[1, 8]))
    xi_b, u_b = full_kkt_bruteforce(inst)
    sol = qp.solve_instance(inst)
    assert np.abs(sol.u - u_b).max() <= 1e-8 * (1 + np.abs(u_b).max())
    assert np.abs(sol.xi - xi_b).max() <= 1e-8 * (1 + np.abs(xi_b).max())
    # a bound binds (the first one moves the solution enough that the second may not)
    assert abs(sol.xi[0, 6] - inst.xhi[0, 6]) <= 1e-9 or abs(sol.xi[1, 8] - inst.xlo[1, 8]) <= 1e-9
    rep = kkt.kkt_residual(inst, sol.xi, sol.u)
    assert rep.kkt <= 1e-9, rep
    # the free optimum violates the boxes, and the checker says so
    assert kkt.kkt_residual(inst, free.xi, free.u).r_feas > 1e-3


def test_admm_fixed_point_with_state_bounds():
    """The Sec. III iteration with X_k a box (the state part of z clipped)
    reaches the same optimum as the interior-point oracle with box rows."""
    from oracle import admm
    batch = W.generate(W.rl_scale_walking(B=2, N=6, seed=5, e_scale=0.05))
    inst = qp.instance(batch, 1)
    free = qp.solve_instance(inst)
    inst.xhi = np.full((6, inst.nx), np.inf)
    inst.xhi[2:5, 8] = free.xi[2:5, 8].max() - 0.05   # cap v_z over three stages
    ref = qp.solve_instance(inst)
    assert np.any(np.abs(ref.xi[2:5, 8] - inst.xhi[2:5, 8]) <= 1e-8)
    si = admm.scaled_instance(inst, 300.0)
    L = admm.lift(si, u_prev=batch.u_prev[1].astype(np.float64) / 300.0)
    run = admm.solve(L, 100.0, 6000, accel=True)
    _, u = admm.primal(L, run.w, si)
    u = u * 300.0
    assert np.abs(u - ref.u).max() <= 1e-6 * np.abs(ref.u).max()
    assert kkt.kkt_residual(inst, ref.xi, ref.u).kkt <= 1e-9


def test_bruteforce_has_active_faces():
    """The tiny cases above exercise active constraints (otherwise the
    enumeration pins nothing beyond the unconstrained case)."""
    n_active = 0
    for seed in (21, 22, 23):
        spec = W.rl_scale_walking(B=1, N=2, schedule="all_stance", seed=seed, ref_noise=1.0)
        inst = qp.instance(W.generate(spec), 0)
        inst.stance[:] = False
        inst.stance[:, 0] = True
        inst.fmax[:] = 150.0
        sol = qp.solve_instance(inst)
        bits, _ = kkt.active_faces(inst, sol.u, tau=1e-9)
        n_active += sum(bin(int(x)).count("1") for x in bits)
    assert n_active >= 2


def test_slsqp_cross_check():
    """scipy's SLSQP on the non-condensed problem (states and inputs as
    variables, dynamics as equalities) agrees with the oracle."""
    spec = W.small_centroidal(B=1, N=3, seed=31, schedule="all_stance")
    inst = qp.instance(W.generate(spec), 0)
    N, nx, nu, cd = inst.N, inst.nx, inst.nu, inst.contact_dim
    su = 100.0  # optimise forces in units of 100 N for conditioning

    def split(z):
        return z[:N * nx].reshape(N, nx), su * z[N * nx:].reshape(N, nu)

    def f(z):
        xi, u = split(z)
        return qp.objective(inst, xi, u)

    def dyn(z):
        xi, u = split(z)
        out, prev = [], inst.xi0
        for k in range(N):
            out.append(xi[k] - inst.A[k] @ prev - inst.Bm[k] @ u[k] - inst.e[k])
            prev = xi[k]
        return np.concatenate(out)

    def faces(z):
        _, u = split(z)
        out = []
        for k in range(N):
            for i in range(inst.nc):
                G, h = qp.contact_faces(cd, inst.mu[k, i], inst.fmax[k, i])
                out.append(h - G @ u[k, i * cd:(i + 1) * cd])
        return np.concatenate(out) / su

    sol = qp.solve_instance(inst)
    z0 = np.concatenate([qp.rollout(inst, np.zeros((N, nu))).ravel(), np.zeros(N * nu)])
    res = so.minimize(f, z0, method="SLSQP",
                      constraints=[{"type": "eq", "fun": dyn}, {"type": "ineq", "fun": faces}],
                      options={"maxiter": 2000, "ftol": 1e-14})
    xi_s, u_s = split(res.x)
    assert res.success
    assert abs(f(res.x) - sol.objective) <= 1e-6 * abs(sol.objective)
    assert np.abs(u_s - sol.u).max() <= 2e-3 * np.abs(sol.u).max()


@pytest.mark.parametrize("maker", [W.small_centroidal, W.rl_scale_walking])
def test_kkt_of_oracle_and_cost_scaling(maker):
    b = W.generate(maker(B=3, seed=41))
    for i in range(b.B):
        inst = qp.instance(b, i)
        sol = qp.solve_instance(inst)
        rep = kkt.kkt_residual(inst, sol.xi, sol.u)
        assert rep.kkt <= 1e-10
        # scaling Q and R by a common s > 0 leaves the optimum unchanged
        inst2 = qp.instance(b, i)
        inst2.Q = inst2.Q * 7.5
        inst2.R = inst2.R * 7.5
        sol2 = qp.solve_instance(inst2)
        assert np.abs(sol2.u - sol.u).max() <= 1e-8 * np.abs(sol.u).max()


def test_all_swing_gives_free_rollout():
    spec = W.rl_scale_walking(B=2, N=10, schedule="all_swing", seed=51, e_scale=0.02)
    b = W.generate(spec)
    for i in range(b.B):
        inst = qp.instance(b, i)
        sol = qp.solve_instance(inst)
        assert np.all(sol.u == 0.0)
        x = inst.xi0
        for k in range(inst.N):
            x = inst.A[k] @ x + inst.e[k]
            assert np.allclose(sol.xi[k], x, rtol=0, atol=1e-12)


def test_local_optimality_sampling():
    """No feasible perturbation of the oracle's inputs lowers the cost."""
    rng = np.random.default_rng(0)
    b = W.generate(W.rl_scale_walking(B=1, N=6, seed=61))
    inst = qp.instance(b, 0)
    sol = qp.solve_instance(inst)
    base = sol.objective
    cd = inst.contact_dim
    tried = 0
    while tried < 200:
        du = rng.normal(0, 1.0, size=sol.u.shape) * inst.stance.repeat(cd, axis=1)
        for t in (1e-3, 1e-2, 1e-1):
            u = sol.u + t * du
            ok = True
            for k in range(inst.N):
                for i in range(inst.nc):
                    if inst.stance[k, i]:
                        G, h = qp.contact_faces(cd, inst.mu[k, i], inst.fmax[k, i])
                        ok &= bool(np.all(G @ u[k, i * cd:(i + 1) * cd] <= h))
            if ok:
                tried += 1
                assert qp.objective(inst, qp.rollout(inst, u), u) >= base - 1e-9 * abs(base)


def test_checker_detects_perturbations():
    b = W.generate(W.rl_scale_walking(B=1, N=10, seed=71))
    inst = qp.instance(b, 0)
    sol = qp.solve_instance(inst)
    # a non-optimal but feasible input sequence: scale the stance forces
    u = sol.u * 0.99
    assert kkt.kkt_residual(inst, qp.rollout(inst, u), u).r_stat > 1e-5
    # broken dynamics
    xi = sol.xi.copy()
    xi[3, 0] += 1e-3
    assert kkt.kkt_residual(inst, xi, sol.u).r_dyn > 5e-5  # 1e-3 / (1 + |g state| 9.81)
    # infeasible force on a swing contact
    st = inst.stance
    k, i = np.argwhere(~st)[0]
    u = sol.u.copy()
    u[k, i * 3 + 2] = 10.0
    assert kkt.kkt_residual(inst, qp.rollout(inst, u), u).r_feas > 1e-3
