"""Pins of the oracle's projection, active-face bits and ADMM (CPU only).

Each pin checks the oracle against something other than itself:
  * the closed-form projection (oracle.project) against a brute force over
    face subsets on random points and points at the apex, edges and faces,
    and against the hand-derived golden projections;
  * the active-face bits against hand-derived golden bits;
  * each ADMM block against the augmented Lagrangian of Sec. III that it
    must minimise (the Lagrangian is evaluated term by term from its
    definition, not from the closed forms), with a planted mistake (the
    printed ebar_k in htilde_k) that the pin catches;
  * the ADMM's fixed point against the interior-point oracle's optimum,
    which the LQR and brute-force pins of test_oracle.py hold in place.
"""
import os
import numpy as np
import pytest

from oracle import admm, kkt
from oracle import project as P
from oracle import qp
from paper_2606_05687_b300 import workload as W

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def special_points(rng, cd, mu, fmax, n):
    """Random points plus points at and near the apex, on edges (several
    tangential faces tight) and beyond n_max."""
    tang, coef, nrm = P.cone(cd, mu)
    pts = [rng.normal(size=(n, cd)) * fmax]
    pts.append(rng.normal(size=(n, cd)) * 1e-6 * fmax)           # near the apex
    pts.append(np.zeros((1, cd)))                                 # the apex
    e = np.zeros((n, cd))
    nn = rng.uniform(0.0, 1.2, size=n) * fmax
    e[:, nrm] = nn
    for j, c in zip(tang, coef):
        tight = rng.random(n) < 0.6
        e[:, j] = np.where(tight, rng.choice([-1.0, 1.0], size=n) * c * nn, rng.uniform(-1, 1, n) * c * nn)
    pts.append(e)                                                 # on faces and edges
    pts.append(e + rng.normal(size=(n, cd)) * 1e-7 * fmax)        # next to them
    return np.concatenate(pts)


@pytest.mark.parametrize("cd,n_pts", [(3, 20000), (6, 2000)])
def test_projection_matches_face_subset_bruteforce(cd, n_pts):
    rng = np.random.default_rng(11 + cd)
    total = 0
    for mu, fmax in ((0.5, 375.0), (0.9, 1500.0), (0.3, 1.0), (0.7, 100.0), (1.0, 10.0)):
        a = special_points(rng, cd, mu, fmax, n_pts // 5)
        x = P.project_many(a, cd, np.full(len(a), mu), np.full(len(a), fmax))
        y = P.project_bruteforce(a, cd, mu, fmax)
        scale = 1.0 + np.abs(a).max(axis=1) + fmax
        assert np.all(np.isfinite(y))
        err = np.abs(x - y).max(axis=1) / scale
        assert err.max() <= 1e-12, (mu, fmax, err.max(), a[np.argmax(err)])
        total += len(a)
    assert total >= n_pts


def test_projection_is_idempotent_and_nonexpansive():
    rng = np.random.default_rng(3)
    for cd in (3, 6):
        a = rng.normal(size=(4000, cd)) * 300.0
        b = rng.normal(size=(4000, cd)) * 300.0
        mu = rng.uniform(0.2, 1.0, 4000)
        fm = rng.uniform(10.0, 500.0, 4000)
        pa = P.project_many(a, cd, mu, fm)
        pb = P.project_many(b, cd, mu, fm)
        assert np.allclose(P.project_many(pa, cd, mu, fm), pa, rtol=0, atol=1e-9)
        assert np.all(np.linalg.norm(pa - pb, axis=1) <= np.linalg.norm(a - b, axis=1) * (1 + 1e-12) + 1e-9)


def load_projection_cases(name):
    cases = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, a, want = (part.split() for part in line.split("|"))
            cases.append((int(head[0]), float(head[1]), float(head[2]), np.array(a, float),
                          np.array(want, float)))
    return cases


def test_projection_golden_hand_derived():
    for cd, mu, fmax, a, want in load_projection_cases("projection_cases.txt"):
        x = P.project(a, cd, mu, fmax)
        assert np.allclose(x, want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max())), (cd, a, x, want)


def test_projection_golden_file_is_reproduced(tmp_path):
    """The committed oracle golden file is what its script writes today, and
    every row agrees with the brute force."""
    import runpy
    g = runpy.run_path(os.path.join(GOLDEN, "make_projection_golden.py"))
    g["main"].__globals__["OUT"] = str(tmp_path / "cases.txt")
    g["main"]()
    with open(tmp_path / "cases.txt") as fh, open(os.path.join(GOLDEN, "projection_oracle_cases.txt")) as ref:
        assert fh.read() == ref.read()
    for cd, mu, fmax, a, want in load_projection_cases("projection_oracle_cases.txt"):
        y = P.project_bruteforce(a[None], cd, mu, fmax)[0]
        scale = 1.0 + np.abs(a).max() + fmax
        assert np.abs(y - want).max() <= 1e-11 * scale


def load_face_cases():
    cases = []
    with open(os.path.join(GOLDEN, "active_faces.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, u, tail = (part.split() for part in line.split("|"))
            cases.append((int(head[0]), float(head[1]), float(head[2]), int(head[3]), np.array(u, float),
                          int(tail[0]), tail[1] == "1"))
    return cases


def one_contact_instance(cd, mu, fmax, contact, u_c):
    nc = 2 if cd == 6 else 8
    nu, nx = cd * nc, 13
    inst = qp.Instance(A=np.eye(nx)[None], Bm=np.zeros((1, nx, nu)), e=np.zeros((1, nx)),
                       Q=np.ones((1, nx)), R=np.ones((1, nu)), ry=np.zeros((1, nx)),
                       ru=np.zeros((1, nu)), mu=np.full((1, nc), mu), fmax=np.full((1, nc), fmax),
                       stance=np.zeros((1, nc), bool), xi0=np.zeros(nx), contact_dim=cd)
    inst.stance[0, contact] = True
    u = np.zeros((1, nu))
    u[0, contact * cd:(contact + 1) * cd] = u_c
    return inst, u


@pytest.mark.parametrize("case", load_face_cases())
def test_active_face_bits_golden(case):
    cd, mu, fmax, contact, u_c, want, _ = case
    inst, u = one_contact_instance(cd, mu, fmax, contact, u_c)
    bits, _ = kkt.active_faces(inst, u)
    assert int(bits[0]) == want, (bin(int(bits[0])), bin(want))


# ---------------------------------------------------------------- ADMM ----

SIGMA = 300.0


def lifted_case(maker, N, seed, b=0, e_scale=0.05, u_prev_scale=60.0, ru_scale=0.0):
    batch = W.generate(maker(B=b + 1, N=N, seed=seed, e_scale=e_scale, u_prev_scale=u_prev_scale))
    inst = qp.instance(batch, b)
    if ru_scale:
        inst.ru = np.random.default_rng(seed).normal(size=inst.ru.shape) * ru_scale
    si = admm.scaled_instance(inst, SIGMA)
    L = admm.lift(si, u_prev=batch.u_prev[b].astype(np.float64) / SIGMA)
    return inst, si, L


def random_iterate(rng, L, scale=0.3):
    w = admm.Iterate(*(rng.normal(size=(L.N, L.nb)) * scale for _ in range(5)))
    w.z = admm.project_lifted(L, w.z)
    return w


def al_of(L, du, xib, w, rho):
    return admm.augmented_lagrangian(L, du, xib, w, rho)


@pytest.mark.parametrize("maker", [W.rl_scale_walking, W.small_centroidal])
def test_block1_minimises_the_augmented_lagrangian(maker):
    """(du, xibar) of block 1 is the minimiser of L_rho over (du, xibar_{1..N})
    at fixed (z, v) and duals: L_rho(x + t d) = L_rho(x - t d) for every
    direction d (zero gradient of a quadratic), and moving costs."""
    inst, si, L = lifted_case(maker, 5, seed=21)
    rho = 100.0
    J, H = admm.caches(L, rho)
    rng = np.random.default_rng(0)
    w = random_iterate(rng, L)
    du, xib = admm.block1(L, J, H, w, rho)
    f0 = al_of(L, du, xib, w, rho)
    for _ in range(20):
        ddu = rng.normal(size=du.shape)
        dxb = rng.normal(size=xib.shape)
        dxb[0] = 0.0  # xibar_0 is data
        t = 1e-3
        fp = al_of(L, du + t * ddu, xib + t * dxb, w, rho)
        fm = al_of(L, du - t * ddu, xib - t * dxb, w, rho)
        curv = 0.5 * (fp + fm) - f0
        assert curv > 0.0
        assert abs(fp - fm) <= 1e-6 * curv + 1e-9 * abs(f0), (fp - fm, curv)


def test_printed_htilde_offset_is_caught():
    """The section prints ebar_k inside htilde_k; with e_k != 0 that update
    is not the minimiser, and the pin above rejects it."""
    inst, si, L = lifted_case(W.rl_scale_walking, 5, seed=21, e_scale=0.2)
    assert np.abs(L.ebar[1:] - L.ebar[:-1]).max() > 1e-3
    rho = 100.0
    J, H = admm.caches(L, rho)
    rng = np.random.default_rng(0)
    w = random_iterate(rng, L)
    du, xib = admm.block1(L, J, H, w, rho, e_next=False)
    f0 = al_of(L, du, xib, w, rho)
    worst = 0.0
    for _ in range(20):
        dxb = rng.normal(size=xib.shape)
        dxb[0] = 0.0
        t = 1e-3
        fp = al_of(L, du, xib + t * dxb, w, rho)
        fm = al_of(L, du, xib - t * dxb, w, rho)
        curv = 0.5 * (fp + fm) - f0
        worst = max(worst, abs(fp - fm) / curv)
    assert worst > 1e-2


@pytest.mark.parametrize("maker", [W.rl_scale_walking, W.small_centroidal])
def test_block2_minimises_the_augmented_lagrangian(maker):
    """(z, v) of block 2 minimises L_rho over z_{k+1} in X_k x U_k and free v_k
    (block 1's du, xibar and the duals fixed): no sampled feasible point
    nearby does better, and v is stationary."""
    inst, si, L = lifted_case(maker, 5, seed=22)
    rho = 100.0
    J, H = admm.caches(L, rho)
    rng = np.random.default_rng(1)
    w = random_iterate(rng, L, scale=1.0)
    du, xib = admm.block1(L, J, H, w, rho)
    z, v = admm.block2(L, du, xib, w)
    at = admm.Iterate(z=z, v=v, theta=w.theta, beta=w.beta, lam=w.lam)
    f0 = al_of(L, du, xib, at, rho)
    assert np.isfinite(f0)
    for t in (1e-1, 1e-3, 1e-5):
        for _ in range(30):
            z2 = admm.project_lifted(L, z + t * rng.normal(size=z.shape))
            v2 = v + t * rng.normal(size=v.shape)
            f = al_of(L, du, xib, admm.Iterate(z=z2, v=v2, theta=w.theta, beta=w.beta, lam=w.lam), rho)
            assert f >= f0 - 1e-9 * abs(f0), (t, f - f0)


@pytest.mark.parametrize("maker,N,seed,iters", [(W.rl_scale_walking, 6, 5, 3000),
                                                (W.small_centroidal, 6, 5, 3000),
                                                (W.rl_scale_walking, 12, 8, 4000)])
@pytest.mark.parametrize("accel", [True, False])
def test_admm_fixed_point_is_the_qp_optimum(maker, N, seed, iters, accel):
    """Run long in FP64, the iteration reaches the interior-point oracle's
    optimum (the unique minimiser of the strictly convex QP), with e_k != 0,
    r^u != 0 and u_{-1} != 0 -- the fixed point of the updates as written
    (with the ebar_{k+1} reading) is the QP's solution."""
    for b in (1, 2):
        inst, si, L = lifted_case(maker, N, seed, b=b, ru_scale=20.0)
        ref = qp.solve_instance(inst)
        rho = 300.0 if maker is W.small_centroidal else 100.0
        # plain ADMM converges linearly but more slowly than the accelerated form
        run = admm.solve(L, rho, iters if accel else 3 * iters, accel=accel)
        xi, u = admm.primal(L, run.w, si)
        u = u * SIGMA
        xi = qp.rollout(inst, u)
        scale = np.abs(ref.u).max()
        assert np.abs(u - ref.u).max() <= 1e-6 * scale, (b, np.abs(u - ref.u).max() / scale)
        assert kkt.kkt_residual(inst, xi, u).kkt <= 1e-7


def test_admm_fixed_point_does_not_depend_on_u_prev():
    """Two different u_{-1} (the velocity form's initial input) give the same
    optimum: Bbar has full column rank, so du <-> u is a bijection."""
    outs = []
    for ups in (0.0, 80.0):
        inst, si, L = lifted_case(W.rl_scale_walking, 6, 5, b=1, u_prev_scale=ups)
        run = admm.solve(L, 100.0, 3000, accel=True)
        outs.append(admm.primal(L, run.w, si)[1] * SIGMA)
    assert np.abs(outs[0] - outs[1]).max() <= 1e-6 * np.abs(outs[0]).max()


def test_checker_absolute_part_of_the_tolerance():
    """With c = kkt_tol_abs / kkt_tol every normalisation 1 + scale becomes
    c + scale: c = 1 is the default, and for a point off the optimum the
    reported residual falls as c grows (a larger absolute allowance)."""
    batch = W.generate(W.rl_scale_walking(B=1, N=6, seed=5))
    inst = qp.instance(batch, 0)
    sol = qp.solve_instance(inst)
    u = sol.u * (1.0 + 1e-4 * np.random.default_rng(0).normal(size=sol.u.shape))
    xi = qp.rollout(inst, u)
    k1 = kkt.kkt_residual(inst, xi, u).kkt
    assert kkt.kkt_residual(inst, xi, u, c=1.0).kkt == k1
    lo, hi = kkt.kkt_residual(inst, xi, u, c=1e3).kkt, kkt.kkt_residual(inst, xi, u, c=1e-3).kkt
    assert lo < k1 < hi
