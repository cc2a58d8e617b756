"""Condensed-QP interior-point oracle (FP64).  Test infrastructure only.

Problem (Sec. III, the LTV-MPC standard form, C = I):

    min  sum_{k=0}^{N-1} 1/2 ||xi_{k+1} - r^y_k||^2_{Q_k} + 1/2 ||u_k - r^u_k||^2_{R_k}
    s.t. xi_{k+1} = A_k xi_k + B_k u_k + e_k,   xi_0 given,
         u_k in U_k = product over contacts of a generalized pyramid
                      {(t, n): |t_j| <= c_j n, 0 <= n <= n_max} (stance)
                      or {0} (swing).

The states are eliminated (condensing): X = Gamma U + X_free, giving a dense
strictly convex QP in the stance inputs only, min 1/2 U'HU + c'U s.t. GU <= h,
(state boxes lo_k <= xi_{k+1} <= hi_k, where given, are rows of G on
Gamma U), solved by Mehrotra's predictor-corrector primal-dual interior-point method
(Nocedal & Wright, Numerical Optimization, 2nd ed., Alg. 16.4).  numpy's
dense solve serves as the linear-algebra step.
"""
from __future__ import annotations

import dataclasses
import os
from concurrent.futures import ProcessPoolExecutor
from typing import Optional, Sequence

import numpy as np

from paper_2606_05687_b300.workload import Batch

from . import project as _project


@dataclasses.dataclass
class Instance:
    """One MPC problem in float64 (promoted from the float32 batch)."""

    A: np.ndarray      # [N,nx,nx]
    Bm: np.ndarray     # [N,nx,nu]
    e: np.ndarray      # [N,nx]
    Q: np.ndarray      # [N,nx] diagonal
    R: np.ndarray      # [N,nu] diagonal
    ry: np.ndarray     # [N,nx]
    ru: np.ndarray     # [N,nu]
    mu: np.ndarray     # [N,nc]
    fmax: np.ndarray   # [N,nc]
    stance: np.ndarray  # bool [N,nc]
    xi0: np.ndarray    # [nx]
    contact_dim: int
    C: Optional[np.ndarray] = None  # [N,nx] diagonal output map of the cost ||C xi - r^y||_Q (None = I)
    xlo: Optional[np.ndarray] = None  # [N,nx] state box lo_k <= xi_{k+1} (None / -inf = unbounded)
    xhi: Optional[np.ndarray] = None  # [N,nx] state box xi_{k+1} <= hi_k (None / +inf = unbounded)

    def cdiag(self) -> np.ndarray:
        return np.ones_like(self.Q) if self.C is None else self.C

    @property
    def N(self):
        return self.A.shape[0]

    @property
    def nx(self):
        return self.A.shape[1]

    @property
    def nu(self):
        return self.Bm.shape[2]

    @property
    def nc(self):
        return self.mu.shape[1]


def instance(batch: Batch, b: int) -> Instance:
    f = lambda x: np.asarray(x[b], dtype=np.float64)
    N = int(batch.horizon[b])
    st = batch.stance()[b]
    return Instance(A=f(batch.A)[:N], Bm=f(batch.Bm)[:N], e=f(batch.e)[:N],
                    Q=f(batch.Q)[:N], R=f(batch.R)[:N], ry=f(batch.ry)[:N],
                    ru=f(batch.ru)[:N], mu=f(batch.mu)[:N], fmax=f(batch.fmax)[:N],
                    stance=st[:N], xi0=f(batch.xi0), contact_dim=batch.contact_dim)


def contact_faces(contact_dim: int, mu: float, fmax: float):
    """Rows (G_i, h_i) of the inequalities G_i u_i <= h_i of one stance contact,
    u_i its contact_dim components (oracle.project.faces: for each tangential j,
    +t_j - c_j n <= 0 and -t_j - c_j n <= 0; then -n <= 0 and n <= n_max)."""
    return _project.faces(contact_dim, mu, fmax)


def condense(inst: Instance):
    """X = Gamma U + X_free with X = [xi_1..xi_N], U = [u_0..u_{N-1}]."""
    N, nx, nu = inst.N, inst.nx, inst.nu
    Gamma = np.zeros((N * nx, N * nu))
    Xf = np.zeros(N * nx)
    x = inst.xi0.copy()
    prev = np.zeros((nx, N * nu))
    for k in range(N):
        x = inst.A[k] @ x + inst.e[k]
        Xf[k * nx:(k + 1) * nx] = x
        row = inst.A[k] @ prev
        row[:, k * nu:(k + 1) * nu] += inst.Bm[k]
        Gamma[k * nx:(k + 1) * nx] = row
        prev = row
    return Gamma, Xf


def assemble(inst: Instance):
    """Dense QP in the stance input components: (H, c, G, h, keep)."""
    N, nx, nu, cd = inst.N, inst.nx, inst.nu, inst.contact_dim
    Gamma, Xf = condense(inst)
    Qd = inst.Q.reshape(-1)
    Cd = inst.cdiag().reshape(-1)
    Rd = inst.R.reshape(-1)
    # 1/2 ||C X - r||^2_Q = 1/2 X'(C Q C)X - (C Q r)'X + const, X = Gamma U + Xf
    H = Gamma.T @ ((Cd * Qd * Cd)[:, None] * Gamma) + np.diag(Rd)
    c = Gamma.T @ (Cd * Qd * (Cd * Xf - inst.ry.reshape(-1))) - Rd * inst.ru.reshape(-1)
    keep = np.zeros(N * nu, dtype=bool)
    for k in range(N):
        for i in range(inst.nc):
            if inst.stance[k, i]:
                keep[k * nu + i * cd:k * nu + (i + 1) * cd] = True
    pos = -np.ones(N * nu, dtype=np.int64)
    pos[keep] = np.arange(keep.sum())
    Grows, hrows = [], []
    for k in range(N):
        for i in range(inst.nc):
            if not inst.stance[k, i]:
                continue
            Gi, hi = contact_faces(cd, inst.mu[k, i], inst.fmax[k, i])
            cols = pos[k * nu + i * cd:k * nu + (i + 1) * cd]
            for r in range(Gi.shape[0]):
                row = np.zeros(keep.sum())
                row[cols] = Gi[r]
                Grows.append(row)
                hrows.append(hi[r])
    nk = int(keep.sum())
    # state boxes X_k on xi_{k+1} = (Gamma U + Xf) rows: finite bounds become rows
    Gk = Gamma[:, keep]
    for lim, sgn in ((inst.xhi, 1.0), (inst.xlo, -1.0)):
        if lim is None:
            continue
        flat = np.asarray(lim, dtype=np.float64).reshape(-1)
        for idx in np.flatnonzero(np.isfinite(flat)):
            Grows.append(sgn * Gk[idx])
            hrows.append(sgn * (flat[idx] - Xf[idx]))
    G = np.array(Grows).reshape(len(Grows), nk)
    h = np.array(hrows)
    return H[np.ix_(keep, keep)], c[keep], G, h, keep


def ipm(H, c, G, h, tol=1e-13, max_iter=200):
    """Mehrotra predictor-corrector for min 1/2 x'Hx + c'x s.t. Gx <= h.

    Returns (x, lam, iterations).  Residuals: r_d = Hx + c + G'lam,
    r_p = Gx + s - h, complementarity mu = s'lam/m, each measured relative to
    the size of the terms that form it.  The iterate with the smallest
    relative residual is returned if the Newton system becomes numerically
    singular before the tolerance is met."""
    n, m = H.shape[0], G.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros(m), 0
    x = np.linalg.solve(H, -c)
    if m == 0:
        return x, np.zeros(0), 0
    s = h - G @ x
    s = np.maximum(s, 1.0)
    lam = np.ones(m)
    best = (np.inf, x, lam, 0)
    for it in range(1, max_iter + 1):
        Hx, Gl = H @ x, G.T @ lam
        rd = Hx + c + Gl
        rp = G @ x + s - h
        mu = s @ lam / m
        scale_d = 1.0 + max(np.abs(c).max(), np.abs(Hx).max(), np.abs(Gl).max())
        scale_p = 1.0 + max(np.abs(h).max(), np.abs(G @ x).max())
        merit = max(np.abs(rd).max() / scale_d, np.abs(rp).max() / scale_p, mu / scale_d)
        if merit < best[0]:
            best = (merit, x, lam, it)
        if merit <= tol:
            return x, lam, it
        W = lam / s
        K = H + G.T @ (W[:, None] * G)

        def direction(rc):
            rhs = -rd - G.T @ (W * rp) + G.T @ (rc / s)
            try:
                dx = np.linalg.solve(K, rhs)
            except np.linalg.LinAlgError:
                dx = np.linalg.lstsq(K, rhs, rcond=None)[0]
            dlam = W * (G @ dx + rp) - rc / s
            ds = -(rc + s * dlam) / lam
            return dx, ds, dlam

        def max_step(v, dv):
            neg = dv < 0
            return min(1.0, float(np.min(-v[neg] / dv[neg]))) if neg.any() else 1.0

        try:
            dx_a, ds_a, dl_a = direction(s * lam)
            a_aff = min(max_step(s, ds_a), max_step(lam, dl_a))
            mu_aff = (s + a_aff * ds_a) @ (lam + a_aff * dl_a) / m
            sigma = (mu_aff / mu) ** 3
            dx, ds, dl = direction(s * lam + ds_a * dl_a - sigma * mu)
        except np.linalg.LinAlgError:
            break
        if not (np.all(np.isfinite(dx)) and np.all(np.isfinite(dl))):
            break
        a = min(max_step(s, ds), max_step(lam, dl))
        a = min(1.0, 0.995 * a)
        x = x + a * dx
        s = s + a * ds
        lam = lam + a * dl
    return best[1], best[2], best[3]


@dataclasses.dataclass
class Solution:
    xi: np.ndarray     # [N,nx] states xi_1..xi_N
    u: np.ndarray      # [N,nu]
    iters: int
    objective: float


def objective(inst: Instance, xi: np.ndarray, u: np.ndarray) -> float:
    dx = inst.cdiag() * xi - inst.ry
    du = u - inst.ru
    return 0.5 * float(np.sum(inst.Q * dx * dx) + np.sum(inst.R * du * du))


def rollout(inst: Instance, u: np.ndarray) -> np.ndarray:
    xi = np.zeros((inst.N, inst.nx))
    x = inst.xi0
    for k in range(inst.N):
        x = inst.A[k] @ x + inst.Bm[k] @ u[k] + inst.e[k]
        xi[k] = x
    return xi


def crossover(H, c, G, h, x, lam, tol=1e-12, max_changes=50):
    """Exact solve on the interior-point method's active set.

    Faces whose multiplier exceeds their slack start as equalities.  The
    equality-constrained QP is solved through its KKT system (least squares,
    since degenerate vertices give dependent rows).  If an inactive face is
    violated it joins the set; if the point admits no non-negative
    multipliers (non-negative least squares leaves a stationarity residual)
    the face with the most negative least-squares multiplier leaves it -- the
    steps of a primal active-set method, warm-started at the IPM's guess.
    Returns the accepted point (feasible, stationary with multipliers >= 0)
    or None."""
    from scipy.optimize import nnls
    if G.shape[0] == 0:
        return None
    n = H.shape[0]
    scale_p = 1.0 + np.abs(h).max()
    act = lam > (h - G @ x)
    for _ in range(max_changes):
        idx = np.flatnonzero(act)
        GA, hA = G[idx], h[idx]
        m = len(idx)
        K = np.block([[H, GA.T], [GA, np.zeros((m, m))]])
        sol = np.linalg.lstsq(K, np.concatenate([-c, hA]), rcond=None)[0]
        xp, mls = sol[:n], sol[n:]
        viol = G @ xp - h
        viol[idx] = -np.inf
        if viol.max() > tol * scale_p:
            act[int(np.argmax(viol))] = True
            continue
        g = H @ xp + c
        scale_d = 1.0 + max(np.abs(c).max(), np.abs(H @ xp).max())
        if m:
            mult, _ = nnls(GA.T, -g, maxiter=50 * m)
            g = g + GA.T @ mult
        if np.abs(g).max() <= tol * scale_d:
            return xp
        if m == 0:
            return None
        act[idx[int(np.argmin(mls))]] = False
    return None


def solve_instance(inst: Instance, tol: float = 1e-13) -> Solution:
    H, c, G, h, keep = assemble(inst)
    x, lam, it = ipm(H, c, G, h, tol=tol)
    if x.size:
        xp = crossover(H, c, G, h, x, lam)
        if xp is not None:
            x = xp
    U = np.zeros(inst.N * inst.nu)
    U[keep] = x
    u = U.reshape(inst.N, inst.nu)
    xi = rollout(inst, u)
    return Solution(xi=xi, u=u, iters=it, objective=objective(inst, xi, u))


def _solve_one(args):
    batch, b = args
    return solve_instance(instance(batch, b))


def solve_batch(batch: Batch, instances: Optional[Sequence[int]] = None,
                workers: int = 1):
    """Solve the listed instances; returns (xi [n,N,nx], u [n,N,nu], iters [n])."""
    ids = list(range(batch.B)) if instances is None else list(instances)
    if workers > 1 and len(ids) > 1:
        import multiprocessing as mp
        with ProcessPoolExecutor(max_workers=workers,
                                 mp_context=mp.get_context("spawn")) as ex:
            sols = list(ex.map(_solve_one, [(batch.subset([b]), 0) for b in ids],
                               chunksize=max(1, len(ids) // (4 * workers))))
    else:
        sols = [solve_instance(instance(batch, b)) for b in ids]
    xi = np.stack([s.xi for s in sols])
    u = np.stack([s.u for s in sols])
    it = np.array([s.iters for s in sols])
    return xi, u, it


def default_workers() -> int:
    return max(1, len(os.sched_getaffinity(0)))
