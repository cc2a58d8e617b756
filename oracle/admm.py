"""The parallel-in-horizon ADMM of Sec. III in FP64 (test infrastructure only).

Imported by the tests and the benchmark's CPU legs, never by the product
path; it shares no code with the CUDA kernels.  Everything is written from
the section's definitions, stage by stage, with dense matrices:

  lifted state    xibar_k = [xi_k; u_{k-1}],
                  Abar_k = [[A_k, B_k], [0, I]],  Bbar_k = [B_k; I],  ebar_k = [e_k; 0];
  cost            1/2 xibar_{k+1}' Qbar_k xibar_{k+1} - qbar_k' xibar_{k+1},
                  Qbar_k = blkdiag(Q_k, R_k), qbar_k = [Q_k r^y_k; R_k r^u_k]
                  (C = I; the stage index on Qbar / qbar is a reading: Q_k is
                  stage-indexed in the standard form);
  splitting       z_{k+1} = xibar_{k+1},  v_k = Bbar_k du_k,
                  z_{k+1} - Abar_k xibar_k - v_k - ebar_k = 0;
  caches          J_k = (Bbar_k' Bbar_k)^{-1} Bbar_k',
                  H_k = (Qbar_k + rho I + rho Abar_{k+1}' Abar_{k+1})^{-1}  (k < N-1),
                  H_{N-1} = (Qbar_{N-1} + rho I)^{-1};
  block 1         du_k = J_k (v_k - beta_k),  xibar_{k+1} = H_k htilde_k,
                  htilde_k = qbar_k + rho (z_{k+1} - theta_k
                             + Abar_{k+1}' (z_{k+2} - v_{k+1} - ebar_{k+1} + lambda_{k+1}))
                  (the section prints ebar_k inside the bracket; stationarity of
                  the augmented Lagrangian in xibar_{k+1} gives ebar_{k+1}, which is
                  the reading used here and pinned by the tests);
  block 2         gamma_k  = Bbar_k du_k + beta_k - Abar_k xibar_k - ebar_k + lambda_k,
                  gtilde_k = xibar_{k+1} + theta_k + Abar_k xibar_k + ebar_k - lambda_k,
                  z_{k+1} = Proj_{X_k x U_k}((2 gtilde_k + gamma_k) / 3),
                  v_k = (z_{k+1} + gamma_k) / 2;
  duals           theta_k += xibar_{k+1} - z_{k+1},  beta_k += Bbar_k du_k - v_k,
                  lambda_k += z_{k+1} - Abar_k xibar_k - v_k - ebar_k.

xibar_0 = [xi_0; u_{-1}] is fixed (the velocity form needs the input applied
before the horizon; the optimum does not depend on it).  X_k is R^nx unless a
state box [lo_k, hi_k] is given (then the state part of z is clipped to it);
U_k is the product of the contact sets of oracle.project.

Acceleration (the section's second remark names Nesterov's scheme with
restart and defers the details): fast ADMM with restart of Goldstein,
O'Donoghue, Setzer and Baraniuk (2014), applied to the second block w = (z, v)
and the scaled duals y = (theta, beta, lambda).  The combined residual is
c_m = rho (||y_m - yhat_m||^2 + ||Bop (w_m - what_m)||^2), Bop being the
coefficients of (z, v) in the three constraint rows, Bop(dz, dv) =
(-dz, -dv, dz - dv).  With c_m < eta c_{m-1}: alpha_{m+1} =
(1 + sqrt(1 + 4 alpha_m^2)) / 2 and the next iteration starts from
w_m + (alpha_m - 1)/alpha_{m+1} (w_m - w_{m-1}) (the same for y); otherwise
alpha_{m+1} = 1, it starts from w_{m-1}, y_{m-1}, and c_m is replaced by
c_{m-1} / eta.

``augmented_lagrangian`` evaluates the section's L_rho directly (the second
sum read as (rho/2) sum ||Bbar_k du_k - v_k + beta_k||^2); the tests pin the
closed-form blocks by checking that each minimises it.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from . import project as proj


@dataclasses.dataclass
class Lifted:
    """The lifted problem of one instance (horizon N)."""

    Abar: np.ndarray   # [N, nb, nb]
    Bbar: np.ndarray   # [N, nb, nu]
    ebar: np.ndarray   # [N, nb]
    Qbar: np.ndarray   # [N, nb] diagonal of Qbar_k
    qbar: np.ndarray   # [N, nb]
    xibar0: np.ndarray  # [nb]
    stance: np.ndarray  # bool [N, nc]
    mu: np.ndarray     # [N, nc]
    fmax: np.ndarray   # [N, nc]
    contact_dim: int
    nx: int
    xlo: Optional[np.ndarray] = None  # [N, nx] state box of xi_{k+1}, or None
    xhi: Optional[np.ndarray] = None
    dx: float = proj.FOOT_HALF_LENGTH
    dy: float = proj.FOOT_HALF_WIDTH

    @property
    def N(self):
        return self.Abar.shape[0]

    @property
    def nb(self):
        return self.Abar.shape[1]

    @property
    def nu(self):
        return self.Bbar.shape[2]


def lift(inst, u_prev=None, xlo=None, xhi=None, dx=proj.FOOT_HALF_LENGTH,
         dy=proj.FOOT_HALF_WIDTH) -> Lifted:
    """Lifted matrices of an ``oracle.qp.Instance`` (u_prev = u_{-1}, default 0)."""
    N, nx, nu = inst.N, inst.nx, inst.nu
    nb = nx + nu
    Abar = np.zeros((N, nb, nb))
    Bbar = np.zeros((N, nb, nu))
    ebar = np.zeros((N, nb))
    for k in range(N):
        Abar[k, :nx, :nx] = inst.A[k]
        Abar[k, :nx, nx:] = inst.Bm[k]
        Abar[k, nx:, nx:] = np.eye(nu)
        Bbar[k, :nx] = inst.Bm[k]
        Bbar[k, nx:] = np.eye(nu)
        ebar[k, :nx] = inst.e[k]
    cd = np.ones_like(inst.Q) if getattr(inst, "C", None) is None else inst.C
    # cost 1/2 ||C xi - r^y||^2_Q on the state part: C'QC and C'Q r^y (C diagonal)
    Qbar = np.concatenate([cd * inst.Q * cd, inst.R], axis=1)
    qbar = np.concatenate([cd * inst.Q * inst.ry, inst.R * inst.ru], axis=1)
    up = np.zeros(nu) if u_prev is None else np.asarray(u_prev, dtype=np.float64)
    if xlo is None and xhi is None and (getattr(inst, "xlo", None) is not None or getattr(inst, "xhi", None) is not None):
        xlo = inst.xlo if inst.xlo is not None else np.full((N, nx), -np.inf)
        xhi = inst.xhi if inst.xhi is not None else np.full((N, nx), np.inf)
    return Lifted(Abar=Abar, Bbar=Bbar, ebar=ebar, Qbar=Qbar, qbar=qbar,
                  xibar0=np.concatenate([inst.xi0, up]), stance=np.asarray(inst.stance, bool),
                  mu=inst.mu, fmax=inst.fmax, contact_dim=inst.contact_dim, nx=nx,
                  xlo=None if xlo is None else np.asarray(xlo, np.float64)[:N],
                  xhi=None if xhi is None else np.asarray(xhi, np.float64)[:N], dx=dx, dy=dy)


@dataclasses.dataclass
class Iterate:
    """ADMM variables of every stage k = 0..N-1: z[k] = z_{k+1}, v[k] = v_k,
    and the scaled duals theta[k], beta[k], lam[k] (each [N, nb])."""

    z: np.ndarray
    v: np.ndarray
    theta: np.ndarray
    beta: np.ndarray
    lam: np.ndarray

    @staticmethod
    def zeros(N, nb):
        return Iterate(*(np.zeros((N, nb)) for _ in range(5)))

    def copy(self):
        return Iterate(*(x.copy() for x in self.astuple()))

    def astuple(self):
        return (self.z, self.v, self.theta, self.beta, self.lam)


def caches(L: Lifted, rho: float):
    """J_k [N, nu, nb] and H_k [N, nb, nb] from their definitions."""
    N, nb = L.N, L.nb
    J = np.stack([np.linalg.solve(L.Bbar[k].T @ L.Bbar[k], L.Bbar[k].T) for k in range(N)])
    H = np.zeros((N, nb, nb))
    for k in range(N):
        M = np.diag(L.Qbar[k]) + rho * np.eye(nb)
        if k < N - 1:
            M = M + rho * L.Abar[k + 1].T @ L.Abar[k + 1]
        H[k] = np.linalg.inv(M)
    return J, H


def project_lifted(L: Lifted, x: np.ndarray) -> np.ndarray:
    """Projection of the lifted vectors x [N, nb] (row k = [xi_{k+1}; u_k]) onto
    X_k x U_k, every stage at once."""
    nx = L.nx
    out = np.empty_like(x)
    xs = x[:, :nx]
    if L.xlo is not None:
        xs = np.minimum(np.maximum(xs, L.xlo), L.xhi)
    out[:, :nx] = xs
    out[:, nx:] = proj.project_input(x[:, nx:], L.stance, L.mu, L.fmax, L.contact_dim, L.dx, L.dy)
    return out


def _mv(M, x):
    """Stage-wise matrix-vector products M[k] @ x[k]."""
    return np.einsum("kij,kj->ki", M, x)


def block1(L: Lifted, J, H, w: Iterate, rho: float, e_next: bool = True):
    """(du [N, nu], xibar [N+1, nb]) from the iterate w, every stage in
    parallel; xibar[0] = xibar_0.  e_next=False uses ebar_k inside htilde_k as
    printed (the tests' planted mistake)."""
    N = L.N
    du = _mv(J, w.v - w.beta)
    h = L.qbar + rho * (w.z - w.theta)
    if N > 1:
        eb = L.ebar[1:] if e_next else L.ebar[:-1]
        h[:-1] += rho * np.einsum("kji,kj->ki", L.Abar[1:], w.z[1:] - w.v[1:] - eb + w.lam[1:])
    xib = np.zeros((N + 1, L.nb))
    xib[0] = L.xibar0
    xib[1:] = _mv(H, h)
    return du, xib


def block2(L: Lifted, du, xib, w: Iterate):
    """(z, v) of the second block from block 1's du, xibar and the duals of w."""
    ax = _mv(L.Abar, xib[:-1])
    gam = _mv(L.Bbar, du) + w.beta - ax - L.ebar + w.lam
    gtl = xib[1:] + w.theta + ax + L.ebar - w.lam
    z = project_lifted(L, (2.0 * gtl + gam) / 3.0)
    v = 0.5 * (z + gam)
    return z, v


def dual_update(L: Lifted, du, xib, z, v, w: Iterate) -> Iterate:
    th = w.theta + xib[1:] - z
    be = w.beta + _mv(L.Bbar, du) - v
    la = w.lam + z - _mv(L.Abar, xib[:-1]) - v - L.ebar
    return Iterate(z=z, v=v, theta=th, beta=be, lam=la)


def step(L: Lifted, J, H, w: Iterate, rho: float, e_next: bool = True):
    """One ADMM iteration from w (the iterate the blocks read); returns
    (new iterate, du, xibar)."""
    du, xib = block1(L, J, H, w, rho, e_next)
    z, v = block2(L, du, xib, w)
    return dual_update(L, du, xib, z, v, w), du, xib


def combined_residual(new: Iterate, hat: Iterate, rho: float) -> float:
    dz = new.z - hat.z
    dv = new.v - hat.v
    dy = sum(float(np.sum((a - b) ** 2)) for a, b in
             ((new.theta, hat.theta), (new.beta, hat.beta), (new.lam, hat.lam)))
    dw = float(np.sum(dz ** 2) + np.sum(dv ** 2) + np.sum((dz - dv) ** 2))
    return rho * (dy + dw)


@dataclasses.dataclass
class Run:
    w: Iterate                 # last iterate w_m
    du: np.ndarray             # last block-1 du
    xib: np.ndarray            # last block-1 xibar [N+1, nb]
    iters: int
    restarts: int
    margins: list              # per iteration |c_m - eta c_{m-1}| / c_m (acceleration decisions)


def solve(L: Lifted, rho: float, iters: int, accel: bool = True, eta: float = 0.999,
          start: Optional[Iterate] = None, e_next: bool = True) -> Run:
    """``iters`` ADMM iterations from ``start`` (default: zeros), with or
    without the accelerated restart scheme above."""
    J, H = caches(L, rho)
    w = Iterate.zeros(L.N, L.nb) if start is None else start.copy()
    w_prev = w.copy()
    hat = w.copy()
    alpha, c_prev = 1.0, np.inf
    restarts = 0
    margins = []
    du = xib = None
    for _ in range(iters):
        new, du, xib = step(L, J, H, hat, rho, e_next)
        if accel:
            c = combined_residual(new, hat, rho)
            margins.append(abs(c - eta * c_prev) / max(c, 1e-300) if np.isfinite(c_prev) else np.inf)
            if c < eta * c_prev:
                a_next = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * alpha * alpha))
                wt = (alpha - 1.0) / a_next
                hat = Iterate(*(x + wt * (x - xp) for x, xp in zip(new.astuple(), w.astuple())))
                alpha, c_prev = a_next, c
            else:
                restarts += 1
                hat = w.copy()  # the iterate before the one just computed
                alpha, c_prev = 1.0, c_prev / eta
        else:
            hat = new
        w_prev, w = w, new
    return Run(w=w, du=du, xib=xib, iters=iters, restarts=restarts, margins=margins)


def primal(L: Lifted, w: Iterate, inst):
    """The output convention of the solver: u_k = the input part of z_{k+1}
    (feasible), xi the forward rollout of u through the (unlifted) dynamics."""
    nx = L.nx
    u = w.z[:, nx:].copy()
    xi = np.zeros((L.N, nx))
    x = inst.xi0
    for k in range(L.N):
        x = inst.A[k] @ x + inst.Bm[k] @ u[k] + inst.e[k]
        xi[k] = x
    return xi, u


def augmented_lagrangian(L: Lifted, du, xib, w: Iterate, rho: float) -> float:
    """L_rho of Sec. III at (du, xibar_{1..N}, z, v) with the scaled duals of w
    (xib[0] must be xibar_0); +inf if some z_{k+1} lies outside X_k x U_k."""
    N = L.N
    if np.abs(project_lifted(L, w.z) - w.z).max() > 1e-12 * (1.0 + np.abs(w.z).max()):
        return np.inf
    val = 0.0
    for k in range(N):
        x1 = xib[k + 1]
        val += 0.5 * float(x1 @ (L.Qbar[k] * x1)) - float(L.qbar[k] @ x1)
        r1 = x1 - w.z[k] + w.theta[k]
        r2 = L.Bbar[k] @ du[k] - w.v[k] + w.beta[k]
        r3 = w.z[k] - L.Abar[k] @ xib[k] - w.v[k] - L.ebar[k] + w.lam[k]
        val += 0.5 * rho * float(r1 @ r1 + r2 @ r2 + r3 @ r3)
    return val


def scaled_instance(inst, sigma: float):
    """The same problem in the input units u / sigma: B sigma, R sigma^2,
    r^u / sigma, n_max / sigma (the friction pyramid is a cone, so its
    coefficients do not change).  ADMM is not scale invariant, so an
    iteration run in these units is the one a solver working in u / sigma
    performs; the optimum maps back by u = sigma u_scaled."""
    import copy
    s = copy.copy(inst)
    s.Bm = inst.Bm * sigma
    s.R = inst.R * sigma * sigma
    s.ru = inst.ru / sigma
    s.fmax = inst.fmax / sigma
    return s
