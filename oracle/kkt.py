"""Primal-only KKT residual checker (FP64).  Test infrastructure only.

The paper defines no optimality measure; this follows the reading adopted for
the build (a KKT residual of the Sec. III standard-form QP computed from any
primal pair (xi, u), needing no duals from the solver):

  r_dyn  = max_k ||xi_{k+1} - A_k xi_k - B_k u_k - e_k||_inf
                 / (1 + max(||A_k xi_k||, ||B_k u_k||, ||e_k||, ||xi_{k+1}||)_inf)
  costates (from the Lagrangian term + y_k'(A_k xi_k + B_k u_k + e_k - xi_{k+1})):
           y_{N-1} = C Q_{N-1}(C xi_N - r_{N-1}),  y_k = C Q_k(C xi_{k+1} - r_k) + A_{k+1}' y_{k+1}
           (C the diagonal output map of the stage cost, I unless given)
  w_k    = R_k(u_k - r^u_k) + B_k' y_k           (gradient of the reduced cost)
  per stance contact i: mu_i >= 0 minimises ||w_i + G_i' mu||^2 + ||diag(g_i(u_i)) mu||^2
           (a non-negative least-squares problem; scipy's exact Lawson-Hanson
           active-set routine is the step that solves it)
  r_stat = max |w_i + G_i' mu_i| / (1 + max(||R(u - r^u)||_inf, ||B'y||_inf))
  r_comp = max |mu_ij g_ij(u_i)| / (1 + ||u||_inf)
  r_feas = max(max_ij g_ij(u_i), max |u_swing|, 0) / (1 + n_max)
  KKT    = max(r_dyn, r_feas, r_stat, r_comp)

With an absolute part (``c`` = kkt_tol_abs / kkt_tol, 1 by default) the
constant 1 in every normalisation becomes c: each term then reads
|residual| / (c + scale), so "KKT <= tol" means |residual| <= tol_abs + tol scale.

State boxes lo_k <= xi_{k+1} <= hi_k (where given) add the feasibility term
max(xi - hi, lo - xi, 0) / (c + |bound|) and multipliers nu_k >= 0 per
bound; those enter every earlier costate, so with boxes the multipliers of
all faces and bounds are found by one non-negative least-squares problem.

Swing contacts carry the equality u_i = 0, whose multiplier is free, so they
contribute no stationarity term.  Active faces (integer output): face j of a
stance contact is active iff g_j(u) >= -tau_act (1 + n_max), tau_act = 1e-5.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.optimize import nnls

from .qp import Instance, contact_faces

TAU_ACT = 1e-5


@dataclasses.dataclass
class KKTReport:
    kkt: float
    r_dyn: float
    r_feas: float
    r_stat: float
    r_comp: float


def costates(inst: Instance, xi: np.ndarray) -> np.ndarray:
    N = inst.N
    y = np.zeros((N, inst.nx))
    nxt = np.zeros(inst.nx)
    for k in range(N - 1, -1, -1):
        cd = inst.cdiag()[k]
        y[k] = cd * inst.Q[k] * (cd * xi[k] - inst.ry[k])
        if k + 1 < N:
            y[k] += inst.A[k + 1].T @ nxt
        nxt = y[k]
    return y


def kkt_residual(inst: Instance, xi: np.ndarray, u: np.ndarray, c: float = 1.0) -> KKTReport:
    xi = np.asarray(xi, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    N, cd = inst.N, inst.contact_dim
    r_dyn = 0.0
    prev = inst.xi0
    for k in range(N):
        ax = inst.A[k] @ prev
        bu = inst.Bm[k] @ u[k]
        res = xi[k] - ax - bu - inst.e[k]
        den = c + max(np.abs(ax).max(), np.abs(bu).max(), np.abs(inst.e[k]).max(),
                        np.abs(xi[k]).max())
        r_dyn = max(r_dyn, np.abs(res).max() / den)
        prev = xi[k]
    y = costates(inst, xi)
    Rdu = inst.R * (u - inst.ru)
    Bty = np.einsum("kij,ki->kj", inst.Bm, y)
    w = Rdu + Bty
    den_stat = c + max(np.abs(Rdu).max(), np.abs(Bty).max())
    den_comp = c + np.abs(u).max()
    r_stat = r_comp = r_feas = 0.0
    for k in range(N):
        for i in range(inst.nc):
            sl = slice(i * cd, (i + 1) * cd)
            fm = inst.fmax[k, i]
            if not inst.stance[k, i]:
                r_feas = max(r_feas, np.abs(u[k, sl]).max() / (c + fm))
                continue
            G, h = contact_faces(cd, inst.mu[k, i], fm)
            g = G @ u[k, sl] - h
            r_feas = max(r_feas, max(g.max(), 0.0) / (c + fm))
            M = np.vstack([G.T, np.diag(g)])
            rhs = np.concatenate([-w[k, sl], np.zeros(len(g))])
            mult, _ = nnls(M, rhs, maxiter=50 * M.shape[1])
            r_stat = max(r_stat, np.abs(w[k, sl] + G.T @ mult).max() / den_stat)
            r_comp = max(r_comp, np.abs(mult * g).max() / den_comp)
    if _has_box(inst):
        r_feas_b, r_stat, r_comp = _box_terms(inst, xi, u, w, den_stat, den_comp, c)
        r_feas = max(r_feas, r_feas_b)
    kkt = max(r_dyn, r_feas, r_stat, r_comp)
    return KKTReport(kkt=kkt, r_dyn=r_dyn, r_feas=r_feas, r_stat=r_stat, r_comp=r_comp)


def _has_box(inst: Instance) -> bool:
    return any(getattr(inst, a, None) is not None and np.isfinite(getattr(inst, a)).any() for a in ("xlo", "xhi"))


def _box_terms(inst: Instance, xi, u, w0, den_stat, den_comp, c):
    """KKT terms with state boxes: the multipliers of every stance face and
    every finite state bound are found together, since a bound's multiplier
    nu_j on xi_{j+1} enters every earlier costate,
        y_k = C Q_k (C xi_{k+1} - r_k) + A_{k+1}' y_{k+1} + nu_k,
        nu_k = nu_up_k - nu_lo_k,
    and through y_k the stationarity of every u_k, k <= j.  One non-negative
    least-squares problem over (mu, nu_up, nu_lo) minimises the stationarity
    residual of the stance inputs plus the complementarity terms g mu and
    slack nu.  Returns (r_feas of the boxes, r_stat, r_comp)."""
    N, nx, nu, cd = inst.N, inst.nx, inst.nu, inst.contact_dim
    lo = inst.xlo if inst.xlo is not None else np.full((N, nx), -np.inf)
    hi = inst.xhi if inst.xhi is not None else np.full((N, nx), np.inf)
    rows_u = [(k, j) for k in range(N) for j in range(nu) if inst.stance[k, j // cd]]
    ridx = {kj: r for r, kj in enumerate(rows_u)}
    cols, comp = [], []
    r_feas = 0.0
    # contact faces
    for k in range(N):
        for i in range(inst.nc):
            if not inst.stance[k, i]:
                continue
            G, h = contact_faces(cd, inst.mu[k, i], inst.fmax[k, i])
            g = G @ u[k, i * cd:(i + 1) * cd] - h
            for f in range(G.shape[0]):
                col = np.zeros(len(rows_u))
                for t in range(cd):
                    col[ridx[(k, i * cd + t)]] = G[f, t]
                cols.append(col)
                comp.append(g[f])
    n_face = len(cols)
    # state bounds: a unit multiplier on xi_{j+1, i} adds Phi(k, j) e_i to y_k
    # for k <= j (Phi(j, j) = I, Phi(k, j) = A_{k+1}' Phi(k+1, j)), hence
    # B_k' Phi(k, j) e_i to the stationarity of u_k
    for j in range(N):
        for i in range(nx):
            for lim, sgn in ((hi[j, i], 1.0), (lo[j, i], -1.0)):
                if not np.isfinite(lim):
                    continue
                slack = sgn * (xi[j, i] - lim)  # <= 0 when feasible
                r_feas = max(r_feas, max(slack, 0.0) / (c + abs(lim)))
                col = np.zeros(len(rows_u))
                e = np.zeros(nx)
                e[i] = sgn
                for k in range(j, -1, -1):
                    if k < j:
                        e = inst.A[k + 1].T @ e
                    bte = inst.Bm[k].T @ e
                    for t in range(nu):
                        if (k, t) in ridx:
                            col[ridx[(k, t)]] = bte[t]
                cols.append(col)
                comp.append(slack)
    Mst = np.array(cols).T if cols else np.zeros((len(rows_u), 0))
    comp = np.array(comp)
    w = np.array([w0[k, t] for k, t in rows_u])
    A = np.vstack([Mst, np.diag(comp)])
    rhs = np.concatenate([-w, np.zeros(len(comp))])
    mult, _ = nnls(A, rhs, maxiter=50 * max(A.shape[1], 1))
    res = w + Mst @ mult
    r_stat = np.abs(res).max() / den_stat if res.size else 0.0
    r_comp = np.abs(mult * comp).max() / den_comp if comp.size else 0.0
    return r_feas, r_stat, r_comp


def active_faces(inst: Instance, u: np.ndarray, tau: float = TAU_ACT):
    """uint64 [N]: bit (i*F + j) set iff face j of stance contact i is active,
    F = faces per contact; plus the per-face slack g/(1+n_max) for the
    ambiguity band.  Faces are ordered as ``contact_faces`` lists them."""
    N, cd = inst.N, inst.contact_dim
    F = len(contact_faces(cd, 0.5, 1.0)[1])
    bits = np.zeros(N, dtype=np.uint64)
    slack = np.full((N, inst.nc, F), -np.inf)
    for k in range(N):
        for i in range(inst.nc):
            if not inst.stance[k, i]:
                continue
            G, h = contact_faces(cd, inst.mu[k, i], inst.fmax[k, i])
            g = (G @ u[k, i * cd:(i + 1) * cd] - h) / (1.0 + inst.fmax[k, i])
            slack[k, i] = g
            for j in range(F):
                if g[j] >= -tau:
                    bits[k] |= np.uint64(1) << np.uint64(i * F + j)
    return bits, slack
