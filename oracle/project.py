"""Contact sets and the exact Euclidean projection onto them (FP64).

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

Contact sets.  Sec. II-B names the friction pyramid and the contact wrench
cone.  Both are read as one generalized pyramid per stance contact,

    P = {(t, n): |t_j| <= c_j n for every tangential component j, 0 <= n <= n_max},

with the normal component n at index 2 of the contact's components:

  * 3-D point force (f_x, f_y, f_z): t = (f_x, f_y), c = (mu, mu);
  * 6-D foot wrench (f_x, f_y, f_z, tau_x, tau_y, tau_z):
    t = (f_x, f_y, tau_x, tau_y, tau_z),
    c = (mu, mu, d_y, d_x, mu min(d_x, d_y)), d_x / d_y the foot half length /
    half width (0.10 m / 0.05 m by default): friction on the tangential force,
    centre of pressure inside the foot, a yaw-torque bound -- a separable inner
    approximation of the wrench cone.

A swing contact's set is {0}.

Projection.  For a fixed n the nearest tangential components are
t_j = clip(a_j, -c_j n, c_j n), so the projection of a = (a_t, a_n) minimises the
one-dimensional convex function

    phi(n) = (n - a_n)^2 + sum_j max(|a_j| - c_j n, 0)^2

over [0, n_max].  phi is piecewise quadratic with breakpoints b_j = |a_j| / c_j;
on the piece where S = {j: b_j > n} it is minimised at

    n_S = (a_n + sum_{j in S} c_j |a_j|) / (1 + sum_{j in S} c_j^2).

The unconstrained minimiser of phi is the n_S of the piece that contains it, so
it is the candidate with the smallest phi; clamping a one-dimensional convex
minimiser to [0, n_max] gives the constrained one.  A component with c_j = 0 is
pinned to t_j = 0.  ``project_bruteforce`` is the independent check: it
enumerates subsets of the faces, projects onto each subset's affine hull and
keeps the nearest feasible point.
"""
from __future__ import annotations

import itertools

import numpy as np

FOOT_HALF_LENGTH = 0.10  # d_x
FOOT_HALF_WIDTH = 0.05   # d_y
NORMAL = 2               # index of the normal component within a contact


def cone(contact_dim: int, mu: float, dx: float = FOOT_HALF_LENGTH, dy: float = FOOT_HALF_WIDTH):
    """(tangential component indices, cone coefficients c_j, normal index)."""
    if contact_dim == 3:
        return [0, 1], [mu, mu], NORMAL
    if contact_dim == 6:
        return [0, 1, 3, 4, 5], [mu, mu, dy, dx, mu * min(dx, dy)], NORMAL
    raise ValueError("contact_dim must be 3 or 6")


def faces(contact_dim: int, mu: float, fmax: float, dx: float = FOOT_HALF_LENGTH,
          dy: float = FOOT_HALF_WIDTH):
    """Rows (G, h) of G x <= h describing P, in the order used for the
    active-face bits: for each tangential j, +t_j - c_j n <= 0 then
    -t_j - c_j n <= 0; then -n <= 0; then n <= n_max."""
    tang, coef, nrm = cone(contact_dim, mu, dx, dy)
    rows, rhs = [], []
    for j, c in zip(tang, coef):
        for sgn in (1.0, -1.0):
            g = np.zeros(contact_dim)
            g[j] = sgn
            g[nrm] = -c
            rows.append(g)
            rhs.append(0.0)
    g = np.zeros(contact_dim)
    g[nrm] = -1.0
    rows.append(g)
    rhs.append(0.0)
    g = np.zeros(contact_dim)
    g[nrm] = 1.0
    rows.append(g)
    rhs.append(fmax)
    return np.array(rows), np.array(rhs)


def project_many(a, contact_dim: int, mu, fmax, dx: float = FOOT_HALF_LENGTH,
                 dy: float = FOOT_HALF_WIDTH) -> np.ndarray:
    """Euclidean projections of the rows of a [M, contact_dim] onto the stance
    sets with friction coefficients mu [M] and force bounds fmax [M]."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, contact_dim)
    M = a.shape[0]
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (M,))
    fmax = np.broadcast_to(np.asarray(fmax, dtype=np.float64), (M,))
    tang, coefs, nrm = cone(contact_dim, mu, dx, dy)
    C = np.stack([np.broadcast_to(np.asarray(c, dtype=np.float64), (M,)) for c in coefs], axis=1)
    an = a[:, nrm]
    at = np.abs(a[:, tang])
    live = C > 0.0
    brk = np.where(live, at / np.where(live, C, 1.0), np.inf)
    order = np.argsort(brk, axis=1, kind="stable")
    Cs = np.take_along_axis(np.where(live, C, 0.0), order, axis=1)
    As = np.take_along_axis(at, order, axis=1)
    m = len(tang)
    # piece p (p = 0..m): S = the components at sorted positions p..m-1, whose
    # breakpoints lie above the piece; suffix sums give every piece's n_S
    num = np.zeros((M, m + 1))
    den = np.ones((M, m + 1))
    for p in range(m):
        num[:, p] = np.sum(Cs[:, p:] * As[:, p:], axis=1)
        den[:, p] = 1.0 + np.sum(Cs[:, p:] ** 2, axis=1)
    cand = (an[:, None] + num) / den
    phi = (cand - an[:, None]) ** 2 + np.sum(
        np.maximum(at[:, None, :] - C[:, None, :] * cand[:, :, None], 0.0) ** 2, axis=2)
    n = cand[np.arange(M), np.argmin(phi, axis=1)]
    n = np.minimum(np.maximum(n, 0.0), fmax)
    out = a.copy()
    out[:, nrm] = n
    lim = C * n[:, None]
    out[:, tang] = np.minimum(np.maximum(a[:, tang], -lim), lim)
    return out


def project(a, contact_dim: int, mu: float, fmax: float, dx: float = FOOT_HALF_LENGTH,
            dy: float = FOOT_HALF_WIDTH) -> np.ndarray:
    """Euclidean projection of one contact's components a onto P (stance)."""
    return project_many(np.asarray(a)[None], contact_dim, [mu], [fmax], dx, dy)[0]


def project_input(u, stance, mu, fmax, contact_dim: int, dx: float = FOOT_HALF_LENGTH,
                  dy: float = FOOT_HALF_WIDTH) -> np.ndarray:
    """Projection of input vectors u [..., nc * contact_dim] onto U_k = prod_i P_i
    (stance [..., nc] selects P_i, a swing contact's set is {0})."""
    u = np.asarray(u, dtype=np.float64)
    nc = np.shape(stance)[-1]
    a = u.reshape(-1, nc, contact_dim)
    st = np.asarray(stance, bool).reshape(-1, nc)
    out = np.zeros_like(a)
    sel = st.reshape(-1)
    flat = a.reshape(-1, contact_dim)
    res = out.reshape(-1, contact_dim)
    res[sel] = project_many(flat[sel], contact_dim, np.asarray(mu).reshape(-1)[sel],
                            np.asarray(fmax).reshape(-1)[sel], dx, dy)
    return res.reshape(u.shape)


def project_bruteforce(a, contact_dim: int, mu: float, fmax: float, max_faces: int = None,
                       dx: float = FOOT_HALF_LENGTH, dy: float = FOOT_HALF_WIDTH) -> np.ndarray:
    """Projections of the rows of a [M, contact_dim] onto one stance set P (one
    mu, one n_max) by enumeration: for every subset S of at most ``max_faces``
    faces (default: the dimension), the projection onto the affine hull
    {x: G_S x = h_S} (a pseudo-inverse for dependent rows), keeping for each
    row the nearest point that satisfies every face."""
    a = np.atleast_2d(np.asarray(a, dtype=np.float64))
    G, h = faces(contact_dim, mu, fmax, dx, dy)
    m = G.shape[0]
    kmax = contact_dim if max_faces is None else max_faces
    tol = 1e-12 * (1.0 + np.abs(a).max(axis=1) + fmax)
    best = np.full_like(a, np.nan)
    best_d = np.full(a.shape[0], np.inf)
    for k in range(kmax + 1):
        for S in itertools.combinations(range(m), k):
            if k:
                GS, hS = G[list(S)], h[list(S)]
                P = GS.T @ np.linalg.pinv(GS @ GS.T)
                x = a - (a @ GS.T - hS) @ P.T
                ok = np.abs(x @ GS.T - hS).max(axis=1) <= tol  # consistent subset
            else:
                x = a
                ok = np.ones(a.shape[0], bool)
            ok &= (x @ G.T - h).max(axis=1) <= tol
            d = np.sum((x - a) ** 2, axis=1)
            take = ok & (d < best_d)
            best[take] = x[take]
            best_d[take] = d[take]
    return best
