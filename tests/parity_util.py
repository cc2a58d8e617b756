"""Shared helpers of the GPU parity tests: oracle references and comparisons."""
from __future__ import annotations

import numpy as np

from oracle import kkt as okkt
from oracle import qp

# Tolerances (FP32 solve against the FP64 oracle)
REL_TRAJ = 1e-4      # relative trajectory / control error
KKT_TOL = 1e-5       # KKT residual of the returned (xi, u), oracle checker
OBJ_GAP = 1e-6       # relative objective gap
TAU_ACT = okkt.TAU_ACT


def oracle_refs(batch, ids):
    """Oracle solutions (xi, u, objective) of the listed instances."""
    out = []
    for b in ids:
        sol = qp.solve_instance(qp.instance(batch, b))
        out.append((sol.xi, sol.u, sol.objective))
    return out


def compare(batch, out, ids, refs=None, check_bits=True):
    """Element-wise comparison of the GPU outputs of instances ``ids`` with
    the oracle; asserts the bars and returns the worst figures."""
    refs = refs if refs is not None else oracle_refs(batch, ids)
    worst = dict(eu=0.0, ex=0.0, kkt=0.0, gap=0.0, band=0)
    for b, (xi_r, u_r, obj_r) in zip(ids, refs):
        N = int(batch.horizon[b])
        inst = qp.instance(batch, b)
        u = out["u"][b, :N].astype(np.float64)
        xi = out["xi"][b, :N].astype(np.float64)
        su = max(np.abs(u_r).max(), 1e-9)
        sx = max(np.abs(xi_r).max(), 1e-9)
        eu = np.abs(u - u_r).max() / su
        ex = np.abs(xi - xi_r).max() / sx
        rep = okkt.kkt_residual(inst, xi, u)
        obj = qp.objective(inst, xi, u)
        gap = abs(obj - obj_r) / max(abs(obj_r), 1e-12)
        assert out["status"][b] == 0, f"instance {b}: status {out['status'][b]}"
        assert eu <= REL_TRAJ, f"instance {b}: control error {eu:.3e}"
        assert ex <= REL_TRAJ, f"instance {b}: state error {ex:.3e}"
        assert rep.kkt <= KKT_TOL, f"instance {b}: oracle-checked KKT {rep.kkt:.3e}"
        assert gap <= OBJ_GAP, f"instance {b}: objective gap {gap:.3e}"
        # the device certificate agrees with the oracle's checker
        assert abs(out["kkt"][b] - rep.kkt) <= 0.2 * rep.kkt + 5e-7, (b, out["kkt"][b], rep.kkt)
        if check_bits:
            ref_bits, slack = okkt.active_faces(inst, u_r)
            sl = -slack  # >= 0 for feasible faces
            F = slack.shape[2]
            band = (sl >= 0.1 * TAU_ACT) & (sl <= 10 * TAU_ACT)
            worst["band"] += int(band.sum())
            gb = out["active_bits"][b, :N]
            for k in range(N):
                for c in range(slack.shape[1]):
                    for f in range(F):
                        if not np.isfinite(slack[k, c, f]) or band[k, c, f]:
                            continue
                        bit = np.uint64(1) << np.uint64(c * F + f)
                        assert (gb[k] & bit) == (ref_bits[k] & bit), (b, k, c, f, slack[k, c, f])
        worst["eu"] = max(worst["eu"], eu)
        worst["ex"] = max(worst["ex"], ex)
        worst["kkt"] = max(worst["kkt"], rep.kkt)
        worst["gap"] = max(worst["gap"], gap)
    return worst


def dynamics_residual(batch, out):
    """max over instances/stages of the FP64 rollout residual of the outputs."""
    A = batch.A.astype(np.float64)
    Bm = batch.Bm.astype(np.float64)
    xi = out["xi"].astype(np.float64)
    u = out["u"].astype(np.float64)
    prev = np.concatenate([batch.xi0[:, None].astype(np.float64), xi[:, :-1]], 1)
    pred = np.einsum("bkij,bkj->bki", A, prev) + np.einsum("bkij,bkj->bki", Bm, u) + batch.e
    den = 1.0 + np.maximum(np.abs(pred).max(-1), np.abs(xi).max(-1))
    return float((np.abs(xi - pred).max(-1) / den).max())


def cone_violation(batch, out):
    """max normalised face violation on stance contacts and max |u| on swing contacts."""
    from oracle.project import cone
    cd = batch.contact_dim
    u = out["u"].astype(np.float64).reshape(batch.B, batch.N, batch.nc, cd)
    st = batch.stance()
    fmax = batch.fmax.astype(np.float64)
    mu = batch.mu.astype(np.float64)
    tang, coefs, nrm = cone(cd, mu)
    n = u[..., nrm]
    worst = np.maximum(-n, n - fmax)
    for t, coef in zip(tang, coefs):
        worst = np.maximum(worst, np.abs(u[..., t]) - coef * n)
    worst = np.where(st, worst / (1.0 + fmax), 0.0)
    swing = np.where(~st[..., None], np.abs(u), 0.0).max()
    return float(worst.max()), float(swing)
