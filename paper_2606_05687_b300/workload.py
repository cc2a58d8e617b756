"""Seeded synthetic centroidal-MPC workloads (inputs only; no solver arithmetic).

This module builds the per-stage data of the linear time-varying MPC problem
stated in Sec. III (the standard form below Eq. (cd_ltv_mpc)):

    min  sum_k 1/2 ||xi_{k+1} - r^y_k||^2_{Q_k} + 1/2 ||u_k - r^u_k||^2_{R_k}
    s.t. xi_{k+1} = A_k xi_k + B_k u_k + e_k,  u_k in U_k

for a batch of independent environments.  It is the single input generator
shared by the CPU oracle, the tests and the benchmark; it holds none of the
solver's arithmetic.

Model (a stand-in for the paper's RL workload, whose simulator is not
available): the 13-state convex centroidal model
x = [p(3), Theta(3) roll/pitch/yaw, v(3), omega(3), g(1)], forward-Euler
discretised with step dt (Sec. II-A uses the same Euler form), so
A_k = I + dt*A_c(psi_k), B_k = dt*B_c(k), e_k = 0 (+ an optional small
linearisation offset used by tests).  The gravity state x_13 = 9.81 is
constant (its A row is a unit row and its B row is zero).

A second model (spec.model = "cd9") is the paper's own 9-state centroidal
model xi = [c, l_G, k_G] of Sec. II-A, linearised about a nominal CoM path
and gravity-compensating forces (see _centroidal9); contact sets, schedules,
input costs and draws are shared with the 13-state model.

Every random number of instance b is drawn from its own generator seeded by
(seed, b), so any subset of a batch can be regenerated without the rest.
All returned arrays are float32 (the values both solvers consume; the oracle
promotes them to float64) except the integer masks and horizons.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

NX = 13
GRAVITY = 9.81
MASS = 60.0
INERTIA_BODY = (2.5, 2.2, 0.6)
COM_HEIGHT = 0.9
FOOT_HALF_LENGTH = 0.10  # d_x, contact-set coefficient for the 6-D wrench cone
FOOT_HALF_WIDTH = 0.05   # d_y


@dataclasses.dataclass(frozen=True)
class WorkloadSpec:
    """Shape and distribution of one synthetic batch."""

    B: int
    N: int
    contact_dim: int          # 3 = point force, 6 = foot wrench
    n_contacts: int           # contacts per stage (nu = n_contacts*contact_dim)
    dt: float = 0.02
    seed: int = 0
    schedule: str = "bernoulli"   # "bernoulli" | "walking" | "all_stance" | "all_swing"
    f_max: float = 1500.0         # normal-force bound per contact
    e_scale: float = 0.0          # std of an optional linearisation offset e_k
    u_prev_scale: float = 0.0     # std of u_{-1} (the velocity-form initial input)
    ref_noise: float = 0.1        # std of the reference / initial-state noise
    model: str = "srb13"          # "srb13": 13-state convex model; "cd9": the 9-state centroidal model
    horizon_min: int = 0          # > 0: per-instance horizons uniform in horizon_min .. N (stage stride N)

    @property
    def nu(self) -> int:
        return self.n_contacts * self.contact_dim


def small_centroidal(B: int = 64, N: int = 10, seed: int = 1001, **kw) -> WorkloadSpec:
    """Two feet with 6-D wrenches (nu=12), Bernoulli(0.7) stance, f_max 1500 N."""
    return WorkloadSpec(B=B, N=N, contact_dim=6, n_contacts=2, seed=seed,
                        schedule=kw.pop("schedule", "bernoulli"),
                        f_max=kw.pop("f_max", 1500.0), **kw)


def rl_scale_walking(B: int = 4096, N: int = 20, seed: int = 1002, **kw) -> WorkloadSpec:
    """Eight 3-D contact points (4 corners per foot, nu=24), walking gait,
    1500 N per foot split over its 4 points (375 N each)."""
    return WorkloadSpec(B=B, N=N, contact_dim=3, n_contacts=8, seed=seed,
                        schedule=kw.pop("schedule", "walking"),
                        f_max=kw.pop("f_max", 375.0), **kw)


def uneven_mixed(B: int = 16384, N: int = 40, seed: int = 1003, **kw) -> list:
    """Uneven batching: half the environments with eight 3-D contact points and
    a walking gait, half with two 6-D foot wrenches and Bernoulli stance;
    horizons uniform in 5 .. N per environment (stage stride N).  Two specs,
    one per contact model (each model is its own solver shape)."""
    n1 = B // 2
    return [rl_scale_walking(B=n1, N=N, seed=seed, horizon_min=5, **kw),
            small_centroidal(B=B - n1, N=N, seed=seed + 1, horizon_min=5, **kw)]


def centroidal9_walking(B: int = 4096, N: int = 20, seed: int = 1004, **kw) -> WorkloadSpec:
    """The walking workload on the 9-state centroidal model of Sec. II-A
    (eight 3-D contact points, nu = 24)."""
    return rl_scale_walking(B=B, N=N, seed=seed, model="cd9", **kw)


def centroidal9_small(B: int = 64, N: int = 10, seed: int = 1005, **kw) -> WorkloadSpec:
    """Two feet with 6-D wrenches on the 9-state centroidal model."""
    return small_centroidal(B=B, N=N, seed=seed, model="cd9", **kw)


@dataclasses.dataclass
class Batch:
    """One batch of stage data, instance-major, float32 unless noted.

    A [B,N,nx,nx]; Bm [B,N,nx,nu]; e [B,N,nx]; Q [B,N,nx] (diagonal);
    R [B,N,nu] (diagonal); ry [B,N,nx]; ru [B,N,nu]; mu [B,N,nc];
    fmax [B,N,nc]; mask uint32 [B,N] (bit c = contact c in stance);
    xi0 [B,nx]; u_prev [B,nu]; horizon int32 [B]; nu int32 [B].
    """

    spec: WorkloadSpec
    A: np.ndarray
    Bm: np.ndarray
    e: np.ndarray
    Q: np.ndarray
    R: np.ndarray
    ry: np.ndarray
    ru: np.ndarray
    mu: np.ndarray
    fmax: np.ndarray
    mask: np.ndarray
    xi0: np.ndarray
    u_prev: np.ndarray
    horizon: np.ndarray
    nu_arr: np.ndarray

    @property
    def B(self) -> int:
        return self.A.shape[0]

    @property
    def N(self) -> int:
        return self.A.shape[1]

    @property
    def nx(self) -> int:
        return self.A.shape[2]

    @property
    def nu(self) -> int:
        return self.Bm.shape[3]

    @property
    def nc(self) -> int:
        return self.mu.shape[2]

    @property
    def contact_dim(self) -> int:
        return self.spec.contact_dim

    def subset(self, idx: Sequence[int]) -> "Batch":
        idx = np.asarray(idx)
        kw = {f.name: getattr(self, f.name)[idx] for f in dataclasses.fields(self)
              if f.name != "spec"}
        return Batch(spec=dataclasses.replace(self.spec, B=len(idx)), **kw)

    def receding(self, xi0: np.ndarray, u_prev: np.ndarray) -> "Batch":
        """The next MPC step of a receding horizon: every stage array moves one
        stage towards the start (the last stage repeated), with the given
        initial state and previous input (float32 [B,nx], [B,nu])."""
        kw = {}
        for f in dataclasses.fields(self):
            v = getattr(self, f.name)
            if f.name in ("spec", "xi0", "u_prev", "horizon", "nu_arr"):
                kw[f.name] = v
            else:
                kw[f.name] = np.concatenate([v[:, 1:], v[:, -1:]], axis=1)
        kw["xi0"] = np.ascontiguousarray(xi0, dtype=np.float32)
        kw["u_prev"] = np.ascontiguousarray(u_prev, dtype=np.float32)
        return Batch(**kw)

    def stance(self) -> np.ndarray:
        """bool [B,N,nc]: contact c of stage k is in stance."""
        bits = (self.mask[..., None] >> np.arange(self.nc, dtype=np.uint32)) & 1
        return bits.astype(bool)


def _rot_z(psi):
    c, s = np.cos(psi), np.sin(psi)
    z, o = np.zeros_like(psi), np.ones_like(psi)
    return np.stack([np.stack([c, -s, z], -1), np.stack([s, c, z], -1),
                     np.stack([z, z, o], -1)], -2)


def _rot_y(a):
    c, s = np.cos(a), np.sin(a)
    z, o = np.zeros_like(a), np.ones_like(a)
    return np.stack([np.stack([c, z, s], -1), np.stack([z, o, z], -1),
                     np.stack([-s, z, c], -1)], -2)


def _rot_x(a):
    c, s = np.cos(a), np.sin(a)
    z, o = np.zeros_like(a), np.ones_like(a)
    return np.stack([np.stack([o, z, z], -1), np.stack([z, c, -s], -1),
                     np.stack([z, s, c], -1)], -2)


def _skew(r):
    x, y, z = r[..., 0], r[..., 1], r[..., 2]
    zero = np.zeros_like(x)
    return np.stack([np.stack([zero, -z, y], -1), np.stack([z, zero, -x], -1),
                     np.stack([-y, x, zero], -1)], -2)


def _draw_instance(spec: WorkloadSpec, b: int) -> dict:
    """All random numbers of instance b, in a fixed order."""
    rng = np.random.default_rng([spec.seed, b])
    N, nu = spec.N, spec.nu
    d = {}
    d["psi0"] = rng.uniform(-math.pi, math.pi)
    d["psi_rate"] = rng.uniform(-1.0, 1.0)
    d["roll_pitch"] = rng.uniform(-0.1, 0.1, size=(N, 2))
    d["foot_off"] = rng.uniform(-0.15, 0.15, size=(N, 2, 2))
    d["Q"] = rng.uniform(1.0, 100.0, size=NX)
    d["R"] = rng.uniform(1e-4, 1e-3, size=nu)
    d["ry_noise"] = rng.normal(0.0, 1.0, size=(N, 12))
    d["xi0_noise"] = rng.normal(0.0, 1.0, size=12)
    d["mu_foot"] = rng.uniform(0.5, 0.9, size=2)
    d["stance_u"] = rng.uniform(0.0, 1.0, size=(N, 2))
    d["period"] = rng.uniform(0.4, 0.8)
    d["phase"] = rng.uniform(0.0, 1.0)
    d["e_noise"] = rng.normal(0.0, 1.0, size=(N, NX))
    d["u_prev_noise"] = rng.normal(0.0, 1.0, size=nu)
    # drawn last, so the draws above do not depend on it
    d["horizon"] = int(rng.integers(spec.horizon_min, N + 1)) if spec.horizon_min > 0 else N
    return d


def generate(spec: WorkloadSpec, instances: Optional[Sequence[int]] = None) -> Batch:
    """Build the batch (or the listed instances of it) described by ``spec``."""
    ids = np.arange(spec.B) if instances is None else np.asarray(instances)
    nb, N, nu, dt = len(ids), spec.N, spec.nu, spec.dt
    if spec.contact_dim not in (3, 6):
        raise ValueError("contact_dim must be 3 or 6")
    if spec.contact_dim == 6 and spec.n_contacts != 2:
        raise ValueError("the wrench model has one contact per foot (2)")
    if spec.contact_dim == 3 and spec.n_contacts != 8:
        raise ValueError("the point-force model has 4 corner points per foot (8)")
    draws = [_draw_instance(spec, int(b)) for b in ids]
    stack = lambda key: np.stack([np.asarray(d[key], dtype=np.float64) for d in draws])

    k = np.arange(N, dtype=np.float64)
    psi = stack("psi0")[:, None] + stack("psi_rate")[:, None] * k[None, :] * dt  # [nb,N]
    rp = stack("roll_pitch")
    Rz = _rot_z(psi)
    Rot = Rz @ _rot_y(rp[..., 1]) @ _rot_x(rp[..., 0])                  # [nb,N,3,3]
    Iinv_w = Rot @ np.diag(1.0 / np.asarray(INERTIA_BODY)) @ np.swapaxes(Rot, -1, -2)

    Ac = np.zeros((nb, N, NX, NX))
    Ac[..., 0:3, 6:9] = np.eye(3)
    Ac[..., 3:6, 9:12] = np.swapaxes(Rz, -1, -2)
    Ac[..., 8, 12] = -1.0
    A = np.eye(NX) + dt * Ac

    # contact positions relative to the CoM, world frame
    off = stack("foot_off")                                               # [nb,N,2,2]
    lateral = np.array([0.1, -0.1])
    foot_local = np.zeros((nb, N, 2, 3))
    foot_local[..., 0] = off[..., 0]
    foot_local[..., 1] = lateral + off[..., 1]
    foot_local[..., 2] = -COM_HEIGHT
    Bc = np.zeros((nb, N, NX, nu))
    if spec.contact_dim == 6:
        pos = np.einsum("bkij,bkfj->bkfi", Rz, foot_local)               # [nb,N,2,3]
        for f in range(2):
            c0 = 6 * f
            Bc[..., 6:9, c0:c0 + 3] = np.eye(3) / MASS
            Bc[..., 9:12, c0:c0 + 3] = Iinv_w @ _skew(pos[:, :, f])
            Bc[..., 9:12, c0 + 3:c0 + 6] = Iinv_w
    else:
        corners = np.array([[1, 1], [1, -1], [-1, 1], [-1, -1]], dtype=np.float64)
        corners = corners * np.array([FOOT_HALF_LENGTH, FOOT_HALF_WIDTH])
        for f in range(2):
            for c in range(4):
                loc = foot_local[:, :, f].copy()
                loc[..., 0] += corners[c, 0]
                loc[..., 1] += corners[c, 1]
                pos = np.einsum("bkij,bkj->bki", Rz, loc)
                c0 = 3 * (4 * f + c)
                Bc[..., 6:9, c0:c0 + 3] = np.eye(3) / MASS
                Bc[..., 9:12, c0:c0 + 3] = Iinv_w @ _skew(pos)
    Bm = dt * Bc

    e = np.zeros((nb, N, NX))
    if spec.e_scale:
        e[..., 0:12] = spec.e_scale * stack("e_noise")[..., 0:12]

    Q = np.repeat(stack("Q")[:, None, :], N, axis=1)
    R = np.repeat(stack("R")[:, None, :], N, axis=1)
    nominal = np.zeros(NX)
    nominal[2] = COM_HEIGHT
    nominal[12] = GRAVITY
    ry = np.broadcast_to(nominal, (nb, N, NX)).copy()
    ry[..., 0:12] += spec.ref_noise * stack("ry_noise")
    xi0 = np.broadcast_to(nominal, (nb, NX)).copy()
    xi0[:, 0:12] += spec.ref_noise * stack("xi0_noise")
    ru = np.zeros((nb, N, nu))
    u_prev = spec.u_prev_scale * stack("u_prev_noise")

    per_foot = spec.n_contacts // 2
    mu = np.repeat(stack("mu_foot"), per_foot, axis=1)                    # [nb,nc]
    mu = np.repeat(mu[:, None, :], N, axis=1)
    fmax = np.full((nb, N, spec.n_contacts), spec.f_max)

    if spec.schedule == "bernoulli":
        foot_stance = stack("stance_u") < 0.7                              # [nb,N,2]
    elif spec.schedule == "walking":
        t = k[None, :] * dt / stack("period")[:, None]
        ph = stack("phase")[:, None] + t
        left = np.mod(ph, 1.0) < 0.6
        right = np.mod(ph + 0.5, 1.0) < 0.6
        foot_stance = np.stack([left, right], -1)
    elif spec.schedule == "all_stance":
        foot_stance = np.ones((nb, N, 2), dtype=bool)
    elif spec.schedule == "all_swing":
        foot_stance = np.zeros((nb, N, 2), dtype=bool)
    else:
        raise ValueError(f"unknown schedule {spec.schedule!r}")
    contact_stance = np.repeat(foot_stance, per_foot, axis=2)             # [nb,N,nc]
    mask = (contact_stance.astype(np.uint32)
            << np.arange(spec.n_contacts, dtype=np.uint32)).sum(-1).astype(np.uint32)

    nominal = None
    if spec.model == "cd9":
        A, Bm, e, Q, ry, xi0, nominal = _centroidal9(spec, stack, psi, contact_stance, nb, N, dt)
    elif spec.model != "srb13":
        raise ValueError(f"unknown model {spec.model!r}")

    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
    out = Batch(spec=dataclasses.replace(spec, B=nb), A=f32(A), Bm=f32(Bm), e=f32(e),
                Q=f32(Q), R=f32(R), ry=f32(ry), ru=f32(ru), mu=f32(mu), fmax=f32(fmax),
                mask=mask, xi0=f32(xi0), u_prev=f32(u_prev),
                horizon=np.asarray([d["horizon"] for d in draws], dtype=np.int32),
                nu_arr=np.full(nb, nu, dtype=np.int32))
    if nominal is not None:
        out.nominal = nominal  # linearisation point of the cd9 model (float64), for checks
    return out


NX9 = 9


def _centroidal9(spec, stack, psi, contact_stance, nb, N, dt):
    """Stage data of the 9-state centroidal model xi = [c, l_G, k_G] (Sec. II-A):
        c+   = c + dt l_G / m
        l_G+ = l_G + dt (m g + sum_i f_i)
        k_G+ = k_G + dt sum_i ((p_i - c) x f_i + tau_i)
    linearised for the LTV standard form at the nominal CoM cbar_k (moving at
    the commanded velocity) and nominal forces fbar_i (gravity compensation
    shared evenly by the stance contacts):
        (p_i - c) x f_i ~ [p_i - cbar]x f_i + [fbar_i]x (c - cbar),
    exact when c = cbar, with error (cbar - c) x (f_i - fbar_i) otherwise.
    Stage cost (Sec. II-B): CoM tracking on c, velocity tracking on
    v = l_G / m (a weight Q_v / m^2 on l_G), angular-momentum regulation on
    k_G (weights 1e-4 .. 1e-2); diagonal Q.  Inputs, contact sets, schedules and R are the 13-state
    workload's."""
    cd, nc = spec.contact_dim, spec.n_contacts
    nu = nc * cd
    k = np.arange(N + 1, dtype=np.float64)
    psi0 = stack("psi0")
    vcmd = 0.5 * np.stack([np.cos(psi0), np.sin(psi0), np.zeros_like(psi0)], -1)      # [nb,3]
    cbar = np.zeros((nb, N + 1, 3))
    cbar[..., 2] = COM_HEIGHT
    cbar += k[None, :, None] * dt * vcmd[:, None, :]
    # contact positions relative to the nominal CoM (world frame): the 13-state
    # model's foot placement
    off = stack("foot_off")                                                          # [nb,N,2,2]
    lateral = np.array([0.1, -0.1])
    Rz = _rot_z(psi)
    lever = np.zeros((nb, N, nc, 3))
    if cd == 6:
        for f in range(2):
            loc = np.zeros((nb, N, 3))
            loc[..., 0] = off[..., f, 0]
            loc[..., 1] = lateral[f] + off[..., f, 1]
            loc[..., 2] = -COM_HEIGHT
            lever[:, :, f] = np.einsum("bkij,bkj->bki", Rz, loc)
    else:
        corners = np.array([[1, 1], [1, -1], [-1, 1], [-1, -1]], dtype=np.float64)
        corners = corners * np.array([FOOT_HALF_LENGTH, FOOT_HALF_WIDTH])
        for f in range(2):
            for c in range(4):
                loc = np.zeros((nb, N, 3))
                loc[..., 0] = off[..., f, 0] + corners[c, 0]
                loc[..., 1] = lateral[f] + off[..., f, 1] + corners[c, 1]
                loc[..., 2] = -COM_HEIGHT
                lever[:, :, 4 * f + c] = np.einsum("bkij,bkj->bki", Rz, loc)
    n_st = contact_stance.sum(-1)                                                    # [nb,N]
    Fbar = np.zeros((nb, N, 3))
    Fbar[..., 2] = np.where(n_st > 0, MASS * GRAVITY, 0.0)                          # sum of fbar_i

    A = np.zeros((nb, N, NX9, NX9))
    A[...] = np.eye(NX9)
    A[..., 0:3, 3:6] = dt / MASS * np.eye(3)
    A[..., 6:9, 0:3] = dt * _skew(Fbar)
    Bm = np.zeros((nb, N, NX9, nu))
    for i in range(nc):
        c0 = i * cd
        Bm[..., 3:6, c0:c0 + 3] = dt * np.eye(3)
        Bm[..., 6:9, c0:c0 + 3] = dt * _skew(lever[:, :, i])
        if cd == 6:
            Bm[..., 6:9, c0 + 3:c0 + 6] = dt * np.eye(3)
    e = np.zeros((nb, N, NX9))
    e[..., 5] = -dt * MASS * GRAVITY
    e[..., 6:9] = -dt * np.einsum("bkij,bkj->bki", _skew(Fbar), cbar[:, :N])
    if spec.e_scale:
        e += spec.e_scale * stack("e_noise")[..., 0:NX9]

    q = stack("Q")[:, 0:NX9].copy()
    q[:, 3:6] /= MASS ** 2
    # angular momentum is regularised, not tracked hard: with weights of the
    # order of the CoM weights the gravity torque about an offset CoM in
    # single support drives the contact forces to their bounds
    q[:, 6:9] *= 1e-4
    Q = np.repeat(q[:, None, :], N, axis=1)
    rn = stack("ry_noise")[..., 0:NX9]                                               # [nb,N,9]
    ry = np.zeros((nb, N, NX9))
    ry[..., 0:3] = cbar[:, 1:] + spec.ref_noise * rn[..., 0:3]
    ry[..., 3:6] = MASS * (vcmd[:, None, :] + spec.ref_noise * rn[..., 3:6])
    ry[..., 6:9] = spec.ref_noise * rn[..., 6:9]
    x0n = stack("xi0_noise")[:, 0:NX9]
    xi0 = np.zeros((nb, NX9))
    xi0[:, 0:3] = cbar[:, 0] + spec.ref_noise * x0n[:, 0:3]
    xi0[:, 3:6] = MASS * (vcmd + spec.ref_noise * x0n[:, 3:6])
    xi0[:, 6:9] = spec.ref_noise * x0n[:, 6:9]
    nominal = {"cbar": cbar, "lever": lever, "fbar_sum": Fbar}
    return A, Bm, e, Q, ry, xi0, nominal
