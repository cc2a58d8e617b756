"""The device's contact-set projection and active-face bits, through the C ABI.

A one-stage problem with B_0 = 0 and R_0 = r I has the Euclidean projection
of r^u onto the input set as its optimum (the state does not depend on u), so a
batch of one-stage instances -- one per golden case, the case's contact in
stance and the others in swing -- makes the solver's output u the device's
projection of each case's point.  The cases are the hand-derived ones
(tests/golden/projection_cases.txt) and those the oracle alone wrote
(tests/golden/projection_oracle_cases.txt, points at and near the apex, on
edges and beyond n_max).  With the polish off the returned u is z of the
ADMM iterate, i.e. the output of block 2's projection (point contacts:
project_point; wrenches: project_contact); with it on, the polish's exact
solve on the faces the projection read off.  The active-face bits of points
that lie on the set are compared with hand-derived bits
(tests/golden/active_faces.txt).

R_0 = 1e-4 I, the input weights of the workloads (the optimum does not
depend on the scale of R).  Tolerances: with the polish the faces are fixed
and the equality-constrained problem is solved exactly, so u is within
2e-5 (1 + max |expected|) of the projection (measured 2e-7).  Without it u
is the ADMM iterate at the certificate's stopping point; the problem is
strongly convex with modulus R_0, so a stationarity residual r moves u by
at most sqrt(nu) r / R_0, and r <= KKT (1 + max |R(u - r^u)|): the bar is
that bound from the reported KKT (about 0.06 N at KKT 2e-6).
"""
import os

import numpy as np
import pytest
import torch

from paper_2606_05687_b300 import workload as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
TOL = 2e-5


@pytest.fixture(scope="module")
def pinmpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc as P
    return P


def load_cases(name, cd):
    out = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, a, want = (part.split() for part in line.split("|"))
            if int(head[0]) != cd:
                continue
            out.append((float(head[1]), float(head[2]), 0, np.array(a, float), np.array(want, float)))
    return out


def load_face_cases(cd):
    out = []
    with open(os.path.join(GOLDEN, "active_faces.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, u, tail = (part.split() for part in line.split("|"))
            if int(head[0]) != cd or tail[1] != "1":
                continue
            out.append((float(head[1]), float(head[2]), int(head[3]), np.array(u, float), int(tail[0])))
    return out


def one_stage_batch(cd, cases):
    """One instance per case (mu, fmax, contact, point): N = 1, A = I, B = 0,
    R = I (callers rescale it), r^u = the point on the case's contact (the
    others in swing)."""
    nc = 2 if cd == 6 else 8
    nu, nx, B = cd * nc, 13, len(cases)
    spec = W.small_centroidal(B=B, N=1) if cd == 6 else W.rl_scale_walking(B=B, N=1)
    f32 = np.float32
    ru = np.zeros((B, 1, nu), f32)
    mu = np.full((B, 1, nc), 0.5, f32)
    fmax = np.full((B, 1, nc), 100.0, f32)
    mask = np.zeros((B, 1), np.uint32)
    for b, (m, fm, c, a, _) in enumerate(cases):
        ru[b, 0, c * cd:(c + 1) * cd] = a
        mu[b, 0, c] = m
        fmax[b, 0, c] = fm
        mask[b, 0] = 1 << c
    return W.Batch(spec=spec, A=np.tile(np.eye(nx, dtype=f32), (B, 1, 1, 1)), Bm=np.zeros((B, 1, nx, nu), f32),
                   e=np.zeros((B, 1, nx), f32), Q=np.ones((B, 1, nx), f32), R=np.ones((B, 1, nu), f32),
                   ry=np.zeros((B, 1, nx), f32), ru=ru, mu=mu, fmax=fmax, mask=mask,
                   xi0=np.zeros((B, nx), f32), u_prev=np.zeros((B, nu), f32),
                   horizon=np.ones(B, np.int32), nu_arr=np.full(B, nu, np.int32))


@pytest.mark.parametrize("cd", [3, 6])
@pytest.mark.parametrize("polish", [1, 0])
def test_device_projection_matches_golden_projections(pinmpc, cd, polish):
    cases = load_cases("projection_cases.txt", cd) + load_cases("projection_oracle_cases.txt", cd)
    batch = one_stage_batch(cd, cases)
    R0 = 1e-4
    batch.R = np.full_like(batch.R, R0)
    out = pinmpc.solve_workload(batch, polish=polish, max_iter=4000)
    assert np.all(out["status"] == pinmpc.CONVERGED), np.flatnonzero(out["status"])
    worst = 0.0
    for b, (_, _, c, a, want) in enumerate(cases):
        u = out["u"][b, 0].astype(np.float64)
        if polish:
            err = np.abs(u[c * cd:(c + 1) * cd] - want).max() / (1.0 + np.abs(want).max())
            assert err <= TOL, (b, cases[b], u[c * cd:(c + 1) * cd])
        else:
            den = 1.0 + R0 * np.abs(u[c * cd:(c + 1) * cd] - a).max()
            bound = np.sqrt(u.size) * float(out["kkt"][b]) * den / R0
            err = np.linalg.norm(u[c * cd:(c + 1) * cd] - want) / bound
            assert err <= 1.0, (b, cases[b], u[c * cd:(c + 1) * cd], bound)
        others = np.delete(u, np.arange(c * cd, (c + 1) * cd))
        assert np.all(others == 0.0)
        worst = max(worst, err)
    print(f"cd {cd} polish {polish}: {len(cases)} projections, worst {worst:.2e}, iters mean {out['iters'].mean():.1f}")


@pytest.mark.parametrize("cd", [3, 6])
def test_device_active_bits_match_hand_derived_bits(pinmpc, cd):
    cases = load_face_cases(cd)
    batch = one_stage_batch(cd, [(m, fm, c, u, None) for m, fm, c, u, _ in cases])
    out = pinmpc.solve_workload(batch)
    assert np.all(out["status"] == pinmpc.CONVERGED)
    for b, (_, _, _, _, want) in enumerate(cases):
        got = int(out["active_bits"][b, 0])
        assert got == want, (b, cases[b], bin(got), bin(want))
