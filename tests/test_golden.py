"""Oracle against hand-derived projections (tests/golden/projection_cases.txt)."""
import os

import numpy as np
import pytest

from oracle import qp

HERE = os.path.dirname(os.path.abspath(__file__))


def load_cases():
    cases = []
    with open(os.path.join(HERE, "golden", "projection_cases.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, ru, want = (part.split() for part in line.split("|"))
            cases.append((int(head[0]), float(head[1]), float(head[2]),
                          np.array(ru, float), np.array(want, float)))
    return cases


def one_stage_projection_instance(cd, mu, fmax, ru):
    """N = 1, one stance contact (the others of the model in swing), B_0 = 0,
    R_0 = I: the optimum is the Euclidean projection of r^u."""
    nc = 2 if cd == 6 else 8
    nu = cd * nc
    nx = 13
    inst = qp.Instance(A=np.eye(nx)[None], Bm=np.zeros((1, nx, nu)), e=np.zeros((1, nx)),
                       Q=np.ones((1, nx)), R=np.ones((1, nu)), ry=np.zeros((1, nx)),
                       ru=np.zeros((1, nu)), mu=np.full((1, nc), mu),
                       fmax=np.full((1, nc), fmax), stance=np.zeros((1, nc), bool),
                       xi0=np.zeros(nx), contact_dim=cd)
    inst.stance[0, 0] = True
    inst.ru[0, :cd] = ru
    return inst


@pytest.mark.parametrize("case", load_cases())
def test_projection_golden(case):
    cd, mu, fmax, ru, want = case
    inst = one_stage_projection_instance(cd, mu, fmax, ru)
    sol = qp.solve_instance(inst)
    assert np.allclose(sol.u[0, :cd], want, rtol=0, atol=1e-10 * max(1.0, np.abs(want).max()))
    assert np.all(sol.u[0, cd:] == 0.0)
