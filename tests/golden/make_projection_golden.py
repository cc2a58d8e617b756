"""Writes projection_oracle_cases.txt: projections onto one contact's set
computed by the FP64 oracle (oracle.project) alone, for the GPU tests.

    python tests/golden/make_projection_golden.py

Seeded; the points mix random draws with points at and near the apex, on
edges and faces, and beyond n_max, for both contact models.  The CPU tests
check that the oracle still reproduces the file and that it agrees with a
face-subset brute force on every row.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import project as P  # noqa: E402

OUT = os.path.join(HERE, "projection_oracle_cases.txt")


def points(rng, cd, mu, fmax, n):
    """n points around one contact's set: random, near the apex, near edges
    (some faces tight, a small offset), and beyond n_max."""
    tang, coef, nrm = P.cone(cd, mu)
    out = []
    for i in range(n):
        kind = i % 4
        a = np.zeros(cd)
        if kind == 0:
            a = rng.normal(size=cd) * 0.6 * fmax
        elif kind == 1:
            a = rng.normal(size=cd) * 1e-3 * fmax
        elif kind == 2:
            nn = rng.uniform(0.1, 0.9) * fmax
            a[nrm] = nn
            for j, c in zip(tang, coef):
                a[j] = rng.choice([-1.0, 1.0]) * c * nn * rng.choice([1.0, rng.uniform(0.0, 1.0)])
            a += rng.normal(size=cd) * 1e-2 * fmax
        else:
            a = rng.normal(size=cd) * 0.4 * fmax
            a[nrm] = rng.uniform(1.0, 2.0) * fmax
        out.append(a)
    return out


def main():
    rng = np.random.default_rng(20260613)
    lines = ["# Projections onto one stance contact's generalized pyramid computed by the",
             "# FP64 oracle (oracle.project) alone; written by make_projection_golden.py.",
             "# dim mu n_max | point | projection"]
    for cd in (3, 6):
        for mu, fmax in ((0.5, 375.0), (0.9, 1500.0), (0.6, 200.0)):
            for a in points(rng, cd, mu, fmax, 24):
                x = P.project(a, cd, mu, fmax)
                lines.append(f"{cd} {mu!r} {fmax!r} | " + " ".join(repr(float(v)) for v in a) + " | "
                             + " ".join(repr(float(v)) for v in x))
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
