"""Landmark guidance reward (Sec. II-C): the oracle against hand-derived
stage indices, the section's limiting cases and invariants; the library's
host-side index computation and argument checks (no device needed)."""
import ctypes
import math
import os

import numpy as np
import pytest

from oracle import landmarks as OL

HERE = os.path.dirname(os.path.abspath(__file__))


def golden_steps():
    rows = []
    with open(os.path.join(HERE, "golden", "landmark_steps.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            head, tail = line.split("|")
            N, nl = (int(x) for x in head.split())
            rows.append((N, nl, [int(x) for x in tail.split()]))
    return rows


@pytest.mark.parametrize("N,nl,want", golden_steps())
def test_oracle_steps_match_hand_derivation(N, nl, want):
    assert OL.landmark_steps(N, OL.uniform_s(nl)) == want


def test_planted_off_by_one_fails_the_golden_steps():
    # the same formula with floor(s N) in place of floor(s (N - 1)) must be caught
    wrong = lambda N, s: [1 + math.floor(x * N) for x in s]
    assert any(wrong(N, OL.uniform_s(nl)) != want for N, nl, want in golden_steps())


def test_first_and_last_landmark_are_next_step_and_horizon_end():
    for N in range(1, 33):
        n = OL.landmark_steps(N, OL.uniform_s(5))
        assert n[0] == 1 and n[-1] == N and n == sorted(n)


def _trajectories(rng, T, B, N, nx):
    return rng.normal(size=(T, B, N, nx))


def test_next_step_limit_and_average_limit():
    # Sec. II-C's remark: alpha = (1, 0, ...) is next-step supervision;
    # alpha_l = 1/N_L is time-averaged tracking
    rng = np.random.default_rng(5)
    T, B, N, nx = 12, 3, 8, 13
    xi = _trajectories(rng, T, B, N, nx)
    q = rng.normal(size=(T, B, 3))
    w = np.array([1.0, 2.0, 0.5])
    nxt = OL.LandmarkReward(N, OL.uniform_s(5), [1, 0, 0, 0, 0], w, 0.7, 0, 3)
    avg = OL.LandmarkReward(N, OL.uniform_s(5), [0.2] * 5, w, 0.7, 0, 3)
    n = OL.landmark_steps(N, OL.uniform_s(5))
    for t in range(T):
        r1, _, _ = nxt.reward(t, q[t])
        r2, _, c2 = avg.reward(t, q[t])
        for b in range(B):
            want1 = 1.0 if t < 1 else math.exp(-np.sum(w * (q[t, b] - xi[t - 1, b, 0, :3]) ** 2) / 0.49)
            terms = [np.sum(w * (q[t, b] - xi[t - nl, b, nl - 1, :3]) ** 2) for nl in n if t - nl >= 0]
            want2 = math.exp(-sum(terms) / 5 / 0.49)
            assert r1[b] == pytest.approx(want1, rel=1e-12) and r2[b] == pytest.approx(want2, rel=1e-12)
            assert c2[b] == len(terms)
        nxt.store(t, xi[t])
        avg.store(t, xi[t])


def test_reward_bounds_perfect_tracking_and_resets():
    rng = np.random.default_rng(6)
    N, B, nx = 6, 4, 13
    lr = OL.LandmarkReward(N, OL.uniform_s(5), OL.PAPER_ALPHA, np.ones(3), 1.0, 0, 3, ticks_per_stage=2)
    xi = rng.normal(size=(B, N, nx))
    r, e, c = lr.reward(0, rng.normal(size=(B, 3)))
    assert np.all(r == 1.0) and np.all(c == 0) and np.all(e == 0)  # nothing stored: all omitted
    lr.store(10, xi)
    n = lr.n
    for l, nl in enumerate(n):
        t = 10 + 2 * nl
        exact = xi[:, nl - 1, :3]
        r, e, c = lr.reward(t, exact)
        assert np.all(r == 1.0) and np.all(c == sum(1 for m in n if m == nl))
        r, _, _ = lr.reward(t, exact + 1.0)
        assert np.all((r > 0) & (r < 1))
    lr.reset(11, [1, 3])  # episodes of envs 1 and 3 begin after the store
    r, _, c = lr.reward(10 + 2 * n[-1], xi[:, n[-1] - 1, :3] + 1.0)
    assert c[1] == 0 and c[3] == 0 and r[1] == 1.0 and r[3] == 1.0 and c[0] > 0 and r[0] < 1


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import landmarks
    return landmarks


def test_library_steps_equal_oracle(L):
    rng = np.random.default_rng(7)
    for N in range(1, 33):
        for nl in range(1, 9):
            s = sorted(rng.uniform(0, 1, size=nl).astype(np.float32))
            s[0] = 0.0
            cfg = L.default_config(16, N, 13, n_landmarks=nl, s=s, alpha=[1.0] * nl)
            # the library takes s_l at its float32 value, as does this call
            assert L.steps(cfg) == OL.landmark_steps(N, [float(np.float32(x)) for x in s])
        assert L.steps(L.default_config(16, N, 13)) == OL.landmark_steps(N, OL.uniform_s(5))


def test_library_rejects_bad_configs_before_any_device_work(L):
    from paper_2606_05687_b300.pinmpc import MPC_ERR_INVALID_ARG, MpcError
    bad = [dict(q_dim=0), dict(q_index=12), dict(n_landmarks=9), dict(ticks_per_stage=0), dict(sigma=0.0),
           dict(s=[0.0, 0.5, 0.25, 0.75, 1.0]), dict(s=[0.0, 0.25, 0.5, 0.75, 1.5]), dict(alpha=[0.5, -1.0])]
    for kw in bad:
        with pytest.raises(MpcError) as ei:
            L.Landmarks(L.default_config(16, 20, 13, **kw))
        assert ei.value.code == MPC_ERR_INVALID_ARG, kw


def test_library_has_no_cpu_fallback(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2606_05687_b300.pinmpc import MPC_ERR_CUDA, MpcError
    with pytest.raises(MpcError) as ei:
        L.Landmarks(L.default_config(16, 20, 13))
    assert ei.value.code == MPC_ERR_CUDA


def test_config_layout_matches_header(tmp_path, L):
    import subprocess
    root = os.path.dirname(HERE)
    fields = [f[0] for f in L.LandmarkConfig._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pinmpc_landmarks.h"', "int main(void){",
             'printf("%zu\\n", sizeof(mpc_landmark_config));']
    lines += [f'printf("%zu\\n", offsetof(mpc_landmark_config, {f}));' for f in fields]
    lines += ["return 0;}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [ctypes.sizeof(L.LandmarkConfig)] + [getattr(L.LandmarkConfig, f).offset for f in fields]
