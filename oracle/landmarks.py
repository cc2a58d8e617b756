"""Landmark guidance reward (Sec. II-C), FP64.  Test infrastructure only.

Written from the section's definitions, with plain Python containers:

    delta_l = n_l dt,  n_l = 1 + floor(s_l (N - 1)),  l = 0 .. N_L - 1;
    a solve at time t stores (t + delta_l, q^t(delta_l)) for every l, where
    q^t(delta_l) is the guided quantity (the CoM c in the paper) of the
    predicted state delta_l ahead, i.e. of the state at stage n_l;
    at time t, e_l(t) = q_t - q^{t - delta_l}(delta_l) for every l whose
    landmark exists (landmarks from before the current episode do not), and
    r_t = exp( - sum_l alpha_l ||e_l(t)||^2_Q / sigma^2 ).

Time is an integer tick; one MPC stage (dt) spans `ticks_per_stage` ticks.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

PAPER_ALPHA = (0.5, 0.25, 0.15, 0.07, 0.03)  # Sec. II-C, the experiments' schedule


def landmark_steps(N: int, s: Sequence[float]) -> List[int]:
    """n_l = 1 + floor(s_l (N - 1)) for each s_l (taken at its given value)."""
    return [1 + math.floor(float(sl) * (N - 1)) for sl in s]


def uniform_s(n_landmarks: int) -> List[float]:
    """s_l = l / (N_L - 1): s_0 = 0 (the next MPC step) and s_{N_L-1} = 1 (the horizon end)."""
    if n_landmarks == 1:
        return [0.0]
    return [l / (n_landmarks - 1) for l in range(n_landmarks)]


class LandmarkReward:
    """Per-environment record of stored landmarks and the reward of Sec. II-C."""

    def __init__(self, N: int, s: Sequence[float], alpha: Sequence[float], q_weight: Sequence[float],
                 sigma: float, q_index: int, q_dim: int, ticks_per_stage: int = 1):
        self.n = landmark_steps(N, s)
        self.alpha = [float(a) for a in alpha]
        self.w = np.asarray(q_weight, dtype=np.float64)[:q_dim]
        self.sigma = float(sigma)
        self.q_index, self.q_dim, self.tps = q_index, q_dim, ticks_per_stage
        # (env, l, maturity tick) -> (tick of the solve, predicted quantity)
        self.stored: Dict[Tuple[int, int, int], Tuple[int, np.ndarray]] = {}
        self.episode_start: Dict[int, int] = {}

    def store(self, tick: int, xi: np.ndarray):
        """xi [B][N][nx]: row k is the predicted state at stage k + 1."""
        for b in range(xi.shape[0]):
            for l, n in enumerate(self.n):
                q = np.asarray(xi[b, n - 1, self.q_index:self.q_index + self.q_dim], dtype=np.float64)
                self.stored[(b, l, tick + n * self.tps)] = (tick, q)

    def reset(self, tick: int, envs):
        for b in envs:
            self.episode_start[int(b)] = tick

    def reward(self, tick: int, q_now: np.ndarray):
        """(reward [B], e [B][N_L][q_dim] with zeros where unavailable, count [B])."""
        B = q_now.shape[0]
        r = np.zeros(B)
        e = np.zeros((B, len(self.n), self.q_dim))
        cnt = np.zeros(B, dtype=np.int64)
        for b in range(B):
            total = 0.0
            for l in range(len(self.n)):
                entry = self.stored.get((b, l, tick))
                if entry is None:
                    continue
                solved_at, q_pred = entry
                if solved_at < self.episode_start.get(b, -math.inf):
                    continue  # predicted in an earlier episode
                err = np.asarray(q_now[b], dtype=np.float64) - q_pred
                e[b, l] = err
                total += self.alpha[l] * float(np.sum(self.w * err * err))
                cnt[b] += 1
            r[b] = math.exp(-total / self.sigma ** 2)
        return r, e, cnt
