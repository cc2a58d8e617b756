"""Landmark epilogue on the GPU against the FP64 oracle (Sec. II-C): seeded
synthetic predicted trajectories stored every other tick with two ticks per
stage, the reward at every tick, episode resets mid-way, a ragged batch; and
storing straight from a solver handle equals storing its copied-out
trajectory."""
import numpy as np
import pytest

from oracle import landmarks as OL
from paper_2606_05687_b300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import landmarks, pinmpc
    return torch, landmarks, pinmpc


def test_reward_matches_oracle_over_ticks_with_resets(env):
    torch, L, _ = env
    rng = np.random.default_rng(2024)
    B_max, B, N, nx, tps, T = 64, 37, 20, 13, 2, 90
    w = rng.uniform(0.5, 2.0, size=3)
    cfg = L.default_config(B_max, N, nx, ticks_per_stage=tps, q_weight=list(w), sigma=0.3)
    lm = L.Landmarks(cfg)
    ref = OL.LandmarkReward(N, [cfg.s[l] for l in range(5)], [cfg.alpha[l] for l in range(5)], w, 0.3, 0, 3, tps)
    dev = torch.device("cuda")
    reward = torch.empty(B, device=dev)
    err = torch.empty((B, 5, 3), device=dev)
    count = torch.empty(B, dtype=torch.int32, device=dev)
    start = 1000  # ticks need not start at zero
    seen = 0
    for i in range(T):
        tick = start + i
        if i == 41:
            mask = (rng.uniform(size=B) < 0.3).astype(np.uint8)
            lm.reset(tick, torch.from_numpy(mask).to(dev), B)
            ref.reset(tick, np.nonzero(mask)[0])
        if i % 2 == 0:
            xi = rng.normal(scale=0.2, size=(B, N, nx)).astype(np.float32)
            lm.store(tick, torch.from_numpy(xi).to(dev), B)
            ref.store(tick, xi.astype(np.float64))
        q = rng.normal(scale=0.2, size=(B, 3)).astype(np.float32)
        lm.reward(tick, torch.from_numpy(q).to(dev), reward, B, err=err, count=count)
        r0, e0, c0 = ref.reward(tick, q.astype(np.float64))
        torch.cuda.synchronize()
        assert np.array_equal(count.cpu().numpy(), c0), i
        # r = exp(-x): the FP32 sum x carries ~8 roundings of relative 2^-24 per
        # term, so |dr / r| <= 8 * 2^-24 * x + expf's error (2 ulp); tested with 2x margin
        x = -np.log(r0)
        tol = 2 * (8 * 2.0 ** -24 * x + 2 * 2.0 ** -23)
        assert np.all(np.abs(reward.cpu().numpy() - r0) <= tol * r0), (i, np.max(np.abs(reward.cpu().numpy() / r0 - 1) / tol))
        assert np.allclose(err.cpu().numpy(), e0, rtol=0, atol=1e-6), i
        seen += int(c0.sum())
    assert seen > 5 * B * 10  # most ticks compare several landmarks
    lm.close()


def test_store_from_solver_equals_store_of_copied_trajectory(env):
    torch, L, P = env
    batch = W.generate(W.small_centroidal(B=16, N=10, seed=9))
    s = P.solver_for(batch)
    out = P.solve_workload(batch, solver=s)
    dev = torch.device("cuda")
    xi = torch.from_numpy(out["xi"]).to(dev)
    cfg = L.default_config(16, 10, 13)
    a, b = L.Landmarks(cfg), L.Landmarks(cfg)
    a.store_solution(s, 7)
    b.store(7, xi, 16)
    q = torch.from_numpy(np.random.default_rng(3).normal(size=(16, 3)).astype(np.float32)).to(dev)
    ra, rb = torch.empty(16, device=dev), torch.empty(16, device=dev)
    for n in L.steps(cfg):
        a.reward(7 + n, q, ra, 16)
        b.reward(7 + n, q, rb, 16)
        torch.cuda.synchronize()
        assert torch.equal(ra, rb) and bool((ra < 1).all())
    with pytest.raises(P.MpcError):
        L.Landmarks(L.default_config(16, 12, 13)).store_solution(s, 0)  # horizon mismatch
    a.close(); b.close(); s.close()
