"""Reduced-precision caches (mpc_config.precision): the per-stage Gram
products behind J_k and H_k on the tensor cores in TF32 or BF16 (FP32
accumulation), with the polish and its refinement recovering the accuracy.

FP32 and TF32 must certify every instance at the same KKT tolerance and
match the FP64 oracle at the same bars as the FP32 path.  BF16 keeps 8 bits
of mantissa in the caches, so its ADMM reads faces off a coarser fixed
point; the polish still certifies what it returns, but an instance may run
out of iterations (measured: 1 of 64 foot-wrench instances at max_iter
1000).  BF16 may therefore leave up to 2 % uncertified, reported as
MPC_MAX_ITER or MPC_STALLED with the certificate above the tolerance, never
as a converged wrong answer; every certified instance
must match the oracle.  The per-instance error against the oracle is
reported beside the FP32 one.  The rounded caches
do change the ADMM iteration: one iteration from a loaded iterate departs
from the FP64 iteration by about the operand rounding (2^-11 for TF32,
2^-8 for BF16) times the caches' condition, which the test checks against
the FP32 mode's departure (ordered FP32 < TF32 < BF16, all bounded)."""
import numpy as np
import pytest
import torch

from oracle import admm
from paper_2606_05687_b300 import pinmpc
from paper_2606_05687_b300 import workload as W

from parity_util import compare
import test_gpu_admm as TA

pytestmark = pytest.mark.gpu
MODES = {"fp32": pinmpc.PREC_FP32, "tf32": pinmpc.PREC_TF32, "bf16": pinmpc.PREC_BF16}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("maker,B,N", [(W.rl_scale_walking, 256, 20), (W.small_centroidal, 64, 10)])
def test_every_precision_certifies_and_matches_the_oracle(mode, maker, B, N):
    TA.ensure_lib()
    batch = W.generate(maker(B=B, N=N, seed=1101))
    out = pinmpc.solve_workload(batch, precision=MODES[mode])
    ok = out["status"] == pinmpc.CONVERGED
    if mode == "bf16":
        assert (~ok).sum() <= max(1, B // 50)
        assert np.all(np.isin(out["status"][~ok], [pinmpc.MAX_ITER, pinmpc.STALLED]))
        assert np.all(out["kkt"][~ok] > 2e-6)
    else:
        assert np.all(ok), np.flatnonzero(~ok)
    assert out["kkt"][ok].max() <= 1e-5
    ids = [b for b in range(0, B, max(1, B // 24)) if ok[b]]
    worst = compare(batch, out, ids)
    print(f"{maker.__name__} {mode}: {ok.sum()}/{B} certified, worst {worst}, iters mean {out['iters'].mean():.1f}, "
          f"polishes mean {out['polishes'].mean():.2f}")


def test_rounded_caches_change_the_iteration_by_their_rounding():
    batch = TA.make_batch("walking")
    sigma, rho = TA.shape_cfg(batch)
    starts = TA.start_iterates(batch, sigma, rho)
    err = {}
    for mode, prec in MODES.items():
        gpu, cfg = TA.gpu_iterations(batch, starts, 1, accel=False, precision=prec)
        worst = 0.0
        for b in range(batch.B):
            _, _, L = TA.lifted(batch, b, sigma)
            run = admm.solve(L, rho, 1, accel=False, start=starts[b])
            for v in TA.VARS:
                o = getattr(run.w, v)
                worst = max(worst, np.abs(getattr(gpu[b], v) - o).max() / (1.0 + np.abs(o).max()))
        err[mode] = worst
    print("one-iteration departure from the FP64 iteration:", err)
    assert err["fp32"] < err["tf32"] < err["bf16"] < 0.5
    assert err["tf32"] > 10 * err["fp32"]
