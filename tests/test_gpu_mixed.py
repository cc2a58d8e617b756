"""Uneven batching (mixed contact models, ragged horizons U{5..N}): the
concurrent per-shape solve equals separate solves with the same handle
settings bit for bit, and sampled instances of both shapes match the oracle."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

from parity_util import compare

pytestmark = pytest.mark.gpu


def test_mixed_shapes_and_ragged_horizons():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc
    from paper_2606_05687_b300.mixed import MixedSolver
    batches = [W.generate(sp) for sp in W.uneven_mixed(B=256, N=40, seed=71)]
    assert batches[0].horizon.min() >= 5 and batches[0].horizon.max() <= 40 and len(set(batches[0].horizon)) > 10
    ms = MixedSolver(batches)
    ms.set_stages([pinmpc.device_inputs(b) for b in batches])
    ms.solve()
    got = ms.results()
    ms.close()
    for b, g in zip(batches, got):
        # the same handle settings (horizon classes) solving the sub-batch alone
        rs = pinmpc.solver_for(b)
        rs.set_horizon_classes(pinmpc.horizon_classes_for(b.N))
        ref = pinmpc.solve_workload(b, solver=rs)
        rs.close()
        assert np.array_equal(g["u"], ref["u"]) and np.array_equal(g["status"], ref["status"])
        assert np.all(g["status"] == 0)
        short = [int(i) for i in np.argsort(b.horizon)[:2]] + [int(np.argmax(b.horizon)), 77]
        compare(b, ref, short)
