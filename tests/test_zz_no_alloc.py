"""mpc_solve_noalloc -- the entry point for callers that may not allocate
device memory (code inside another owner's captured CUDA graph, a simulator
step with a fixed memory pool, a real-time loop kept clear of the allocator).

It must give the same answers as the regular handle-based entry point
(mpc_set_stages + mpc_solve_batch + mpc_get_traj), within the parity
tolerance of the other GPU tests, on two calls in a row that share its fixed
scratch array, and meet the parity bars against the FP64 oracle directly.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

from parity_util import KKT_TOL, REL_TRAJ, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc
    return pinmpc


def _noalloc(P, batch):
    import torch
    t = P.device_inputs(batch, "cuda")
    B, N = batch.B, batch.N
    xi = torch.empty((B, N, batch.nx), dtype=torch.float32, device="cuda")
    u = torch.empty((B, N, batch.nu), dtype=torch.float32, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    it = torch.empty(B, dtype=torch.int32, device="cuda")
    kk = torch.empty(B, dtype=torch.float32, device="cuda")
    cfg = P.default_config(batch.nx, batch.nc, batch.contact_dim, B, N)
    P.solve_noalloc(cfg, B, N, **t, xi=xi, u=u, status=st, iters=it, kkt=kk)
    torch.cuda.synchronize()
    return dict(xi=xi.cpu().numpy(), u=u.cpu().numpy(), status=st.cpu().numpy(), kkt=kk.cpu().numpy(),
                iters=it.cpu().numpy())


def test_no_alloc_matches_regular_entry_point_twice(P):
    batches = [W.generate(W.rl_scale_walking(B=48, N=20, seed=2024)),
               W.generate(W.small_centroidal(B=40, N=10, seed=2025))]
    for batch in batches:  # two calls in a row through the shared scratch
        ref = P.solve_workload(batch)
        got = _noalloc(P, batch)
        assert np.array_equal(got["status"], ref["status"])
        assert np.all(got["status"] == 0) and got["kkt"].max() <= KKT_TOL
        su = np.abs(ref["u"]).max(axis=(1, 2))
        sx = np.abs(ref["xi"]).max(axis=(1, 2))
        eu = (np.abs(got["u"] - ref["u"]).max(axis=(1, 2)) / su).max()
        ex = (np.abs(got["xi"] - ref["xi"]).max(axis=(1, 2)) / sx).max()
        assert eu <= REL_TRAJ and ex <= REL_TRAJ, (eu, ex)


def test_no_alloc_meets_the_oracle_bars(P):
    """The no-allocation path against the FP64 oracle itself: trajectories,
    oracle-checked KKT, objective gap and the device certificate, on both
    contact models (the active-face bits are not among its outputs)."""
    for batch, ids in ((W.generate(W.rl_scale_walking(B=24, N=20, seed=2028)), [0, 5, 11, 17, 23]),
                       (W.generate(W.small_centroidal(B=16, N=10, seed=2029)), [0, 3, 8, 15])):
        got = _noalloc(P, batch)
        compare(batch, got, ids, check_bits=False)


def test_no_alloc_rejects_batches_beyond_its_scratch(P):
    import torch
    batch = W.generate(W.rl_scale_walking(B=400, N=20, seed=2026))
    with pytest.raises(P.MpcError) as ei:
        _noalloc(P, batch)
    assert ei.value.code == P.MPC_ERR_UNSUPPORTED
    assert "scratch" in str(ei.value)
    torch.cuda.synchronize()


def test_no_alloc_rejects_horizons_beyond_its_kernel(P):
    # its single kernel holds a whole instance in shared memory: 24 stages at
    # most for point contacts (nu = 24), while the handle path takes 64
    import torch
    batch = W.generate(W.rl_scale_walking(B=4, N=25, seed=2027))
    with pytest.raises(P.MpcError) as ei:
        _noalloc(P, batch)
    assert ei.value.code == P.MPC_ERR_UNSUPPORTED
    assert "shared memory" in str(ei.value)
    torch.cuda.synchronize()
