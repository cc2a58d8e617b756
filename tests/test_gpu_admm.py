"""The paper's ADMM on its own (polish off) through the C ABI, against the
FP64 oracle of the Sec. III iteration (oracle.admm).

The device state of an instance (both buffers of z, v, theta, beta, lambda
per stage, in the solver's internal units u / sigma) is written with
mpc_load_state, a solve of exactly M iterations runs with the polish off
(max_iter = check_start = M), and mpc_save_state (shift 0) reads the iterate
back.  The oracle runs the same M iterations in FP64 from the same
(FP32-rounded) iterate, with dense J_k = (Bbar'Bbar)^{-1}Bbar' and
H_k = (Qbar + rho I + rho Abar_{k+1}'Abar_{k+1})^{-1} -- the device applies
them in a factored form, so this checks the caches (A1), block 1 with the
ebar_{k+1} reading (A2), block 2 and the projection (A3), the duals (A4) and
the restart scheme (A5) against their definitions.

Tolerances (FP32 against FP64).  One iteration applies H_{k-1} (through
W_j and D') and J_k (through S_j) and a handful of stage products; a
rounding error of a few ulps (2^-24) is amplified by the condition numbers
of these solves, at most kappa(H) ~ 90 (walking), 210 (wrenches) and 610
(9-state model) on these batches, so the forward-error bound n kappa(H) u
reaches 1.3e-3 on the 9-state model.  Measured: 9e-7 (walking) to 5.7e-5.
The bar is |gpu - oracle| <= 2e-4 (1 + max |oracle variable|) per variable
for one iteration.  Over M iterations rounding accumulates at most linearly,
since plain ADMM is non-expansive: 2e-4 still holds at M = 200 plain
iterations from a cold start (small iterates early on); 12 accelerated
iterations, whose extrapolation adds up to one more multiple of the previous
step's error per iteration, get 2e-3 (measured 6.6e-4).  Accelerated runs
are compared while the oracle's restart decisions are not within 1e-3
(relative) of their threshold, where the two precisions could decide
differently.  The bars discriminate: the printed reading of htilde_k
(ebar_k in place of ebar_{k+1}) moves one iteration by 6e-3 (9-state model)
to 4e-2 on these batches, and the test checks that the device is more than
ten bars away from it.
"""
import numpy as np
import pytest
import torch

from oracle import admm, qp
from paper_2606_05687_b300 import pinmpc
from paper_2606_05687_b300 import workload as W


def ensure_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()

pytestmark = pytest.mark.gpu

VARS = ("z", "v", "theta", "beta", "lam")


def nbp_of(solver, N):
    f = solver.state_floats(N)
    return (f - 8) // (10 * N)


def pack_state(solver, N, iterates, B):
    """Store rows for B instances: buffer 0 holds each oracle Iterate (first Nh
    stages), buffer 1 zeros, current-buffer index 0."""
    F = solver.state_floats(N)
    nbp = nbp_of(solver, N)
    rows = np.zeros((B, F), np.float32)
    for b, it in enumerate(iterates):
        if it is None:
            continue
        v = rows[b, :10 * N * nbp].reshape(2, N, 5, nbp)
        nh, nb = it.z.shape
        for q, name in enumerate(VARS):
            v[0, :nh, q, :nb] = getattr(it, name)
    return rows


def unpack_state(solver, N, rows, horizons, nb):
    nbp = nbp_of(solver, N)
    out = []
    for b in range(rows.shape[0]):
        cb = int(rows[b, 10 * N * nbp + 4:10 * N * nbp + 5].view(np.int32)[0])
        v = rows[b, :10 * N * nbp].reshape(2, N, 5, nbp)[cb]
        nh = int(horizons[b])
        out.append(admm.Iterate(*(v[:nh, q, :nb].astype(np.float64) for q in range(5))))
    return out


def gpu_iterations(batch, starts, M, accel, **cfg):
    """M ADMM iterations on the GPU from the given iterates (None = cold),
    polish off; returns (iterates after M, solver config)."""
    ensure_lib()
    s = pinmpc.solver_for(batch, polish=0, accel=int(accel), max_iter=M, check_start=M, kkt_tol=1e-30, **cfg)
    t = pinmpc.device_inputs(batch)
    B, N = batch.B, batch.N
    s.set_stages(B, N, **t)
    store = torch.from_numpy(pack_state(s, N, starts, B)).cuda()
    s.load_state(store, None, B)
    s.solve(B)
    out = torch.zeros_like(store)
    s.save_state(out, None, B, shift=0)
    torch.cuda.synchronize()
    its = unpack_state(s, N, out.cpu().numpy(), batch.horizon, batch.nx + batch.nu)
    cfgc = s.cfg
    s.close()
    return its, cfgc


def lifted(batch, b, sigma):
    inst = qp.instance(batch, b)
    si = admm.scaled_instance(inst, sigma)
    L = admm.lift(si, u_prev=batch.u_prev[b].astype(np.float64) / sigma)
    return inst, si, L


def rounded(it):
    return admm.Iterate(*(x.astype(np.float32).astype(np.float64) for x in it.astuple()))


def start_iterates(batch, sigma, rho, m0=10, noise=0.05, seed=0):
    """Realistic iterates: m0 oracle iterations from zero, every second
    instance perturbed (so block 2 meets other projection pieces)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(batch.B):
        _, _, L = lifted(batch, b, sigma)
        w = admm.solve(L, rho, m0, accel=True).w
        if b % 2:
            w = admm.Iterate(*(x + noise * (1.0 + np.abs(x).max()) * rng.normal(size=x.shape)
                               for x in w.astuple()))
        out.append(rounded(w))
    return out


def compare(batch, gpu, starts, M, accel, cfg, tol, margin=1e-3):
    """Runs the oracle from the same starts; returns (worst relative error,
    instances compared).  Fails on any compared instance above tol."""
    sigma, rho = float(cfg.u_scale), float(cfg.rho)
    eta = float(np.float32(cfg.restart_eta))
    worst, compared = 0.0, 0
    for b in range(batch.B):
        _, _, L = lifted(batch, b, sigma)
        run = admm.solve(L, rho, M, accel=accel, eta=eta, start=starts[b])
        if accel and run.margins and min(run.margins[1:] or [np.inf]) < margin:
            continue  # a restart decision too close to call in FP32
        compared += 1
        for name in VARS:
            o = getattr(run.w, name)
            g = getattr(gpu[b], name)
            err = np.abs(g - o).max() / (1.0 + np.abs(o).max())
            assert err <= tol, (b, name, err)
            worst = max(worst, err)
    return worst, compared


SHAPES = {
    # (generator, B, N, extra spec arguments)
    "walking": (W.rl_scale_walking, 48, 8, dict(e_scale=0.05, u_prev_scale=60.0)),
    "wrench": (W.small_centroidal, 48, 10, dict(e_scale=0.05, u_prev_scale=60.0)),
    "wrench_pair": (W.small_centroidal, 12, 40, dict(horizon_min=30, e_scale=0.05)),
    "cd9_walking": (W.centroidal9_walking, 32, 8, dict(u_prev_scale=60.0)),
}


def make_batch(name, seed=71):
    maker, B, N, kw = SHAPES[name]
    batch = W.generate(maker(B=B, N=N, seed=seed, **kw))
    # a nonzero input reference exercises qbar's R r^u part
    batch.ru = (np.random.default_rng(seed).normal(size=batch.ru.shape) * 15.0).astype(np.float32)
    return batch


def shape_cfg(batch):
    cfg = pinmpc.default_config(batch.nx, batch.nc, batch.contact_dim, batch.B, batch.N)
    return float(cfg.u_scale), float(cfg.rho)


@pytest.mark.parametrize("name", list(SHAPES))
def test_one_iteration_matches_the_oracle(name):
    batch = make_batch(name)
    sigma, rho = shape_cfg(batch)
    starts = start_iterates(batch, sigma, rho)
    gpu, cfg = gpu_iterations(batch, starts, 1, accel=False)
    worst, n = compare(batch, gpu, starts, 1, False, cfg, tol=2e-4)
    assert n == batch.B
    # the same iteration with the printed offset ebar_k inside htilde_k
    printed = 0.0
    for b in range(batch.B):
        _, _, L = lifted(batch, b, sigma)
        run = admm.solve(L, rho, 1, accel=False, start=starts[b], e_next=False)
        printed = max(printed, max(np.abs(getattr(gpu[b], v) - getattr(run.w, v)).max()
                                   / (1.0 + np.abs(getattr(run.w, v)).max()) for v in VARS))
    print(f"{name}: worst {worst:.2e}; against the printed htilde offset {printed:.2e}")
    assert printed > 10 * 2e-4


@pytest.mark.parametrize("name", list(SHAPES))
def test_accelerated_iterations_match_the_oracle(name):
    batch = make_batch(name)
    sigma, rho = shape_cfg(batch)
    starts = start_iterates(batch, sigma, rho)
    M = 12
    gpu, cfg = gpu_iterations(batch, starts, M, accel=True)
    worst, n = compare(batch, gpu, starts, M, True, cfg, tol=2e-3)
    assert n >= batch.B // 2, n


@pytest.mark.parametrize("name", ["walking", "wrench"])
def test_two_hundred_plain_iterations_from_cold_match_the_oracle(name):
    """The paper's budget of 200 iterations, plain ADMM, from a cold start."""
    batch = make_batch(name)
    gpu, cfg = gpu_iterations(batch, [None] * batch.B, 200, accel=False)
    nb = batch.nx + batch.nu
    starts = [admm.Iterate.zeros(int(batch.horizon[b]), nb) for b in range(batch.B)]
    compare(batch, gpu, starts, 200, False, cfg, tol=2e-4)


@pytest.mark.parametrize("accel", [1, 0])
@pytest.mark.parametrize("which", ["walking", "wrench"])
def test_plain_admm_reaches_the_oracle_optimum(which, accel):
    """The paper's method alone (polish off), run until its certificate reads
    KKT <= 1e-5 (checked every 10 iterations, cap 20000): FP32 ADMM converges
    slowly and some instances stall above the tolerance (the polish exists
    for them), so at least 80 % must certify; every certified instance
    matches the FP64 optimum within what its residual allows.  The condensed
    QP is strongly convex with modulus >= R_min (the smallest input weight),
    so a point whose stationarity residual is r (infinity norm, per input)
    lies within sqrt(n) r / R_min of the optimum in the 2-norm, n the number
    of inputs; r is at most KKT (1 + max(|R(u - r^u)|, |B'y|)) by the
    checker's normalisation (feasibility and complementarity errors of the
    certified points are far smaller).  u must be within that bound (with the
    oracle checker's KKT of the returned point); xi, the rollout of u, moves
    much less (bar 1e-3 relative, measured <= 1e-5)."""
    from oracle import kkt as okkt
    if which == "walking":
        batch = W.generate(W.rl_scale_walking(B=64, N=5, seed=7, schedule="all_stance", e_scale=0.05,
                                              u_prev_scale=60.0))
    else:
        batch = W.generate(W.small_centroidal(B=64, N=5, seed=7, schedule="all_stance", e_scale=0.05))
    ensure_lib()
    out = pinmpc.solve_workload(batch, polish=0, accel=accel, kkt_tol=1e-5, max_iter=20000, check_start=10,
                                check_every=10, check_growth=1.0)
    ok = np.flatnonzero(out["status"] == pinmpc.CONVERGED)
    assert len(ok) >= 0.8 * batch.B, (len(ok), out["kkt"])
    assert np.all(out["kkt"][ok] <= 1e-5)
    worst = 0.0
    for b in ok:
        inst = qp.instance(batch, b)
        ref = qp.solve_instance(inst)
        u = out["u"][b].astype(np.float64)
        xi = out["xi"][b].astype(np.float64)
        rep = okkt.kkt_residual(inst, xi, u)
        assert rep.kkt <= 2e-5
        y = okkt.costates(inst, xi)
        den = 1.0 + max(np.abs(inst.R * (u - inst.ru)).max(),
                        np.abs(np.einsum("kij,ki->kj", inst.Bm, y)).max())
        bound = np.sqrt(u.size) * rep.kkt * den / inst.R.min()
        eu_abs = np.linalg.norm(u - ref.u)
        ex = np.abs(xi - ref.xi).max() / np.abs(ref.xi).max()
        assert eu_abs <= bound and ex <= 1e-3, (b, eu_abs, bound, ex)
        worst = max(worst, eu_abs / bound)
    print(f"{which} accel {accel}: {len(ok)}/{batch.B} certified, iterations median {np.median(out['iters']):.0f}, "
          f"worst u error / bound {worst:.2f}")
