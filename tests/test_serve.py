"""Continuous batching (serve.py): arrival generator on CPU; on the GPU, a
request's result does not depend on the batch it was served in, and a short
load run certifies every request."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W


def test_poisson_arrivals():
    from paper_2606_05687_b300.serve import poisson_arrivals
    a = poisson_arrivals(2000.0, 2.0, 64, seed=3)
    assert np.all(np.diff(a[:, 0]) > 0) and a[-1, 0] < 2.0 and a[0, 0] >= 0.0
    assert abs(len(a) - 4000) < 4 * np.sqrt(4000)          # Poisson count around rate * duration
    assert a[:, 1].min() >= 0 and a[:, 1].max() < 64


@pytest.fixture(scope="module")
def pinmpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc as P
    return P


@pytest.mark.gpu
def test_served_results_equal_standalone(pinmpc):
    from paper_2606_05687_b300.serve import BatchServer
    batch = W.generate(W.rl_scale_walking(B=64, N=20, seed=21))
    ref = pinmpc.solve_workload(batch)
    pool = pinmpc.device_inputs(batch)
    srv = BatchServer(pool, batch.nx, batch.nc, batch.contact_dim, B_max=24, N=batch.N, n_handles=2)
    srv.keep_results = True
    order = [5, 63, 5, 17, 0, 33, 17, 40, 2, 63] + list(range(0, 64, 3))
    for e in order[:7]:
        srv.submit(e)          # one at a time
    srv.submit(order[7:])      # and as a block
    srv.drain()
    assert srv.batches >= 2 and srv.n == len(order)
    for r, e in enumerate(order):
        assert srv.env[r] == e and srv.status[r] == 0
        got = srv.results[r]
        assert np.array_equal(got["u"], ref["u"][e]), e
        assert np.array_equal(got["xi"], ref["xi"][e]), e
    srv.close()


@pytest.mark.gpu
def test_short_load_run(pinmpc):
    from paper_2606_05687_b300.serve import BatchServer, poisson_arrivals, serve_load
    batch = W.generate(W.rl_scale_walking(B=256, N=20, seed=22))
    pool = pinmpc.device_inputs(batch)
    srv = BatchServer(pool, batch.nx, batch.nc, batch.contact_dim, B_max=256, N=batch.N, n_handles=2)
    rep = serve_load(srv, poisson_arrivals(20000.0, 0.2, 256, seed=1))
    print(rep)
    assert rep["certified"] == rep["requests"] > 0
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    srv.close()


@pytest.mark.gpu
def test_saved_state_equals_handle_warm_start_across_slots(pinmpc):
    # mpc_save_state / mpc_load_state move each environment's state between
    # slots exactly: a permuted re-batch starts from the same iterate as the
    # in-place receding warm start
    import torch
    batch = W.generate(W.rl_scale_walking(B=48, N=20, seed=23))
    a = pinmpc.solver_for(batch)
    first = pinmpc.solve_workload(batch, solver=a)
    nxt = batch.receding(first["xi"][:, 0], first["u"][:, 0])
    a.warm_start(1)
    ref = pinmpc.solve_workload(nxt, solver=a)
    b = pinmpc.solver_for(batch)
    pinmpc.solve_workload(batch, solver=b)
    rng = np.random.default_rng(4)
    rows = rng.permutation(64)[:48].astype(np.int32)                 # env e -> store row rows[e]
    store = torch.zeros((64, b.state_floats(20)), device="cuda")
    b.save_state(store, torch.from_numpy(rows).cuda(), 48, shift=1)
    q = rng.permutation(48)                                           # slot s of the next batch holds env q[s]
    b.set_stages(48, 20, **pinmpc.device_inputs(nxt.subset(q)))
    b.load_state(store, torch.from_numpy(rows[q]).cuda(), 48)
    b.solve(48)
    u = torch.empty((48, 20, 24), device="cuda")
    it = torch.empty(48, dtype=torch.int32, device="cuda")
    b.get_traj(None, u, None, it, None, None)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), ref["u"][q]) and np.array_equal(it.cpu().numpy(), ref["iters"][q])
    a.close()
    b.close()


@pytest.mark.gpu
def test_served_warm_state_and_resets(pinmpc):
    # with warm_shift 0 on unchanged stage data, an environment's second request
    # starts from its first solution (as a handle's warm_start(0) would) and a
    # reset one starts cold again, bit for bit, whatever the batching
    from paper_2606_05687_b300.serve import BatchServer
    batch = W.generate(W.rl_scale_walking(B=40, N=20, seed=24))
    s = pinmpc.solver_for(batch)
    cold = pinmpc.solve_workload(batch, solver=s)
    s.warm_start(0)
    warm = pinmpc.solve_workload(batch, solver=s)
    s.close()
    srv = BatchServer(pinmpc.device_inputs(batch), batch.nx, batch.nc, batch.contact_dim, B_max=16, N=batch.N,
                      n_handles=2, warm_shift=0)
    srv.keep_results = True
    first = list(range(40))
    srv.submit(first)
    srv.drain()
    srv.reset([3, 7])
    second = [7, 39, 0, 3, 12] + list(range(13, 39, 2))
    for e in second[:3]:
        srv.submit(e)
    srv.submit(second[3:])
    srv.drain()
    assert srv.warm_loads == len(second) - 2
    for r, e in enumerate(first):
        assert srv.status[r] == 0 and np.array_equal(srv.results[r]["u"], cold["u"][e])
    for i, e in enumerate(second):
        r = len(first) + i
        want = cold if e in (3, 7) else warm
        assert srv.status[r] == 0 and np.array_equal(srv.results[r]["u"], want["u"][e]), e
    srv.close()


@pytest.mark.gpu
def test_back_to_back_requests_follow_serial_order(pinmpc):
    # requests of one environment that land on different handles while the
    # previous one is still on the GPU: each starts from the state its
    # predecessor saved, exactly as a single handle's warm starts in series
    from paper_2606_05687_b300.serve import BatchServer
    batch = W.generate(W.rl_scale_walking(B=12, N=20, seed=25))
    s = pinmpc.solver_for(batch)
    serial = [pinmpc.solve_workload(batch, solver=s)]
    for _ in range(3):
        s.warm_start(0)
        serial.append(pinmpc.solve_workload(batch, solver=s))
    s.close()
    for rep in range(2):
        srv = BatchServer(pinmpc.device_inputs(batch), batch.nx, batch.nc, batch.contact_dim, B_max=1, N=batch.N,
                          n_handles=3, warm_shift=0)
        srv.keep_results = True
        order = [5, 5, 5, 5, 9, 2, 9]
        srv.submit(order)          # all queued at once: consecutive requests go to different handles
        srv.drain()
        seen = {}
        for r, e in enumerate(order):
            k = seen.get(e, 0)
            seen[e] = k + 1
            assert srv.status[r] == 0
            assert np.array_equal(srv.results[r]["u"], serial[k]["u"][e]), (rep, r, e, k)
        srv.close()
