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
