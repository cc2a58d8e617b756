"""Per-kernel timing and work counters of the C ABI (observability; no
counterpart in the paper): the event pairs cover exactly the launches a
solve makes, and the pivot counts agree with the polish counts."""
import numpy as np
import pytest

from paper_2606_05687_b300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pinmpc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc as P
    return P


def test_kernel_times_cover_each_launch_class(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=128, N=20, seed=1002))
    s = pinmpc.solver_for(batch)
    t = pinmpc.device_inputs(batch)
    s.set_stages(batch.B, batch.N, **t)
    s.solve(batch.B)
    assert all(n == 0 for _, n in s.kernel_times().values())  # timing is off by default
    s.set_kernel_timing(True)
    for _ in range(2):
        s.set_stages(batch.B, batch.N, **t)
        s.solve(batch.B)
    kt = s.kernel_times(reset=True)
    assert kt["pack"][1] == 2 and kt["factor"][1] == 2
    assert kt["round"][1] >= 2 and kt["round"][1] == kt["polish"][1]
    assert all(ms > 0.0 for ms, n in kt.values() if n > 0)
    assert all(n == 0 for _, n in s.kernel_times().values())  # reset cleared the totals
    s.set_kernel_timing(False)
    s.solve(batch.B)
    assert all(n == 0 for _, n in s.kernel_times().values())
    s.close()


def test_pivot_counts(pinmpc):
    batch = W.generate(W.rl_scale_walking(B=128, N=20, seed=1002))
    out = pinmpc.solve_workload(batch)
    pol, piv = out["polishes"], out["pivots"]
    assert np.all(out["status"] == 0)
    # every Riccati scan eliminates between 0 and nu free pivots per stage
    assert np.all(piv >= 0) and np.all(piv <= pol * batch.N * batch.nu)
    assert np.all((pol == 0) == (piv == 0))


def test_measured_fma_peak_is_near_the_derived_one(pinmpc):
    """The FMA microbenchmark lands near SMs x 128 lanes x 2 x max clock."""
    import torch
    props = torch.cuda.get_device_properties(0)
    t = pinmpc.measure_fma_peak(0, iters=2048)
    derived = props.multi_processor_count * 128 * 2 * 2.032e9 / 1e12
    assert 0.5 * derived < t < 1.1 * derived, (t, derived)
    with pytest.raises(pinmpc.MpcError):
        pinmpc.measure_fma_peak(0, iters=0)
