"""The C-ABI library builds, loads, exports every declared symbol and matches
the header's struct layout (CPU only: no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pinmpc.h")
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h")]


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05687_b300 import pinmpc
    return pinmpc


def declared_functions():
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpc_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(P):
    lib = P.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, flags=re.M), n


def test_struct_layout_matches_header(tmp_path, P):
    src = tmp_path / "layout.c"
    fields_cfg = [f[0] for f in P.MpcConfig._fields_]
    fields_view = [f[0] for f in P.StageView._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pinmpc.h"', "int main(void){",
             'printf("%zu\\n", sizeof(mpc_config));']
    lines += [f'printf("%zu\\n", offsetof(mpc_config, {f}));' for f in fields_cfg]
    lines += ['printf("%zu\\n", sizeof(mpc_stage_view));']
    lines += [f'printf("%zu\\n", offsetof(mpc_stage_view, {f}));' for f in fields_view]
    lines += ["return 0;}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(P.MpcConfig)] + [getattr(P.MpcConfig, f).offset for f in fields_cfg]
    want += [ctypes.sizeof(P.StageView)] + [getattr(P.StageView, f).offset for f in fields_view]
    assert got == want


def test_status_codes_match_header(tmp_path, P):
    names = ["MPC_CONVERGED", "MPC_MAX_ITER", "MPC_NONFINITE", "MPC_BAD_SET", "MPC_TIMEOUT", "MPC_BAD_HORIZON",
             "MPC_BAD_DIM", "MPC_STALLED", "MPC_RUNNING"]
    src = tmp_path / "codes.c"
    src.write_text("\n".join(['#include <stdio.h>', '#include "pinmpc.h"', "int main(void){"] +
                             [f'printf("%d\\n", (int){n});' for n in names] + ["return 0;}"]))
    exe = tmp_path / "codes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == [P.CONVERGED, P.MAX_ITER, P.NONFINITE, P.BAD_SET, P.TIMEOUT, P.BAD_HORIZON, P.BAD_DIM,
                   P.STALLED, P.RUNNING]


def test_defaults_and_limits(P):
    cfg = P.default_config(13, 8, 3, 4096, 20)
    assert cfg.rho == 100.0 and cfg.u_scale == 300.0 and cfg.kkt_tol == pytest.approx(2e-6)
    assert cfg.polish == 1 and cfg.accel == 1
    lib = P.load()
    assert lib.mpc_max_horizon(13, 24) == 64  # one warp per stage, two CTAs above 32
    assert lib.mpc_max_horizon(13, 12) == 64
    assert lib.mpc_max_horizon(13, 7) == 0


def test_argument_errors_without_device(P):
    lib = P.load()
    h = ctypes.c_void_p()
    bad = P.default_config(13, 8, 4, 16, 20)
    assert lib.mpc_create(ctypes.byref(bad), ctypes.byref(h)) == P.MPC_ERR_INVALID_ARG
    assert b"contact_dim" in lib.mpc_last_error(None)
    unsup = P.default_config(12, 8, 3, 16, 20)
    assert lib.mpc_create(ctypes.byref(unsup), ctypes.byref(h)) == P.MPC_ERR_UNSUPPORTED
    too_long = P.default_config(13, 8, 3, 16, 65)
    assert lib.mpc_create(ctypes.byref(too_long), ctypes.byref(h)) == P.MPC_ERR_UNSUPPORTED
    neg = P.default_config(13, 8, 3, 16, 20, rho=-1.0)
    assert lib.mpc_create(ctypes.byref(neg), ctypes.byref(h)) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_set_stages(None, None, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_solve_batch(None, 1, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_get_stats(None, None, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_get_pivots(None, None, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_warm_start(None, 1, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_set_kernel_timing(None, 1) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_set_graph_mode(None, 1) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_state_floats(None, 20) == 0
    assert lib.mpc_set_round_events(None, None, 0) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_set_horizon_classes(None, None, 0) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_measure_fma_peak(0, 16, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_save_state(None, None, None, 1, 1, 1, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_load_state(None, None, None, 1, 1, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_get_graph_stats(None, None, None) == P.MPC_ERR_INVALID_ARG
    assert lib.mpc_get_kernel_times(None, None, None, 0) == P.MPC_ERR_INVALID_ARG
    lib.mpc_destroy(None)


def test_no_device_is_an_error_not_a_fallback(P):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(P.MpcError) as ei:
        P.Solver(P.default_config(13, 8, 3, 16, 20))
    assert ei.value.code == P.MPC_ERR_CUDA


def test_workspace_and_state_estimates_on_the_host(P):
    """mpc_workspace_estimate / mpc_state_floats_estimate size a handle for a
    memory budget without a device: linear in B_max, errors for unbuilt
    shapes (the GPU tests check the estimate equals mpc_workspace_bytes)."""
    w1 = P.workspace_estimate(P.default_config(13, 8, 3, 100, 20))
    w2 = P.workspace_estimate(P.default_config(13, 8, 3, 200, 20))
    w3 = P.workspace_estimate(P.default_config(13, 8, 3, 300, 20))
    assert 0 < w1 < w2 < w3 and (w3 - w2) == (w2 - w1)
    # per instance at N = 20: records (47 KB), factor cache (33 KB), ADMM state (32 KB), gains (25 KB), outputs
    assert 130_000 < (w2 - w1) / 100 < 160_000
    lib = P.load()
    out = ctypes.c_uint64()
    assert lib.mpc_workspace_estimate(ctypes.byref(P.default_config(12, 8, 3, 16, 20)), ctypes.byref(out)) == \
        P.MPC_ERR_UNSUPPORTED
    assert lib.mpc_workspace_estimate(ctypes.byref(P.default_config(13, 8, 3, 0, 20)), ctypes.byref(out)) == \
        P.MPC_ERR_INVALID_ARG
    assert lib.mpc_workspace_estimate(None, ctypes.byref(out)) == P.MPC_ERR_INVALID_ARG
    cfg = P.default_config(13, 8, 3, 16, 20)
    assert P.state_floats_estimate(cfg, 20) == 2 * 5 * 20 * 40 + 8
    assert P.state_floats_estimate(cfg, 0) == 0 and P.state_floats_estimate(cfg, 65) == 0
