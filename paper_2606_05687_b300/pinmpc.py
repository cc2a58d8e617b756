"""Thin ctypes binding of the C ABI in include/pinmpc.h (argument marshalling only).

Every step of the solve runs in the CUDA library ``libpinmpc.so`` built from
``csrc/``; this module only converts Python/torch arguments to the C structs
and raw pointers.  A missing library raises ``ImportError`` (there is no
Python or CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpinmpc.so")

MPC_OK, MPC_ERR_INVALID_ARG, MPC_ERR_OOM, MPC_ERR_CUDA, MPC_ERR_STATE, MPC_ERR_UNSUPPORTED = range(6)
CONVERGED, MAX_ITER, NONFINITE, BAD_SET, TIMEOUT, BAD_HORIZON, BAD_DIM, STALLED = range(8)
RUNNING = -1  # status of an instance whose solve has not finished it yet
PREC_FP32, PREC_TF32, PREC_BF16 = range(3)  # mpc_config.precision
STATUS_NAMES = {0: "MPC_OK", 1: "MPC_ERR_INVALID_ARG", 2: "MPC_ERR_OOM", 3: "MPC_ERR_CUDA",
                4: "MPC_ERR_STATE", 5: "MPC_ERR_UNSUPPORTED"}


class MpcConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("n_contacts", ctypes.c_int32),
                ("contact_dim", ctypes.c_int32), ("B_max", ctypes.c_int32),
                ("N_max", ctypes.c_int32), ("rho", ctypes.c_float), ("u_scale", ctypes.c_float),
                ("max_iter", ctypes.c_int32), ("kkt_tol", ctypes.c_float),
                ("check_start", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("check_growth", ctypes.c_float),
                ("polish", ctypes.c_int32), ("accel", ctypes.c_int32),
                ("restart_eta", ctypes.c_float), ("refine_steps", ctypes.c_int32),
                ("refine_alpha", ctypes.c_float), ("foot_half_length", ctypes.c_float),
                ("foot_half_width", ctypes.c_float), ("mem_budget", ctypes.c_uint64),
                ("device", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("kkt_tol_abs", ctypes.c_float)]


_P = ctypes.c_void_p


class StageView(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("N", ctypes.c_int32), ("A", _P), ("Bm", _P), ("e", _P),
                ("Q", _P), ("R", _P), ("ry", _P), ("ru", _P), ("mu", _P), ("fmax", _P),
                ("mask", _P), ("xi0", _P), ("u_prev", _P), ("horizon", _P), ("C", _P), ("nu", _P),
                ("stage_stride", ctypes.c_int32), ("xlo", _P), ("xhi", _P)]


KERNEL_CLASSES = 4
KERNEL_CLASS_NAMES = ("pack", "factor", "round", "polish")

_lib = None


def load() -> ctypes.CDLL:
    """Load libpinmpc.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first")
    lib = ctypes.CDLL(LIB_PATH)
    lib.mpc_default_config.argtypes = [ctypes.POINTER(MpcConfig)] + [ctypes.c_int32] * 5
    lib.mpc_default_config.restype = ctypes.c_int
    lib.mpc_max_horizon.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.mpc_max_horizon.restype = ctypes.c_int32
    lib.mpc_create.argtypes = [ctypes.POINTER(MpcConfig), ctypes.POINTER(ctypes.c_void_p)]
    lib.mpc_create.restype = ctypes.c_int
    lib.mpc_set_stages.argtypes = [ctypes.c_void_p, ctypes.POINTER(StageView), ctypes.c_void_p]
    lib.mpc_set_stages.restype = ctypes.c_int
    lib.mpc_solve_batch.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    lib.mpc_solve_batch.restype = ctypes.c_int
    lib.mpc_get_traj.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_void_p]
    lib.mpc_get_traj.restype = ctypes.c_int
    lib.mpc_get_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.mpc_get_stats.restype = ctypes.c_int
    lib.mpc_warm_start.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    lib.mpc_warm_start.restype = ctypes.c_int
    lib.mpc_state_floats.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.mpc_state_floats.restype = ctypes.c_int64
    lib.mpc_save_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_void_p]
    lib.mpc_save_state.restype = ctypes.c_int
    lib.mpc_load_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_void_p]
    lib.mpc_load_state.restype = ctypes.c_int
    lib.mpc_set_round_events.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    lib.mpc_set_round_events.restype = ctypes.c_int
    lib.mpc_measure_fma_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    lib.mpc_measure_fma_peak.restype = ctypes.c_int
    lib.mpc_set_horizon_classes.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
    lib.mpc_set_horizon_classes.restype = ctypes.c_int
    lib.mpc_set_graph_mode.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.mpc_set_graph_mode.restype = ctypes.c_int
    lib.mpc_get_graph_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.mpc_get_graph_stats.restype = ctypes.c_int
    lib.mpc_get_pivots.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.mpc_get_pivots.restype = ctypes.c_int
    lib.mpc_set_kernel_timing.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.mpc_set_kernel_timing.restype = ctypes.c_int
    lib.mpc_get_kernel_times.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
    lib.mpc_get_kernel_times.restype = ctypes.c_int
    lib.mpc_solve_noalloc.argtypes = [ctypes.POINTER(MpcConfig), ctypes.POINTER(StageView)] + [ctypes.c_void_p] * 6
    lib.mpc_solve_noalloc.restype = ctypes.c_int
    lib.mpc_noalloc_last_error.argtypes = []
    lib.mpc_noalloc_last_error.restype = ctypes.c_char_p
    lib.mpc_destroy.argtypes = [ctypes.c_void_p]
    lib.mpc_destroy.restype = None
    lib.mpc_last_error.argtypes = [ctypes.c_void_p]
    lib.mpc_last_error.restype = ctypes.c_char_p
    lib.mpc_workspace_bytes.argtypes = [ctypes.c_void_p]
    lib.mpc_workspace_bytes.restype = ctypes.c_uint64
    lib.mpc_workspace_estimate.argtypes = [ctypes.POINTER(MpcConfig), ctypes.POINTER(ctypes.c_uint64)]
    lib.mpc_workspace_estimate.restype = ctypes.c_int
    lib.mpc_state_floats_estimate.argtypes = [ctypes.POINTER(MpcConfig), ctypes.c_int32]
    lib.mpc_state_floats_estimate.restype = ctypes.c_int64
    _lib = lib
    return lib


class MpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def default_config(nx: int, n_contacts: int, contact_dim: int, B_max: int, N_max: int,
                   **overrides) -> MpcConfig:
    lib = load()
    cfg = MpcConfig()
    st = lib.mpc_default_config(ctypes.byref(cfg), nx, n_contacts, contact_dim, B_max, N_max)
    if st != MPC_OK:
        raise MpcError(st, "mpc_default_config")
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(f"mpc_config has no field {k!r}")
        setattr(cfg, k, v)
    return cfg


def workspace_estimate(cfg: MpcConfig) -> int:
    """Device bytes mpc_create would allocate for ``cfg`` (host-side, no device)."""
    lib = load()
    out = ctypes.c_uint64()
    st = lib.mpc_workspace_estimate(ctypes.byref(cfg), ctypes.byref(out))
    if st != MPC_OK:
        raise MpcError(st, "mpc_workspace_estimate")
    return int(out.value)


def state_floats_estimate(cfg: MpcConfig, N: int) -> int:
    """Floats of one instance's warm state at stride N for ``cfg``'s shape (no handle)."""
    return int(load().mpc_state_floats_estimate(ctypes.byref(cfg), int(N)))


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensors passed to the C ABI must be contiguous")
        return t.data_ptr()
    if hasattr(t, "ctypes"):  # numpy
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the C ABI must be C-contiguous")
        return t.ctypes.data
    raise TypeError(f"unsupported buffer type {type(t)}")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Solver:
    """One ``mpc_handle``: create, set stages, solve, read results."""

    def __init__(self, cfg: MpcConfig):
        self.lib = load()
        self.cfg = cfg
        h = ctypes.c_void_p()
        st = self.lib.mpc_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != MPC_OK:
            raise MpcError(st, self.lib.mpc_last_error(None).decode())
        self.h = h
        self.nu = cfg.n_contacts * cfg.contact_dim

    def _check(self, st: int, what: str):
        if st != MPC_OK:
            raise MpcError(st, f"{what}: {self.lib.mpc_last_error(self.h).decode()}")

    def set_stages(self, B: int, N: int, *, A, Bm, Q, R, ry, mu, fmax, mask, xi0, e=None,
                   ru=None, u_prev=None, horizon=None, C=None, nu=None, stage_stride=0, xlo=None, xhi=None,
                   stream=None):
        v = StageView(B=B, N=N, A=_ptr(A), Bm=_ptr(Bm), e=_ptr(e), Q=_ptr(Q), R=_ptr(R),
                      ry=_ptr(ry), ru=_ptr(ru), mu=_ptr(mu), fmax=_ptr(fmax), mask=_ptr(mask),
                      xi0=_ptr(xi0), u_prev=_ptr(u_prev), horizon=_ptr(horizon), C=_ptr(C), nu=_ptr(nu),
                      stage_stride=int(stage_stride), xlo=_ptr(xlo), xhi=_ptr(xhi))
        self._keep = (A, Bm, Q, R, ry, mu, fmax, mask, xi0, e, ru, u_prev, horizon, C, nu, xlo, xhi)
        self._check(self.lib.mpc_set_stages(self.h, ctypes.byref(v), _stream_ptr(stream)),
                    "mpc_set_stages")

    def solve(self, B: int, stream=None):
        self._check(self.lib.mpc_solve_batch(self.h, B, _stream_ptr(stream)), "mpc_solve_batch")

    def get_traj(self, xi=None, u=None, status=None, iters=None, kkt=None, active_bits=None,
                 stream=None):
        self._check(self.lib.mpc_get_traj(self.h, _ptr(xi), _ptr(u), _ptr(status), _ptr(iters),
                                          _ptr(kkt), _ptr(active_bits), _stream_ptr(stream)),
                    "mpc_get_traj")

    def get_stats(self, polishes=None, stream=None):
        self._check(self.lib.mpc_get_stats(self.h, _ptr(polishes), _stream_ptr(stream)),
                    "mpc_get_stats")

    def warm_start(self, shift: int = 1, stream=None):
        """Start the next solve from the last solve's final iterate shifted by `shift` stages."""
        self._check(self.lib.mpc_warm_start(self.h, int(shift), _stream_ptr(stream)), "mpc_warm_start")

    def get_pivots(self, pivots=None, stream=None):
        self._check(self.lib.mpc_get_pivots(self.h, _ptr(pivots), _stream_ptr(stream)),
                    "mpc_get_pivots")

    def state_floats(self, N: int) -> int:
        return int(self.lib.mpc_state_floats(self.h, N))

    def save_state(self, store, idx, B: int, shift: int = 1, stream=None):
        """Rows idx[b] of the device tensor `store` receive instance b's state (b < B)."""
        self._check(self.lib.mpc_save_state(self.h, _ptr(store), _ptr(idx), store.shape[0], B, shift,
                                            _stream_ptr(stream)), "mpc_save_state")

    def load_state(self, store, idx, B: int, stream=None):
        """Instances b < B of the next solve start from rows idx[b] of `store`."""
        self._check(self.lib.mpc_load_state(self.h, _ptr(store), _ptr(idx), store.shape[0], B, _stream_ptr(stream)),
                    "mpc_load_state")

    def set_round_events(self, events):
        """Record each of `events` (torch.cuda.Event, already created by a record,
        or raw cudaEvent_t handles) after the matching round of every later solve."""
        raw = [e.cuda_event if hasattr(e, "cuda_event") else int(e) for e in events]
        arr = (ctypes.c_void_p * max(len(raw), 1))(*raw)
        self._check(self.lib.mpc_set_round_events(self.h, arr, len(raw)), "mpc_set_round_events")
        self._round_events = list(events)

    def set_graph_mode(self, enable: bool):
        self._check(self.lib.mpc_set_graph_mode(self.h, 1 if enable else 0), "mpc_set_graph_mode")

    def graph_stats(self):
        """(graphs captured, solves replayed) so far."""
        c, r = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.mpc_get_graph_stats(self.h, ctypes.byref(c), ctypes.byref(r)), "mpc_get_graph_stats")
        return c.value, r.value

    def set_horizon_classes(self, caps):
        """Round-kernel horizon classes (ascending stage counts; [] = one class)."""
        arr = (ctypes.c_int32 * max(len(caps), 1))(*[int(c) for c in caps])
        self._check(self.lib.mpc_set_horizon_classes(self.h, arr if caps else None, len(caps)),
                    "mpc_set_horizon_classes")

    def set_kernel_timing(self, enable: bool):
        self._check(self.lib.mpc_set_kernel_timing(self.h, 1 if enable else 0), "mpc_set_kernel_timing")

    def kernel_times(self, reset: bool = True):
        """{class: (total ms, launches)} for the classes pack, factor, round, polish."""
        ms = (ctypes.c_double * KERNEL_CLASSES)()
        n = (ctypes.c_int64 * KERNEL_CLASSES)()
        self._check(self.lib.mpc_get_kernel_times(self.h, ms, n, 1 if reset else 0), "mpc_get_kernel_times")
        return {name: (ms[i], int(n[i])) for i, name in enumerate(KERNEL_CLASS_NAMES)}

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.mpc_workspace_bytes(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_noalloc(cfg: MpcConfig, B: int, N: int, *, A, Bm, Q, R, ry, mu, fmax, mask, xi0,
                  xi, u, status, iters, kkt, e=None, ru=None, u_prev=None, horizon=None, stream=None):
    """mpc_solve_noalloc: solve from caller-owned device buffers into
    caller-owned device outputs, allocating nothing on the device."""
    lib = load()
    v = StageView(B=B, N=N, A=_ptr(A), Bm=_ptr(Bm), e=_ptr(e), Q=_ptr(Q), R=_ptr(R), ry=_ptr(ry),
                  ru=_ptr(ru), mu=_ptr(mu), fmax=_ptr(fmax), mask=_ptr(mask), xi0=_ptr(xi0),
                  u_prev=_ptr(u_prev), horizon=_ptr(horizon))
    st = lib.mpc_solve_noalloc(ctypes.byref(cfg), ctypes.byref(v), _ptr(xi), _ptr(u), _ptr(status),
                               _ptr(iters), _ptr(kkt), _stream_ptr(stream))
    if st != MPC_OK:
        raise MpcError(st, lib.mpc_noalloc_last_error().decode())


def device_inputs(batch, device="cuda", pin_host=False):
    """The arrays of a ``workload.Batch`` as torch tensors on ``device`` (or in
    pinned host memory with ``pin_host``), keyed by the stage-view names."""
    import numpy as np
    import torch
    out = {}
    for name in ("A", "Bm", "e", "Q", "R", "ry", "ru", "mu", "fmax", "xi0", "u_prev"):
        out[name] = torch.from_numpy(np.ascontiguousarray(getattr(batch, name)))
    out["mask"] = torch.from_numpy(np.ascontiguousarray(batch.mask).view(np.int32))
    out["horizon"] = torch.from_numpy(np.ascontiguousarray(batch.horizon))
    for k, t in out.items():
        out[k] = t.pin_memory() if pin_host else t.to(device)
    return out


def measure_fma_peak(device: int = 0, iters: int = 4096) -> float:
    """Measured FP32 FMA throughput of the device, TFLOP/s."""
    lib = load()
    out = ctypes.c_double()
    st = lib.mpc_measure_fma_peak(device, iters, ctypes.byref(out))
    if st != MPC_OK:
        raise MpcError(st, "mpc_measure_fma_peak")
    return out.value


# Horizon classes for ragged batches: 10 stages (two CTAs per SM), 20 (the
# 640-thread form with TMA prefetch), 32 (one CTA), then the stride itself.
RAGGED_CLASSES = (10, 20, 32)


def horizon_classes_for(N: int) -> list:
    """The RAGGED_CLASSES below a stage stride N."""
    return [c for c in RAGGED_CLASSES if c < N]


def round_schedule(cfg: MpcConfig) -> list:
    """The iteration at which each round of a solve ends (its certificate
    check): check_start, then intervals starting at check_every, each
    check_growth times the previous, capped at max_iter."""
    ends, m0, interval = [], 0, float(cfg.check_every)
    while True:
        if m0 == 0:
            m1 = min(cfg.check_start, cfg.max_iter)
        else:
            m1 = int(min(m0 + interval, cfg.max_iter))
            interval *= cfg.check_growth
        ends.append(m1)
        if m1 >= cfg.max_iter:
            return ends
        m0 = m1


def solver_for(batch, **overrides) -> Solver:
    """A Solver sized for ``batch`` (nx 13, its contact model), config overrides applied."""
    cfg = default_config(batch.nx, batch.nc, batch.contact_dim, batch.B, batch.N, **overrides)
    return Solver(cfg)


def solve_workload(batch, solver: Optional[Solver] = None, device="cuda", **overrides):
    """Solve every instance of ``batch`` on the GPU; returns numpy arrays
    (xi [B,N,nx], u [B,N,nu], status, iters, kkt, active_bits, polishes, pivots)."""
    import numpy as np
    import torch
    s = solver or solver_for(batch, **overrides)
    t = device_inputs(batch, device)
    B, N = batch.B, batch.N
    s.set_stages(B, N, **t)
    s.solve(B)
    dev = torch.device(device)
    xi = torch.empty((B, N, batch.nx), dtype=torch.float32, device=dev)
    u = torch.empty((B, N, batch.nu), dtype=torch.float32, device=dev)
    st = torch.empty(B, dtype=torch.int32, device=dev)
    it = torch.empty(B, dtype=torch.int32, device=dev)
    kk = torch.empty(B, dtype=torch.float32, device=dev)
    bits = torch.empty((B, N), dtype=torch.int64, device=dev)
    npol = torch.empty(B, dtype=torch.int32, device=dev)
    npiv = torch.empty(B, dtype=torch.int32, device=dev)
    s.get_traj(xi, u, st, it, kk, bits)
    s.get_stats(npol)
    s.get_pivots(npiv)
    torch.cuda.synchronize(dev)
    return dict(xi=xi.cpu().numpy(), u=u.cpu().numpy(), status=st.cpu().numpy(),
                iters=it.cpu().numpy(), kkt=kk.cpu().numpy(),
                active_bits=bits.cpu().numpy().view(np.uint64), polishes=npol.cpu().numpy(),
                pivots=npiv.cpu().numpy())
