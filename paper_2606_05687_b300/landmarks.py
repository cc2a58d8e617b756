"""ctypes binding of the landmark epilogue (include/pinmpc_landmarks.h).

Argument marshalling only: storing landmarks and evaluating the guidance
reward run in the library's kernels (csrc/landmarks.cu).  Batch buffers are
device tensors (float32, int32 or uint8 as documented in the header).
"""
from __future__ import annotations

import ctypes
from typing import Optional

from . import pinmpc
from .pinmpc import MPC_OK, MpcError, _ptr, _stream_ptr

MAX_LANDMARKS = 8
MAX_GUIDED_DIM = 8


class LandmarkConfig(ctypes.Structure):
    _fields_ = [("n_landmarks", ctypes.c_int32), ("horizon", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("q_index", ctypes.c_int32), ("q_dim", ctypes.c_int32), ("ticks_per_stage", ctypes.c_int32),
                ("B_max", ctypes.c_int32), ("device", ctypes.c_int32),
                ("s", ctypes.c_float * MAX_LANDMARKS), ("alpha", ctypes.c_float * MAX_LANDMARKS),
                ("q_weight", ctypes.c_float * MAX_GUIDED_DIM), ("sigma", ctypes.c_float)]


_bound = False


def _lib() -> ctypes.CDLL:
    global _bound
    lib = pinmpc.load()
    if not _bound:
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        cfgp = ctypes.POINTER(LandmarkConfig)
        lib.mpc_landmark_default_config.argtypes = [cfgp, I32, I32, I32]
        lib.mpc_landmark_steps.argtypes = [cfgp, P]
        lib.mpc_landmark_create.argtypes = [cfgp, ctypes.POINTER(ctypes.c_void_p)]
        lib.mpc_landmark_store.argtypes = [P, I64, P, I32, P]
        lib.mpc_landmark_store_solution.argtypes = [P, P, I64, P]
        lib.mpc_landmark_reward.argtypes = [P, I64, P, P, P, P, I32, P]
        lib.mpc_landmark_reset.argtypes = [P, I64, P, I32, P]
        lib.mpc_landmark_last_error.argtypes = [P]
        lib.mpc_landmark_last_error.restype = ctypes.c_char_p
        lib.mpc_landmark_destroy.argtypes = [P]
        lib.mpc_landmark_destroy.restype = None
        for n in ("mpc_landmark_default_config", "mpc_landmark_steps", "mpc_landmark_create", "mpc_landmark_store",
                  "mpc_landmark_store_solution", "mpc_landmark_reward", "mpc_landmark_reset"):
            getattr(lib, n).restype = ctypes.c_int
        _bound = True
    return lib


def default_config(B_max: int, horizon: int, nx: int = 13, **overrides) -> LandmarkConfig:
    """The paper's setting (N_L = 5, s_l = l/4, alpha = .5/.25/.15/.07/.03, CoM
    position, Q = I, sigma = 1, one tick per stage); list-valued overrides
    (s, alpha, q_weight) fill the leading entries."""
    cfg = LandmarkConfig()
    st = _lib().mpc_landmark_default_config(ctypes.byref(cfg), B_max, horizon, nx)
    if st != MPC_OK:
        raise MpcError(st, "mpc_landmark_default_config")
    for k, v in overrides.items():
        if k in ("s", "alpha", "q_weight"):
            arr = getattr(cfg, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        elif hasattr(cfg, k):
            setattr(cfg, k, v)
        else:
            raise AttributeError(f"mpc_landmark_config has no field {k!r}")
    return cfg


def steps(cfg: LandmarkConfig) -> list:
    """n_l = 1 + floor(s_l (N - 1)) as the library computes them."""
    out = (ctypes.c_int32 * MAX_LANDMARKS)()
    st = _lib().mpc_landmark_steps(ctypes.byref(cfg), out)
    if st != MPC_OK:
        raise MpcError(st, "mpc_landmark_steps")
    return list(out[:cfg.n_landmarks])


class Landmarks:
    """One ``mpc_landmarks`` object: landmark rings of B_max environments."""

    def __init__(self, cfg: LandmarkConfig):
        self.lib = _lib()
        self.cfg = cfg
        h = ctypes.c_void_p()
        st = self.lib.mpc_landmark_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != MPC_OK:
            raise MpcError(st, self.lib.mpc_landmark_last_error(None).decode())
        self.h = h

    def _check(self, st: int, what: str):
        if st != MPC_OK:
            raise MpcError(st, f"{what}: {self.lib.mpc_landmark_last_error(self.h).decode()}")

    def store(self, tick: int, xi, B: int, stream=None):
        self._check(self.lib.mpc_landmark_store(self.h, tick, _ptr(xi), B, _stream_ptr(stream)), "mpc_landmark_store")

    def store_solution(self, solver: "pinmpc.Solver", tick: int, stream=None):
        self._check(self.lib.mpc_landmark_store_solution(self.h, solver.h, tick, _stream_ptr(stream)),
                    "mpc_landmark_store_solution")

    def reward(self, tick: int, q_now, reward, B: int, err=None, count=None, stream=None):
        self._check(self.lib.mpc_landmark_reward(self.h, tick, _ptr(q_now), _ptr(reward), _ptr(err), _ptr(count), B,
                                                 _stream_ptr(stream)), "mpc_landmark_reward")

    def reset(self, tick: int, mask, B: int, stream=None):
        self._check(self.lib.mpc_landmark_reset(self.h, tick, _ptr(mask), B, _stream_ptr(stream)), "mpc_landmark_reset")

    def close(self):
        if self.h:
            self.lib.mpc_landmark_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
