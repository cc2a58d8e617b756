"""Batched parallel-in-horizon MPC-QP solver (pi^n MPC, Sec. III) for B300.

The solver lives in a C-ABI shared library built from ``csrc/`` (CUDA for
sm_103a); ``pinmpc`` is its thin ctypes binding and ``workload`` the seeded
synthetic input generator.
"""
