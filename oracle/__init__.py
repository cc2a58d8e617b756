"""FP64 CPU oracle for the batched centroidal LTV-MPC solve (test infrastructure).

This package is test infrastructure.  Only the tests, the package's smoke
check and the benchmark's CPU legs may import it.  It shares no code with the
CUDA path.  It solves the assembled (condensed) quadratic program of Sec. III
directly, by a dense primal-dual interior-point method, so its answer is the
plain definition of what the parallel-in-horizon ADMM converges to (the
unique optimum of a strictly convex QP); and it writes out the section's ADMM
iteration itself, with dense J_k and H_k, so the GPU's iterates can be
checked step by step.

Modules
    qp         condensed QP assembly + Mehrotra predictor-corrector IPM + crossover
    kkt        primal-only KKT residual checker and active-face bits
    project    contact sets and the exact Euclidean projection onto them
    admm       the Sec. III ADMM (lifted form, closed-form blocks, fast ADMM with restart)
    landmarks  the landmark guidance of Sec. II-C

Parity status: the QP optimum, the KKT checker, the active-face bits and the
projection are pinned by tests against closed forms (finite-horizon LQR),
hand-derived golden values, brute-force enumeration (active sets, face
subsets), library routines and invariants.  The ADMM blocks are pinned by the
augmented Lagrangian they minimise and by their fixed point, the pinned QP
optimum.  The paper prints no iterate values, so ADMM iteration counts are
not pinned to the paper; the GPU's iterates are compared with this module's.
"""
