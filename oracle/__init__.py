"""FP64 CPU oracle for the batched centroidal LTV-MPC solve (test infrastructure).

This package is test infrastructure.  Only the tests, the package's smoke
check and the benchmark's CPU-baseline leg may import it.  It shares no code
with the CUDA path: it solves the assembled (condensed) quadratic program of
Sec. III directly, by a dense primal-dual interior-point method, so its answer
is the plain definition of what the parallel-in-horizon ADMM converges to
(the unique optimum of a strictly convex QP).

Modules
    qp        condensed QP assembly + Mehrotra predictor-corrector IPM
    kkt       primal-only KKT residual checker and active-face bits
    project   exact Euclidean projection onto a generalized friction pyramid

Parity status: the QP optimum, the KKT checker and the projection are pinned
by tests against closed forms (finite-horizon LQR), brute-force active-set
enumeration, library routines and invariants.  ADMM iterates and iteration
counts are "parity unpinned": the paper prints no iterate values.
"""
