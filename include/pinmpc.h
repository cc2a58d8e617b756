/*
 * pinmpc.h -- C ABI of the batched parallel-in-horizon MPC-QP solver.
 *
 * Each instance b of a batch is the linear time-varying MPC problem of
 * Sec. III (the standard form stated there, with C = I):
 *
 *   min  sum_{k=0}^{N-1} 1/2 ||C_k xi_{k+1} - r^y_k||^2_{Q_k} + 1/2 ||u_k - r^u_k||^2_{R_k}
 *   s.t. xi_{k+1} = A_k xi_k + B_k u_k + e_k,   xi_0 given,
 *        xi_{k+1} in X_k (an optional box),
 *        u_k in U_k  (a product over contacts of contact sets),
 * with C_k diagonal (I unless given).
 *
 * Contact sets (Sec. II-B names the friction pyramid and the contact wrench
 * cone): a stance contact's components (t, n) lie in the generalized pyramid
 * {|t_j| <= c_j n, 0 <= n <= n_max}; a swing contact's components are 0.
 *   contact_dim 3 (point force f_x, f_y, f_z):   t = (f_x, f_y), c = (mu, mu)
 *   contact_dim 6 (foot wrench f, tau):           t = (f_x, f_y, tau_x, tau_y, tau_z),
 *       c = (mu, mu, d_y, d_x, mu*min(d_x, d_y)), d_x/d_y the foot half length/width.
 *
 * The solver is the velocity-form, variable-splitting ADMM of Sec. III
 * (lifted state [xi_k; u_{k-1}], splits z = lifted state and v = Bbar du,
 * closed-form horizon-parallel updates with per-stage caches J_k, H_k, and
 * Nesterov acceleration with restart).  Every stage update of an iteration
 * runs in parallel; there is no Riccati recursion in the iteration and no
 * assembled QP.  To certify the tolerance the solver may additionally fix
 * the active faces read off the iterate and solve that equality-constrained
 * LQR exactly (a "polish", a backward Riccati scan), accepting it only when
 * an on-device KKT certificate passes.
 *
 * Conventions
 *   - All functions return an mpc_status; none aborts or traps.
 *   - Floating-point data is FP32, row-major, instance-major: stage arrays are
 *     [B][S][...] with S = the view's stage_stride (default its N <= N_max),
 *     of which the first N stages of each instance are read.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*; NULL = the legacy default stream) and is asynchronous unless
 *     stated otherwise.
 *   - A handle is not thread-safe: use one handle per host thread/stream.
 *   - Pointers may be device pointers or host pointers (pinned host memory
 *     keeps the copies asynchronous); the library detects which.
 */
#ifndef PINMPC_H
#define PINMPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mpc_status {
    MPC_OK = 0,
    MPC_ERR_INVALID_ARG = 1,  /* bad dimension, null required pointer, bad value */
    MPC_ERR_OOM = 2,          /* workspace does not fit the memory budget / device */
    MPC_ERR_CUDA = 3,         /* a CUDA call failed; see mpc_last_error */
    MPC_ERR_STATE = 4,        /* call out of order (e.g. solve before set_stages) */
    MPC_ERR_UNSUPPORTED = 5   /* valid request outside the compiled shapes or limits */
} mpc_status;

/* Per-instance result codes written by mpc_get_traj's status array. */
enum {
    MPC_CONVERGED = 0,  /* KKT certificate <= kkt_tol */
    MPC_MAX_ITER = 1,   /* iteration cap reached; outputs are the last iterate, or the best
                           polished point if one came within 4 kkt_tol and closer */
    MPC_NONFINITE = 2,  /* NaN/Inf in this instance's inputs */
    MPC_BAD_SET = 3,    /* empty contact set (n_max < 0 or mu < 0 on a stance contact) */
    MPC_TIMEOUT = 4,    /* reserved for bounded device-side waits */
    MPC_BAD_HORIZON = 5, /* horizon[b] outside [1, N] */
    MPC_BAD_DIM = 6,     /* nu[b] not a multiple of contact_dim in [0, nu] */
    MPC_STALLED = 7,     /* stopped before the cap: a polished point's certificate came
                            within 4 kkt_tol and the faces of the iterate then held for two
                            checks; outputs are that point, kkt its certificate (the FP32
                            floor of the certificate rises with the horizon, so past ~40
                            stages a few instances on the right faces sit above kkt_tol) */
    MPC_RUNNING = -1     /* not finished yet: read before the solve has passed
                            the round that finishes the instance */
};

/* Solver configuration; fill with mpc_default_config then adjust. */
typedef struct mpc_config {
    int32_t nx;            /* state dimension: 13, or 9 (the 9-state centroidal model) */
    int32_t n_contacts;    /* contacts per stage: 8 (contact_dim 3) or 2 (contact_dim 6) */
    int32_t contact_dim;   /* 3 or 6; nu = n_contacts * contact_dim */
    int32_t B_max;         /* largest batch passed to mpc_set_stages */
    int32_t N_max;         /* largest horizon (see mpc_max_horizon) */
    float rho;             /* ADMM penalty (scaled form), > 0 (Sec. III's rho) */
    float u_scale;         /* internal input scale sigma: the solver works in u/sigma */
    int32_t max_iter;      /* ADMM iteration cap (the paper's experiments use 200) */
    float kkt_tol;         /* certificate tolerance on the KKT residual */
    int32_t check_start;   /* first iteration at which a certificate check runs */
    int32_t check_every;   /* iterations between the first and second checks */
    float check_growth;    /* each later interval is the previous one times this (>= 1): the few
                              instances left after the first checks run more cheap ADMM
                              iterations per polish round */
    int32_t polish;        /* 1: polish on the read-off active set before certifying;
                              0: certify the ADMM iterate itself (the plain method) */
    int32_t accel;         /* 1: fast ADMM with restart; 0: plain ADMM */
    float restart_eta;     /* restart threshold eta in (0, 1) */
    int32_t refine_steps;  /* after a failed polish: up to this many active-set updates, each
                              reading the faces off Proj(u - refine_alpha * grad) and polishing again;
                              in the first two rounds -- each later round doubles it, up to 32, for
                              the few instances still running */
    float refine_alpha;    /* step of that projected-gradient active-set update (scaled units) */
    float foot_half_length;/* d_x of the wrench cone (contact_dim 6) */
    float foot_half_width; /* d_y of the wrench cone (contact_dim 6) */
    uint64_t mem_budget;   /* device bytes this handle may allocate; 0 = no limit */
    int32_t device;        /* CUDA device ordinal */
    int32_t precision;     /* operands of the per-stage Gram products behind the ADMM caches
                              (B_k B_k' and T_k D'^-1 T_k' with T_k = [A_k B_k], Sec. III's
                              J_k and H_k): MPC_PREC_FP32 (default), or MPC_PREC_TF32 /
                              MPC_PREC_BF16 on the tensor cores with FP32 accumulation.  The
                              iteration, the polish and the certificate stay FP32: the
                              certified KKT bound holds for every mode (the polish and its
                              refinement recover what the rounded caches lose) */
    float kkt_tol_abs;     /* absolute part of the certificate's tolerance: each KKT term must
                              satisfy |residual| <= kkt_tol_abs + kkt_tol * scale, its scale
                              being n_max (feasibility), max(|R(u - r^u)|, |B'y|)
                              (stationarity) or |u|_inf (complementarity); the reported kkt is
                              max |residual| / (kkt_tol_abs / kkt_tol + scale).  0 = kkt_tol
                              (the default: |residual| / (1 + scale) <= kkt_tol) */
} mpc_config;

/* mpc_config.precision */
enum { MPC_PREC_FP32 = 0, MPC_PREC_TF32 = 1, MPC_PREC_BF16 = 2 };

/* Stage data of one batch.  Arrays are instance-major with stage stride N. */
typedef struct mpc_stage_view {
    int32_t B;              /* instances in this batch, 1..B_max */
    int32_t N;              /* stage stride of the arrays, 1..N_max */
    const float* A;         /* [B][N][nx][nx]  required */
    const float* Bm;        /* [B][N][nx][nu]  required */
    const float* e;         /* [B][N][nx]      NULL = 0 */
    const float* Q;         /* [B][N][nx]      diagonal of Q_k, > 0, required */
    const float* R;         /* [B][N][nu]      diagonal of R_k, > 0, required */
    const float* ry;        /* [B][N][nx]      state reference r^y_k, required */
    const float* ru;        /* [B][N][nu]      input reference r^u_k, NULL = 0 */
    const float* mu;        /* [B][N][nc]      friction coefficient per contact, required */
    const float* fmax;      /* [B][N][nc]      normal-force bound per contact, required */
    const uint32_t* mask;   /* [B][N]          bit c set = contact c in stance, required */
    const float* xi0;       /* [B][nx]         initial state, required */
    const float* u_prev;    /* [B][nu]         u_{-1} of the velocity form, NULL = 0 */
    const int32_t* horizon; /* [B]            per-instance horizon <= N, NULL = N */
    const float* C;         /* [B][N][nx]     diagonal of the output map C_k of the stage cost
                                              1/2 ||C_k xi_{k+1} - r^y_k||^2_{Q_k} (Sec. III's standard
                                              form); NULL = I.  Diagonal maps only (a weight or a
                                              selection per state component); a zero entry drops that
                                              component from the cost */
    const int32_t* nu;      /* [B]            inputs present in instance b: a multiple of contact_dim
                                              up to the handle's nu; its first nu[b] / contact_dim
                                              contacts take part, the others are absent (held at 0,
                                              whatever their mask bits).  NULL = all.  Another count
                                              gives that instance the status MPC_BAD_DIM */
    int32_t stage_stride;   /* stages between consecutive instances in the stage arrays, >= N (the
                               arrays are [B][stage_stride][...] and the first N stages of each
                               instance are read); 0 = N */
    const float* xlo;       /* [B][N][nx]     state box X_k of Sec. III's standard form,       */
    const float* xhi;       /* [B][N][nx]     xlo_k <= xi_{k+1} <= xhi_k (+-INFINITY: unbounded
                                              component); either or both NULL = unbounded.  The
                                              ADMM projects the state part of z onto the box; the
                                              polish holds the bounds its iterate sits at exactly
                                              (an equality row of the first stage, at or before the
                                              bound's, whose inputs move the component; up to 4 per
                                              stage) or else by an augmented Lagrangian, and the
                                              certificate includes their feasibility and multipliers */
} mpc_stage_view;

typedef struct mpc_handle mpc_handle;

/* Fill *cfg with defaults for the given problem shape (rho 100, u_scale
 * 300, max_iter 1000, kkt_tol 2e-6 -- a fifth of the 1e-5 target: the
 * certificate bounds the KKT residual, and where only R pins a direction
 * (the split of a foot's net force over its corner contacts) the input error
 * can reach ~30x that residual -- checks at iterations 12, 32, 72, 152, ...
 * (check_start 12, check_every 20, check_growth 2), polish on with up to 3
 * refinement steps of alpha 0.01, acceleration on with eta 0.999, foot
 * 0.10 x 0.05 m).  For foot wrenches (contact_dim 6) on the 13-state model:
 * rho 300, check_start 32 (checks at 32, 52, 92, ...), up to 4 refinement
 * steps of alpha 0.001.  The check schedule, the refinement step and rho are
 * this implementation's choices (the paper checks convergence every
 * iteration and has no polish); they were chosen by measured throughput on
 * the walking and small centroidal workloads of each shape. */
mpc_status mpc_default_config(mpc_config* cfg, int32_t nx, int32_t n_contacts,
                              int32_t contact_dim, int32_t B_max, int32_t N_max);

/* Largest horizon N_max that mpc_create accepts for (nx, nu): 64 for both
 * built shapes (one warp per stage; above 32 stages each ADMM round runs as a
 * thread-block cluster of two CTAs per instance, half of the stages in each);
 * 0 if the shape is not built.  mpc_solve_noalloc has a lower limit of its
 * own (below). */
int32_t mpc_max_horizon(int32_t nx, int32_t nu);

/* Validate cfg, select its device and allocate the workspace (owned by the
 * handle).  MPC_ERR_OOM if the workspace exceeds mem_budget or the device's
 * free memory; MPC_ERR_UNSUPPORTED outside the build's limits. */
mpc_status mpc_create(const mpc_config* cfg, mpc_handle** out);

/* Copy and repack the batch's stage data into the workspace on `stream`
 * (Sec. III's stage matrices, scaled internally by u_scale).  The caller may
 * reuse its buffers once `stream` has passed this call. */
mpc_status mpc_set_stages(mpc_handle* h, const mpc_stage_view* v, void* stream);

/* Solve instances [0, B) of the last set_stages batch on `stream`
 * (asynchronous: the whole round schedule up to max_iter is enqueued and the
 * call returns without waiting; instances that finish leave the later
 * rounds' work lists).  Convergence is reported per instance, not here. */
mpc_status mpc_solve_batch(mpc_handle* h, int32_t B, void* stream);

/* Copy results of the last solve to caller buffers (device or host; any
 * pointer may be NULL to skip it):
 *   xi          [B][N][nx]  states xi_1..xi_N (xi_0 excluded)
 *   u           [B][N][nu]  inputs u_0..u_{N-1}
 *   status      [B]         MPC_CONVERGED / MPC_MAX_ITER / ...
 *   iters       [B]         ADMM iterations run
 *   kkt         [B]         KKT certificate of the returned (xi, u)
 *   active_bits [B][N]      bit (c*F + f) = face f of contact c active, with
 *                           F = 2*(contact_dim==3 ? 2 : 5) + 2 faces per contact
 *                           ordered (+t_1, -t_1, +t_2, -t_2, ..., -n <= 0, n <= n_max);
 *                           a face is active when g_f(u) >= -1e-5 (1 + n_max)
 * Stages at or beyond an instance's horizon are written as 0.  Device or
 * host pointers: with pageable host memory this call synchronizes `stream`;
 * with device or page-locked (pinned) memory it is asynchronous, and the
 * results are there once `stream` has passed this call. */
mpc_status mpc_get_traj(mpc_handle* h, float* xi, float* u, int32_t* status,
                        int32_t* iters, float* kkt, uint64_t* active_bits, void* stream);

/* Per-instance solver statistics of the last solve: polishes [B] = number
 * of active-set polish attempts (Riccati scans) the instance ran.  Device
 * or host pointer; pageable host memory synchronizes `stream` (see
 * mpc_get_traj). */
mpc_status mpc_get_stats(mpc_handle* h, int32_t* polishes, void* stream);

/* Receding-horizon warm start: the next mpc_solve_batch starts instances
 * [0, B) of the last solve from their final ADMM iterate (z, v and the
 * scaled duals theta, beta, lambda) moved `shift` stages towards the start of
 * each instance's horizon, the last stage repeated into the freed tail, with
 * the acceleration restarted; shift 0 re-solves from the final iterate.
 * Call after mpc_solve_batch and before (or after) mpc_set_stages of the next
 * batch, with the same horizon stride N; one solve consumes it.  A warm start
 * changes the iterate the method starts from, not the problem: the certified
 * solution is the same (same tolerance).  Requires a previous solve
 * (MPC_ERR_STATE) and 0 <= shift < N (MPC_ERR_INVALID_ARG).  The paper solves
 * each MPC step cold; this is the standard receding-horizon practice. */
mpc_status mpc_warm_start(mpc_handle* h, int32_t shift, void* stream);

/* Free pivots the polish eliminated in the last solve, per instance [B]:
 * summed over its Riccati scans, the number of free input components of
 * every stage (the elimination steps actually run).  A work count for
 * throughput accounting; no counterpart in the paper.  Device or host
 * pointer; pageable host memory synchronizes `stream` (see mpc_get_traj). */
mpc_status mpc_get_pivots(mpc_handle* h, int32_t* pivots, void* stream);

/* Per-kernel device timing (no counterpart in the paper; off by default).
 * While enabled, mpc_set_stages and mpc_solve_batch record a CUDA event pair
 * around every kernel they launch, on the caller's stream.
 * mpc_get_kernel_times waits for the recorded events, adds their durations to
 * per-class totals and copies the totals out: ms[c] milliseconds and
 * launches[c] launches of class c = 0 pack, 1 factor, 2 ADMM round,
 * 3 polish (host arrays of MPC_KERNEL_CLASSES entries; either may be NULL);
 * reset != 0 clears the totals afterwards.  Events are created on first use
 * and reused; failure to create one leaves that launch untimed. */
#define MPC_KERNEL_CLASSES 4
mpc_status mpc_set_kernel_timing(mpc_handle* h, int32_t enable);
mpc_status mpc_get_kernel_times(mpc_handle* h, double* ms, int64_t* launches, int32_t reset);

/* Early results (no counterpart in the paper; for servers that answer each
 * request as soon as its instance is certified).  Every instance's status
 * reads MPC_RUNNING from the start of mpc_solve_batch until the round that
 * finishes it writes its final status, trajectory and certificate.  With
 * events[r] (cudaEvent_t, caller-owned; NULL entries skipped) for r < n,
 * every later mpc_solve_batch records events[r] on its stream right after
 * round r (checks at check_start, then the growing intervals): work waiting
 * on it (mpc_get_traj on another stream, for instance) sees the instances
 * finished by then with their final results.  n = 0 clears the events;
 * changing them frees the cached solve graphs. */
mpc_status mpc_set_round_events(mpc_handle* h, void* const* events, int32_t n);

/* Per-environment warm state (no counterpart in the paper; it extends the
 * receding-horizon warm start of mpc_warm_start to callers that re-form
 * their batches, such as a server that batches whichever environments have
 * pending requests, so an environment lands in a different slot each time).
 * The state of one instance is its final ADMM iterate (both buffers of
 * (z, v, theta, beta, lambda)) and acceleration scalars:
 * mpc_state_floats(h, N) floats at horizon stride N (0 for a null handle or
 * N outside [1, N_max]).
 *   mpc_save_state: after a solve, row idx[b] of `store` receives instance
 *     b's state for b < B (B <= the solved batch), its stages moved `shift`
 *     stages towards the start of its horizon as in mpc_warm_start; idx NULL
 *     means row b.  An instance whose solve failed saves a cold (zero) state.
 *   mpc_load_state: instances b < B of the batch set by mpc_set_stages
 *     start the next mpc_solve_batch from row idx[b] of `store` (saved at
 *     the same N); the others start cold.  Put the environments with saved
 *     state first in the batch.
 * `store` (`rows` rows) and `idx` ([B] int32, or NULL) are caller-owned
 * device memory of the handle's device; host or other-device pointers are
 * rejected with MPC_ERR_INVALID_ARG before anything is launched.  Indices
 * outside [0, rows) are not written (save) or start cold (load).  A save
 * whose idx names one row for several slots writes that row from all of them
 * at once (a mix): give -1 to every slot but one.  Both calls are
 * asynchronous on `stream`. */
int64_t mpc_state_floats(mpc_handle* h, int32_t N);
/* mpc_state_floats for cfg's shape without a handle (host only; 0 for an
 * unbuilt shape or N outside [1, 64]): for sizing a store by a memory budget. */
int64_t mpc_state_floats_estimate(const mpc_config* cfg, int32_t N);
mpc_status mpc_save_state(mpc_handle* h, float* store, const int32_t* idx, int32_t rows, int32_t B, int32_t shift,
                          void* stream);
mpc_status mpc_load_state(mpc_handle* h, const float* store, const int32_t* idx, int32_t rows, int32_t B,
                          void* stream);

/* FP32 FMA throughput of `device` in TFLOP/s (FMA = 2 flops) into *tflops:
 * a kernel of 8 independent FMA chains per thread, 8 CTAs of 256 threads per
 * SM, `iters` steps per chain, timed with CUDA events after one warm-up
 * launch.  The measured denominator beside the derived SMs x 128 lanes x 2
 * x clock peak of a roofline; a measurement utility with no counterpart in
 * the paper.  Allocates and frees a small output buffer.
 * MPC_ERR_INVALID_ARG (null tflops, iters < 1, bad device), MPC_ERR_OOM,
 * MPC_ERR_CUDA. */
mpc_status mpc_measure_fma_peak(int32_t device, int32_t iters, double* tflops);

/* Horizon classes (optional; default one class).  The paper's method is
 * parallel in the horizon: one warp per stage, an instance's round held by
 * one CTA sized for the handle's stage stride N, so an instance with a short
 * horizon occupies a CTA sized for N.  With classes, each ADMM round runs
 * once per class: instances whose horizon is at most caps[0] on CTAs sized
 * for caps[0] stages (several per SM when they fit), those up to caps[1] on
 * the next size, ..., the rest on CTAs sized for N.  The instances still
 * running after a round join their class's list.  Results are identical
 * with and without classes (the same arithmetic per instance); only the
 * placement differs.  Each solve adds one launch per class and round.
 *   caps: n ascending stage counts in [1, N_max] (host memory, copied); caps
 *         at or above a solve's N are ignored by that solve.  n: 0 .. 3
 *         (0 = one class).  MPC_ERR_INVALID_ARG otherwise.  Drops the
 *         captured graphs (mpc_set_graph_mode).
 * This is an implementation choice with no counterpart in the paper. */
mpc_status mpc_set_horizon_classes(mpc_handle* h, const int32_t* caps, int32_t n);

/* CUDA-graph replay of the solve (no counterpart in the paper; a launch-cost
 * aid).  With enable != 0, mpc_solve_batch records its device work (flag
 * resets, the factor kernel and the whole round schedule) into a CUDA graph
 * on an internal stream the first time it meets a (B, N, warm-start count)
 * combination, keeps up to 4 such graphs, and thereafter enqueues the
 * solve as one graph launch on `stream`: the results are bit-identical to
 * the direct launches, the host cost per solve drops to one call.  While
 * per-kernel timing is on, solves use direct launches.  enable = 0 frees
 * the graphs.  mpc_get_graph_stats: graphs captured and solves replayed so
 * far (either pointer may be NULL). */
mpc_status mpc_set_graph_mode(mpc_handle* h, int32_t enable);
mpc_status mpc_get_graph_stats(mpc_handle* h, int64_t* captures, int64_t* replays);

/* Solve a batch without allocating any device memory (no counterpart in the
 * paper; this is a deployment aid).  For callers that may not allocate: code
 * inside someone else's captured CUDA graph, a simulator step that owns a
 * fixed memory pool and forbids cudaMalloc on its hot path, or a real-time
 * loop that must stay clear of the allocator.  It runs on the calling
 * thread's current CUDA device, and the caller passes buffers of that device
 * only (host pointers and other GPUs' memory are rejected: staging them
 * would allocate):
 * the stage view as for mpc_set_stages, and the outputs xi [B][N][nx],
 * u [B][N][nu], status, iters, kkt [B] as for mpc_get_traj.  The solver's
 * scratch (packed records, face bits, polish counts) is a fixed 8 MiB static
 * device array that every GPU loading the library holds until process exit;
 * a batch needing more (about 170 instances at N=20, nu=24) is rejected with
 * MPC_ERR_UNSUPPORTED and a message (mpc_noalloc_last_error).  The first call
 * on a device looks up the array's device address and opts the kernel into
 * its shared memory, so make that first call before any stream capture.
 * Every call shares the one array: calls whose work overlaps on the GPU
 * (different streams, or host threads) race and must be serialized by the
 * caller.  Each call rewrites every scratch word it reads, so nothing carries
 * over from the previous call.  Its single kernel holds a whole instance in
 * shared memory, which caps the horizon at 24 stages for nu = 24 (32 for
 * nu = 12); a longer one is rejected with MPC_ERR_UNSUPPORTED. */
mpc_status mpc_solve_noalloc(const mpc_config* cfg, const mpc_stage_view* v, float* xi, float* u,
                             int32_t* status, int32_t* iters, float* kkt, void* stream);

/* Message of the last failed mpc_solve_noalloc on this host thread. */
const char* mpc_noalloc_last_error(void);

/* Free the handle and its workspace (synchronizes the device first). */
void mpc_destroy(mpc_handle* h);

/* Last error message of h (or of the last failed mpc_create when h is NULL). */
const char* mpc_last_error(mpc_handle* h);

/* Bytes of device memory the handle owns. */
uint64_t mpc_workspace_bytes(mpc_handle* h);

/* Device bytes mpc_create would allocate for cfg (the value
 * mpc_workspace_bytes reports right after creation), computed on the host
 * without a device and without allocating, so that a caller can admit work
 * by a device-memory budget before creating handles.  A handle that later
 * receives host-memory inputs adds a staging buffer of the batch's input size
 * on first use.  No counterpart in the paper.  MPC_ERR_INVALID_ARG (null
 * pointers, bad dimensions), MPC_ERR_UNSUPPORTED (shape not built, N_max
 * above mpc_max_horizon's limit). */
mpc_status mpc_workspace_estimate(const mpc_config* cfg, uint64_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* PINMPC_H */
