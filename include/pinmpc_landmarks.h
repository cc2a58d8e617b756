/* Landmark guidance on the GPU: the epilogue of the solve (Sec. II-C).
 *
 * Each MPC solve at time t predicts a trajectory xi^t; Sec. II-C keeps a few
 * "landmarks" of it,
 *     delta_l = n_l dt,   n_l = 1 + floor(s_l (N - 1)),   l = 0 .. N_L - 1,
 *     stored as (t + delta_l, q^t(delta_l)),
 * where q is a guided quantity of the state (the CoM c in the paper's CoM
 * reward; the same construction serves CoM velocity or momentum).  When the
 * rollout reaches time t, each landmark predicted for t is compared with
 * the realised quantity,
 *     e_l(t) = q_t - q^{t - delta_l}(delta_l),
 * landmarks that are unavailable (not stored, or stored before the current
 * episode began) are left out, and the guidance reward is
 *     r_t = exp( - sum_l alpha_l ||e_l(t)||^2_{Q_q} / sigma^2 )   in (0, 1].
 *
 * Time is an integer tick (the caller's clock: e.g. policy steps); one MPC
 * stage spans ticks_per_stage ticks, so landmark l of a store at tick t
 * matures at tick t + n_l * ticks_per_stage.  The object keeps, per
 * environment and landmark, a ring of maturing predictions in device memory
 * (depth: the smallest power of two above N * ticks_per_stage).
 *
 * All pointers to batch data are device pointers; every call is
 * asynchronous on `stream` (NULL: the legacy default stream).  Calls return
 * MPC_OK or an error status (mpc_status of pinmpc.h) with a message from
 * mpc_landmark_last_error; argument errors are detected on the host before
 * anything is enqueued.
 */
#ifndef PINMPC_LANDMARKS_H
#define PINMPC_LANDMARKS_H

#include <stdint.h>

#include "pinmpc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MPC_MAX_LANDMARKS 8
#define MPC_MAX_GUIDED_DIM 8

typedef struct mpc_landmark_config {
    int32_t n_landmarks;     /* N_L, 1 .. MPC_MAX_LANDMARKS */
    int32_t horizon;         /* N of the stored trajectories, >= 1 */
    int32_t nx;              /* state dimension of the stored trajectories */
    int32_t q_index;         /* first state component of the guided quantity (0: CoM position
                                of the 13-state model) */
    int32_t q_dim;           /* its number of components, 1 .. MPC_MAX_GUIDED_DIM */
    int32_t ticks_per_stage; /* ticks per MPC stage (dt), >= 1 */
    int32_t B_max;           /* environments */
    int32_t device;          /* CUDA device ordinal */
    float s[MPC_MAX_LANDMARKS];        /* s_l in [0, 1], nondecreasing (Sec. II-C: s_0 = 0,
                                          s_{N_L-1} = 1) */
    float alpha[MPC_MAX_LANDMARKS];    /* alpha_l >= 0 (the paper: decreasing, > 0) */
    float q_weight[MPC_MAX_GUIDED_DIM]; /* diagonal of Q_q, >= 0 */
    float sigma;             /* sigma > 0 */
} mpc_landmark_config;

typedef struct mpc_landmarks mpc_landmarks;

/* The paper's setting: N_L = 5, s_l = l / (N_L - 1), alpha = {0.5, 0.25,
 * 0.15, 0.07, 0.03} (Sec. II-C), the CoM position (components 0..2),
 * Q_q = I, sigma = 1, one tick per stage. */
mpc_status mpc_landmark_default_config(mpc_landmark_config* cfg, int32_t B_max, int32_t horizon, int32_t nx);

/* Stage indices n_l of cfg (n[l] for l < N_L; host only, no device). */
mpc_status mpc_landmark_steps(const mpc_landmark_config* cfg, int32_t* n);

/* Validate cfg and allocate the rings (every slot empty, every episode
 * started at the beginning of time). */
mpc_status mpc_landmark_create(const mpc_landmark_config* cfg, mpc_landmarks** out);

/* Store the landmarks of B trajectories predicted at tick `tick`:
 * xi [B][N][nx] (row k = state at stage k + 1, the layout of mpc_get_traj),
 * landmark l of environment b = xi[b][n_l - 1][q_index .. q_index + q_dim). */
mpc_status mpc_landmark_store(mpc_landmarks* lm, int64_t tick, const float* xi, int32_t B, void* stream);

/* The same from the last solve of handle h (its device-resident output,
 * no copy); enqueue it on the stream that solve was enqueued on. */
mpc_status mpc_landmark_store_solution(mpc_landmarks* lm, mpc_handle* h, int64_t tick, void* stream);

/* Reward at tick `tick` for the realised quantities q_now [B][q_dim]:
 * reward [B]; optionally err [B][N_L][q_dim] (e_l, zero where unavailable)
 * and count [B] (landmarks available).  Either optional pointer may be NULL. */
mpc_status mpc_landmark_reward(mpc_landmarks* lm, int64_t tick, const float* q_now, float* reward, float* err,
                               int32_t* count, int32_t B, void* stream);

/* Episodes of the environments b < B with mask[b] != 0 begin at `tick`:
 * their landmarks stored before it become unavailable. */
mpc_status mpc_landmark_reset(mpc_landmarks* lm, int64_t tick, const uint8_t* mask, int32_t B, void* stream);

/* Message of the last failed call on lm (or of the last failed create when lm is NULL). */
const char* mpc_landmark_last_error(mpc_landmarks* lm);

/* Free the rings (synchronizes the device first). */
void mpc_landmark_destroy(mpc_landmarks* lm);

#ifdef __cplusplus
}
#endif

#endif /* PINMPC_LANDMARKS_H */
