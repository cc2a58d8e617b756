// Landmark guidance (Sec. II-C): storage of a solve's landmarks in per-
// environment rings and the guidance reward, as small kernels over the
// environments.
//   store:  thread (b, l) writes q^t(delta_l) = xi_b[n_l - 1][q_index ..] and
//           its maturity tick t + n_l * ticks_per_stage into ring slot
//           maturity mod depth of (b, l);
//   reward: thread b compares q_now[b] with the slots of tick t that hold
//           exactly tick t and were stored at or after b's episode start
//           (t - delta_l >= start[b]), and sums alpha_l ||e_l||^2_Q;
//   reset:  thread b moves b's episode start.
// A slot written at tick t' is overwritten only by a store at t' + k depth,
// k >= 1; depth > N ticks_per_stage, so every landmark survives to maturity.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <new>
#include <string>

#include "../../include/pinmpc_landmarks.h"
#include "internal.h"

namespace {

constexpr int64_t kEmpty = INT64_MIN;  // tick of a slot never written

struct LmParams {
    int n[MPC_MAX_LANDMARKS];        // n_l
    float alpha[MPC_MAX_LANDMARKS];  // alpha_l
    float w[MPC_MAX_GUIDED_DIM];     // diagonal of Q_q
};

__global__ void lm_fill_kernel(int64_t* p, size_t n, int64_t v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void lm_store_kernel(const float* xi, int B, int N, int nx, int q_index, int q_dim, int nl, LmParams prm,
                                int tps, int64_t tick, int depth, int64_t* ticks, float* vals) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * nl) return;
    const int b = i / nl, l = i % nl;
    const int64_t mat = tick + (int64_t)prm.n[l] * tps;
    const size_t e = ((size_t)b * nl + l) * depth + (size_t)(mat & (int64_t)(depth - 1));
    const float* src = xi + ((size_t)b * N + (prm.n[l] - 1)) * nx + q_index;
    for (int j = 0; j < q_dim; ++j) vals[e * q_dim + j] = src[j];
    ticks[e] = mat;
}

__global__ void lm_reward_kernel(int B, int nl, int q_dim, LmParams prm, int tps, int64_t tick, int depth,
                                 const int64_t* ticks, const float* vals, const int64_t* start, const float* q_now,
                                 float inv_sigma2, float* reward, float* err, int* count) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const size_t slot = (size_t)(tick & (int64_t)(depth - 1));
    const int64_t st = start[b];
    float acc = 0.0f;
    int cnt = 0;
    for (int l = 0; l < nl; ++l) {
        const size_t e = ((size_t)b * nl + l) * depth + slot;
        const bool ok = ticks[e] == tick && tick - (int64_t)prm.n[l] * tps >= st;
        float s2 = 0.0f;
        for (int j = 0; j < q_dim; ++j) {
            const float d = ok ? q_now[(size_t)b * q_dim + j] - vals[e * q_dim + j] : 0.0f;
            s2 = fmaf(prm.w[j] * d, d, s2);
            if (err) err[((size_t)b * nl + l) * q_dim + j] = d;
        }
        if (ok) {
            acc = fmaf(prm.alpha[l], s2, acc);
            ++cnt;
        }
    }
    reward[b] = expf(-acc * inv_sigma2);
    if (count) count[b] = cnt;
}

__global__ void lm_reset_kernel(int B, const uint8_t* mask, int64_t tick, int64_t* start) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B && mask[b]) start[b] = tick;
}

thread_local std::string g_lm_create_error;

}  // namespace

struct mpc_landmarks {
    mpc_landmark_config cfg{};
    LmParams prm{};
    int depth = 0;
    int64_t* ticks = nullptr;  // [B_max][N_L][depth]
    float* vals = nullptr;     // [B_max][N_L][depth][q_dim]
    int64_t* start = nullptr;  // [B_max] episode start ticks
    std::string error;
};

static mpc_status lm_fail(mpc_landmarks* lm, mpc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    (lm ? lm->error : g_lm_create_error) = buf;
    return st;
}

static mpc_status lm_cuda(mpc_landmarks* lm, cudaError_t e, const char* what) {
    return lm_fail(lm, MPC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// n_l = 1 + floor(s_l (N - 1)) (Sec. II-C); validates the parameters on the way.
static mpc_status lm_steps(const mpc_landmark_config* c, int* n, std::string* why) {
    auto bad = [&](const char* m) {
        if (why) *why = m;
        return MPC_ERR_INVALID_ARG;
    };
    if (!c) return bad("null config");
    if (c->n_landmarks < 1 || c->n_landmarks > MPC_MAX_LANDMARKS) return bad("n_landmarks outside 1..8");
    if (c->horizon < 1) return bad("horizon must be >= 1");
    if (c->q_dim < 1 || c->q_dim > MPC_MAX_GUIDED_DIM) return bad("q_dim outside 1..8");
    if (c->nx < 1 || c->q_index < 0 || c->q_index + c->q_dim > c->nx) return bad("q_index + q_dim exceeds nx");
    if (c->ticks_per_stage < 1) return bad("ticks_per_stage must be >= 1");
    if ((int64_t)c->horizon * c->ticks_per_stage >= (int64_t)1 << 20) return bad("horizon * ticks_per_stage must be < 2^20");
    if (c->B_max < 1) return bad("B_max must be >= 1");
    if (!(c->sigma > 0.0f) || !std::isfinite(c->sigma)) return bad("sigma must be > 0");
    for (int l = 0; l < c->n_landmarks; ++l) {
        const float s = c->s[l];
        if (!(s >= 0.0f && s <= 1.0f)) return bad("s_l outside [0, 1]");
        if (l > 0 && s < c->s[l - 1]) return bad("s_l must be nondecreasing");
        if (!(c->alpha[l] >= 0.0f) || !std::isfinite(c->alpha[l])) return bad("alpha_l must be >= 0");
        n[l] = 1 + (int)std::floor((double)s * (double)(c->horizon - 1));
        if (n[l] > c->horizon) n[l] = c->horizon;
    }
    for (int j = 0; j < c->q_dim; ++j)
        if (!(c->q_weight[j] >= 0.0f) || !std::isfinite(c->q_weight[j])) return bad("q_weight must be >= 0");
    return MPC_OK;
}

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

extern "C" {

mpc_status mpc_landmark_default_config(mpc_landmark_config* cfg, int32_t B_max, int32_t horizon, int32_t nx) {
    if (!cfg) return MPC_ERR_INVALID_ARG;
    *cfg = mpc_landmark_config{};
    cfg->n_landmarks = 5;
    cfg->horizon = horizon;
    cfg->nx = nx;
    cfg->q_index = 0;
    cfg->q_dim = 3;
    cfg->ticks_per_stage = 1;
    cfg->B_max = B_max;
    cfg->device = 0;
    const float alpha[5] = {0.5f, 0.25f, 0.15f, 0.07f, 0.03f};
    for (int l = 0; l < 5; ++l) {
        cfg->s[l] = (float)l / 4.0f;
        cfg->alpha[l] = alpha[l];
    }
    for (int j = 0; j < MPC_MAX_GUIDED_DIM; ++j) cfg->q_weight[j] = 1.0f;
    cfg->sigma = 1.0f;
    return MPC_OK;
}

mpc_status mpc_landmark_steps(const mpc_landmark_config* cfg, int32_t* n) {
    if (!cfg || !n) return MPC_ERR_INVALID_ARG;
    int tmp[MPC_MAX_LANDMARKS];
    const mpc_status st = lm_steps(cfg, tmp, nullptr);
    if (st != MPC_OK) return st;
    for (int l = 0; l < cfg->n_landmarks; ++l) n[l] = tmp[l];
    return MPC_OK;
}

mpc_status mpc_landmark_create(const mpc_landmark_config* cfg, mpc_landmarks** out) {
    g_lm_create_error.clear();
    if (!cfg || !out) return lm_fail(nullptr, MPC_ERR_INVALID_ARG, "null config or output pointer");
    *out = nullptr;
    LmParams prm{};
    std::string why;
    if (lm_steps(cfg, prm.n, &why) != MPC_OK) return lm_fail(nullptr, MPC_ERR_INVALID_ARG, "%s", why.c_str());
    for (int l = 0; l < cfg->n_landmarks; ++l) prm.alpha[l] = cfg->alpha[l];
    for (int j = 0; j < cfg->q_dim; ++j) prm.w[j] = cfg->q_weight[j];
    int depth = 1;
    while (depth <= cfg->horizon * cfg->ticks_per_stage) depth <<= 1;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return lm_fail(nullptr, MPC_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (cfg->device < 0 || cfg->device >= ndev) return lm_fail(nullptr, MPC_ERR_INVALID_ARG, "bad device ordinal %d", cfg->device);
    if ((e = cudaSetDevice(cfg->device)) != cudaSuccess) return lm_fail(nullptr, MPC_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    mpc_landmarks* lm = new (std::nothrow) mpc_landmarks();
    if (!lm) return lm_fail(nullptr, MPC_ERR_OOM, "host allocation failed");
    lm->cfg = *cfg;
    lm->prm = prm;
    lm->depth = depth;
    const size_t slots = (size_t)cfg->B_max * cfg->n_landmarks * depth;
    if (cudaMalloc(&lm->ticks, slots * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&lm->vals, slots * cfg->q_dim * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&lm->start, (size_t)cfg->B_max * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        mpc_landmark_destroy(lm);
        return lm_fail(nullptr, MPC_ERR_OOM, "cudaMalloc of the landmark rings (%zu slots) failed", slots);
    }
    lm_fill_kernel<<<256, 256>>>(lm->ticks, slots, kEmpty);
    lm_fill_kernel<<<64, 256>>>(lm->start, (size_t)cfg->B_max, kEmpty);
    if ((e = cudaMemset(lm->vals, 0, slots * cfg->q_dim * sizeof(float))) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        mpc_landmark_destroy(lm);
        return lm_fail(nullptr, MPC_ERR_CUDA, "landmark ring initialisation: %s", cudaGetErrorString(e));
    }
    *out = lm;
    return MPC_OK;
}

mpc_status mpc_landmark_store(mpc_landmarks* lm, int64_t tick, const float* xi, int32_t B, void* stream) {
    if (!lm) return MPC_ERR_INVALID_ARG;
    const mpc_landmark_config& c = lm->cfg;
    if (!xi) return lm_fail(lm, MPC_ERR_INVALID_ARG, "null trajectory pointer");
    if (B < 1 || B > c.B_max) return lm_fail(lm, MPC_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, c.B_max);
    if (tick == kEmpty) return lm_fail(lm, MPC_ERR_INVALID_ARG, "tick INT64_MIN is reserved");
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return lm_cuda(lm, e, "cudaSetDevice");
    const int n = B * c.n_landmarks;
    lm_store_kernel<<<(n + 127) / 128, 128, 0, as_stream(stream)>>>(xi, B, c.horizon, c.nx, c.q_index, c.q_dim,
                                                                   c.n_landmarks, lm->prm, c.ticks_per_stage, tick,
                                                                   lm->depth, lm->ticks, lm->vals);
    if ((e = cudaGetLastError()) != cudaSuccess) return lm_cuda(lm, e, "landmark store launch");
    return MPC_OK;
}

mpc_status mpc_landmark_store_solution(mpc_landmarks* lm, mpc_handle* h, int64_t tick, void* stream) {
    if (!lm) return MPC_ERR_INVALID_ARG;
    const float* xi = nullptr;
    int B = 0, N = 0, nx = 0, dev = 0;
    if (!pinmpc::solution_trajectory(h, &xi, &B, &N, &nx, &dev))
        return lm_fail(lm, MPC_ERR_STATE, "the solver handle has no solution");
    const mpc_landmark_config& c = lm->cfg;
    if (N != c.horizon || nx != c.nx || dev != c.device)
        return lm_fail(lm, MPC_ERR_INVALID_ARG, "solution N=%d nx=%d device %d does not match horizon=%d nx=%d device %d",
                       N, nx, dev, c.horizon, c.nx, c.device);
    return mpc_landmark_store(lm, tick, xi, B, stream);
}

mpc_status mpc_landmark_reward(mpc_landmarks* lm, int64_t tick, const float* q_now, float* reward, float* err,
                               int32_t* count, int32_t B, void* stream) {
    if (!lm) return MPC_ERR_INVALID_ARG;
    const mpc_landmark_config& c = lm->cfg;
    if (!q_now || !reward) return lm_fail(lm, MPC_ERR_INVALID_ARG, "null q_now or reward pointer");
    if (B < 1 || B > c.B_max) return lm_fail(lm, MPC_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, c.B_max);
    if (tick == kEmpty) return lm_fail(lm, MPC_ERR_INVALID_ARG, "tick INT64_MIN is reserved");
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return lm_cuda(lm, e, "cudaSetDevice");
    const float inv_sigma2 = 1.0f / (c.sigma * c.sigma);
    lm_reward_kernel<<<(B + 127) / 128, 128, 0, as_stream(stream)>>>(
        B, c.n_landmarks, c.q_dim, lm->prm, c.ticks_per_stage, tick, lm->depth, lm->ticks, lm->vals, lm->start, q_now,
        inv_sigma2, reward, err, count);
    if ((e = cudaGetLastError()) != cudaSuccess) return lm_cuda(lm, e, "landmark reward launch");
    return MPC_OK;
}

mpc_status mpc_landmark_reset(mpc_landmarks* lm, int64_t tick, const uint8_t* mask, int32_t B, void* stream) {
    if (!lm) return MPC_ERR_INVALID_ARG;
    const mpc_landmark_config& c = lm->cfg;
    if (!mask) return lm_fail(lm, MPC_ERR_INVALID_ARG, "null mask pointer");
    if (B < 1 || B > c.B_max) return lm_fail(lm, MPC_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, c.B_max);
    if (tick == kEmpty) return lm_fail(lm, MPC_ERR_INVALID_ARG, "tick INT64_MIN is reserved");
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return lm_cuda(lm, e, "cudaSetDevice");
    lm_reset_kernel<<<(B + 127) / 128, 128, 0, as_stream(stream)>>>(B, mask, tick, lm->start);
    if ((e = cudaGetLastError()) != cudaSuccess) return lm_cuda(lm, e, "landmark reset launch");
    return MPC_OK;
}

const char* mpc_landmark_last_error(mpc_landmarks* lm) { return lm ? lm->error.c_str() : g_lm_create_error.c_str(); }

void mpc_landmark_destroy(mpc_landmarks* lm) {
    if (!lm) return;
    cudaSetDevice(lm->cfg.device);
    cudaDeviceSynchronize();
    cudaFree(lm->ticks);
    cudaFree(lm->vals);
    cudaFree(lm->start);
    cudaGetLastError();
    delete lm;
}

}  // extern "C"
