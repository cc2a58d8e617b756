// Host side of the C ABI declared in include/pinmpc.h.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pinmpc.h"
#include "admm.cuh"
#include "polish_cta.cuh"
#include "round_cluster.cuh"
#include "internal.h"
#include "warm_state.cuh"

using namespace pinmpc;

namespace {

// Shapes the library is compiled for: (nx, nu, contact_dim).
using D24 = Dims<13, 24, 3>;  // 8 point contacts (4 corners per foot)
using D12 = Dims<13, 12, 6>;  // 2 foot wrenches
// the 9-state centroidal model xi = [c, l_G, k_G] with the same contact models
using C24 = Dims<9, 24, 3>;
using C12 = Dims<9, 12, 6>;

thread_local std::string g_create_error;

struct Shape {
    int srec, tail;
    void (*launch_pack)(const PackArgs&, int B, cudaStream_t);
    int (*polish_smem)(int N);
    int (*state_floats)(int N);
    cudaError_t (*set_round_attrs)(int round_bytes, int polish_bytes);
    void (*launch_round)(const RoundArgs&, int B, int smem, cudaStream_t);
    void (*launch_polish)(const RoundArgs&, int B, int smem, cudaStream_t);
    int (*round_smem)(int N, bool dbl);
    int (*cache_floats)(int N);
    void (*launch_factor)(const FactorArgs&, cudaStream_t);
    int (*resident_per_sm)(int kernel, int N, int smem);  // kernel 0 round, 1 polish
    void (*launch_warm_shift)(float* state, const float* rec, int irec, int n_rec, int B, int N, int shift,
                              cudaStream_t s);
    cudaError_t (*set_warm_attr)(int bytes);
    void (*launch_state_copy)(const float* src, const int* sidx, int src_rows, float* dst, const int* didx, int dst_rows,
                              const float* rec, int irec, int n_rec, int B, int N, int shift, cudaStream_t s);
    cudaError_t (*set_state_copy_attr)(int bytes);
    void (*launch_bin)(const RoundArgs&, int B, cudaStream_t);
};

template <class D>
void launch_pack_t(const PackArgs& a, int B, cudaStream_t s) { pack_kernel<D><<<B, 256, 0, s>>>(a); }
template <class D>
int polish_smem_t(int N) { return CtaSmem<D>(N).total * 4; }
template <class D>
int state_floats_t(int N) { return RoundState<D>::floats(N); }
// above 32 stages the round runs as CTA pairs, each holding ceil(N/2) stages
template <class D>
int round_smem_t(int N, bool dbl) { return N > 32 ? RoundSmem<D>((N + 1) / 2, false).bytes() : RoundSmem<D>(N, dbl).bytes(); }
template <class D>
int cache_floats_t(int N) { return RoundSmem<D>::cache_floats(N); }
template <class D>
void launch_factor_t(const FactorArgs& a, cudaStream_t s) {
    const int warps = a.B * a.N;
    const int grid = (warps + kFactorWarps - 1) / kFactorWarps;
    if (a.precision == kPrecTF32) factor_kernel<D, kPrecTF32><<<grid, 32 * kFactorWarps, 0, s>>>(a);
    else if (a.precision == kPrecBF16) factor_kernel<D, kPrecBF16><<<grid, 32 * kFactorWarps, 0, s>>>(a);
    else factor_kernel<D><<<grid, 32 * kFactorWarps, 0, s>>>(a);
}
template <class D, bool BOX>
cudaError_t set_round_attrs_b(int round_bytes, int polish_bytes) {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(round2_kernel<D, 640, false, BOX>, attr, round_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(round2_kernel<D, 1024, false, BOX>, attr, round_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(round2_kernel<D, 640, true, BOX>, attr, round_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(round2_kernel<D, 1024, true, BOX>, attr, round_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(round_cl_kernel<D, 640, BOX>, attr, round_bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(round_cl_kernel<D, 1024, BOX>, attr, round_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(polish_cta_kernel<D, BOX>, attr, polish_bytes);
}
template <class D>
cudaError_t set_round_attrs_t(int round_bytes, int polish_bytes) {
    const cudaError_t e = set_round_attrs_b<D, false>(round_bytes, polish_bytes);
    return e != cudaSuccess ? e : set_round_attrs_b<D, true>(round_bytes, polish_bytes);
}
// The round kernel's launch form (the state-box variant when boxes are set).
template <class D, bool BOX>
void launch_round_b(const RoundArgs& a, int B, int smem, cudaStream_t s) {
    // register-heavy form for up to 20 stages per CTA (640 threads), 64-register
    // form above; B persistent workers: CTAs, or CTA pairs above 32 stages.
    // The launch's stage capacity is a.cap (its horizon class's, N for one class).
    const int n = a.cap;
    if (n > 32) {
        const int nl = (n + 1) / 2;
        if (nl <= 20) round_cl_kernel<D, 640, BOX><<<2 * B, 32 * nl, smem, s>>>(a);
        else round_cl_kernel<D, 1024, BOX><<<2 * B, 32 * nl, smem, s>>>(a);
    } else if (n < a.N) {
        // a horizon class below N: CTAs sized for n stages
        if (n <= 20) round2_kernel<D, 640, true, BOX><<<B, 32 * n, smem, s>>>(a);
        else round2_kernel<D, 1024, true, BOX><<<B, 32 * n, smem, s>>>(a);
    } else if (n <= 20) {
        round2_kernel<D, 640, false, BOX><<<B, 32 * n, smem, s>>>(a);
    } else {
        round2_kernel<D, 1024, false, BOX><<<B, 32 * n, smem, s>>>(a);
    }
}
template <class D>
void launch_round_t(const RoundArgs& a, int B, int smem, cudaStream_t s) {
    if (a.xbox) launch_round_b<D, true>(a, B, smem, s);
    else launch_round_b<D, false>(a, B, smem, s);
}
template <class D>
void launch_bin_t(const RoundArgs& a, int B, cudaStream_t s) {
    bin_classes_kernel<D><<<(B + 255) / 256, 256, 0, s>>>(a);
}
template <class D>
void launch_polish_t(const RoundArgs& a, int B, int smem, cudaStream_t s) {
    if (a.xbox) polish_cta_kernel<D, true><<<B, kPT, smem, s>>>(a);
    else polish_cta_kernel<D><<<B, kPT, smem, s>>>(a);
}
template <class D>
int resident_per_sm_t(int kernel, int N, int smem) {
    int n = 0;
    cudaError_t e;
    if (kernel == 0 && N > 32) {
        // one CTA of a pair per SM: its shared memory is above half an SM's
        return 1;
    } else if (kernel == 0) {
        if (N <= 20) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, round2_kernel<D, 640>, 32 * N, smem);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, round2_kernel<D, 1024>, 32 * N, smem);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, polish_cta_kernel<D>, kPT, smem);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n > 0 ? n : 1;
}
template <class D>
void launch_warm_shift_t(float* state, const float* rec, int irec, int n_rec, int B, int N, int shift, cudaStream_t s) {
    warm_shift_kernel<D><<<B, 256, RoundState<D>::var_floats(N) * sizeof(float), s>>>(state, rec, irec, n_rec, N, shift);
}
template <class D>
cudaError_t set_warm_attr_t(int bytes) {
    return cudaFuncSetAttribute(warm_shift_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
template <class D>
void launch_state_copy_t(const float* src, const int* sidx, int src_rows, float* dst, const int* didx, int dst_rows,
                         const float* rec, int irec, int n_rec, int B, int N, int shift, cudaStream_t s) {
    state_copy_kernel<D><<<B, 256, RoundState<D>::var_floats(N) * sizeof(float), s>>>(
        src, sidx, src_rows, dst, didx, dst_rows, rec, irec, n_rec, N, shift);
}
template <class D>
cudaError_t set_state_copy_attr_t(int bytes) {
    return cudaFuncSetAttribute(state_copy_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
template <class D>
Shape make_shape() {
    return Shape{D::SREC,         D::TAIL,           launch_pack_t<D>,     polish_smem_t<D>,     state_floats_t<D>,
                 set_round_attrs_t<D>, launch_round_t<D>, launch_polish_t<D>, round_smem_t<D>,
                 cache_floats_t<D>, launch_factor_t<D>, resident_per_sm_t<D>, launch_warm_shift_t<D>,
                 set_warm_attr_t<D>, launch_state_copy_t<D>, set_state_copy_attr_t<D>, launch_bin_t<D>};
}

bool pick_shape(int nx, int nc, int cd, Shape* out) {
    if (nx == 13 && cd == 3 && nc == 8) { *out = make_shape<D24>(); return true; }
    if (nx == 13 && cd == 6 && nc == 2) { *out = make_shape<D12>(); return true; }
    if (nx == 9 && cd == 3 && nc == 8) { *out = make_shape<C24>(); return true; }
    if (nx == 9 && cd == 6 && nc == 2) { *out = make_shape<C12>(); return true; }
    return false;
}

constexpr int kSmemLimit = 227 * 1024;
// factor on the refinement step from the fifth round on (rounds 0-3 keep the
// configured step): the instances still running there are mostly caught in
// an active-set cycle of the refinement, which the longer step breaks
constexpr float kRefineAlphaLate = 3.0f;

int max_optin_smem(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        cudaGetLastError();
        v = kSmemLimit;
    }
    return v;
}

}  // namespace

struct mpc_handle {
    mpc_config cfg{};
    Shape shape{};
    int nu = 0, nc = 0;
    int irec = 0;          // floats per instance record
    float* rec = nullptr;  // [B_max][irec]
    float* out_xi = nullptr;
    float* out_u = nullptr;
    int* out_status = nullptr;
    int* out_iters = nullptr;
    float* out_kkt = nullptr;
    unsigned long long* out_bits = nullptr;
    int* out_npol = nullptr;
    int* out_piv = nullptr;      // [B_max] free pivots eliminated by the polish
    float* cache = nullptr;      // [B_max][N_max][2][nx][16] S_j, W_j (padded rows)
    float* state = nullptr;      // [B_max][state floats] ADMM iterate between rounds
    uint32_t* modes = nullptr;   // [B_max][N_max][nc]
    uint32_t* lastm = nullptr;   // [B_max][N_max][nc]
    int* done = nullptr;         // [B_max]
    int* flags = nullptr;        // [B_max] input-check bits of the factor kernel
    float* xbox = nullptr;       // [B_max][N_max][2][nx] state boxes of the last set_stages
    uint32_t* smodes = nullptr;  // [B_max][N_max] state bounds of the latest z
    uint32_t* slast = nullptr;   // [B_max][N_max] state bounds of the last polish
    bool box_set = false;        // the last set_stages gave state boxes
    int* lists = nullptr;        // [2][kMaxClasses][B_max] instances still running, by round parity and horizon class
    int* work = nullptr;         // [kMaxClasses] round cursors, then list counts [2][kMaxClasses]
    int ncls_req = 0;            // horizon classes below N (mpc_set_horizon_classes), ascending caps
    int cls_req[kMaxClasses] = {};
    int sms = 0;                 // streaming multiprocessors of the device
    int optin_smem = 0;          // opt-in shared memory per CTA
    int round_attr = 0;          // dynamic shared memory the round kernel is set up for
    int warm_B = 0, warm_N = 0;  // a warm start is pending for instances [0, warm_B) at horizon stride warm_N
    float* Kst = nullptr;        // [B_max][N_max][nu + kNCB][nx+1] polish gains (and bound multiplier gains)
    float* staging = nullptr;  // device copies of host-memory inputs
    // host-input copies run on their own stream: they wait only until the
    // previous pack has read the staging buffer, so they overlap the solve
    // queued before them on the caller's stream
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t staged = nullptr, consumed = nullptr;
    bool consumed_valid = false;
    size_t staging_floats = 0;
    uint64_t bytes = 0;
    int B_set = 0, N_set = 0;
    bool have_stages = false, have_solution = false;
    int B_solved = 0;
    // per-kernel timing (mpc_set_kernel_timing): event pairs recorded around
    // launches, resolved into totals by mpc_get_kernel_times
    struct TimedLaunch {
        int cls;
        cudaEvent_t start, stop;
    };
    bool timing = false;
    // CUDA-graph replay of the solve (mpc_set_graph_mode): the enqueued
    // sequence captured on capture_stream, one executable graph per
    // (B, N, double buffering, warm-start count), most recent last
    struct SolveGraph {
        int B, N, dbl, warm_B;
        bool box;
        cudaGraphExec_t exec;
    };
    bool graph_mode = false;
    std::vector<cudaEvent_t> round_events;  // recorded after each round's polish (mpc_set_round_events)
    cudaStream_t capture_stream = nullptr;
    std::vector<SolveGraph> graphs;
    int64_t graph_captures = 0, graph_replays = 0;
    std::vector<cudaEvent_t> event_pool;
    std::vector<TimedLaunch> pending;
    double kernel_ms[MPC_KERNEL_CLASSES] = {};
    int64_t kernel_launches[MPC_KERNEL_CLASSES] = {};
    std::string err;
};

namespace {

enum : int { kClassPack = 0, kClassFactor = 1, kClassRound = 2, kClassPolish = 3 };

// Waits for the recorded launches, adds their durations to the totals and
// returns their events to the pool.
void resolve_timed(mpc_handle* h) {
    for (const auto& t : h->pending) {
        float ms = 0.0f;
        if (cudaEventSynchronize(t.stop) == cudaSuccess && cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
            h->kernel_ms[t.cls] += ms;
            h->kernel_launches[t.cls] += 1;
        } else {
            cudaGetLastError();
        }
        h->event_pool.push_back(t.start);
        h->event_pool.push_back(t.stop);
    }
    h->pending.clear();
}

bool take_event(mpc_handle* h, cudaEvent_t* ev) {
    if (!h->event_pool.empty()) {
        *ev = h->event_pool.back();
        h->event_pool.pop_back();
        return true;
    }
    if (cudaEventCreate(ev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Launches through `launch` on stream s, bracketed by an event pair when timing is on.
template <class F>
cudaError_t timed_launch(mpc_handle* h, int cls, cudaStream_t s, F&& launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    bool timed = h->timing;
    if (timed && h->pending.size() >= 4096) resolve_timed(h);
    if (timed && !take_event(h, &a)) timed = false;
    if (timed && !take_event(h, &b)) {
        h->event_pool.push_back(a);
        timed = false;
    }
    if (timed && cudaEventRecord(a, s) != cudaSuccess) {
        cudaGetLastError();
        h->event_pool.push_back(a);
        h->event_pool.push_back(b);
        timed = false;
    }
    launch();
    const cudaError_t e = cudaGetLastError();
    if (timed) {
        if (cudaEventRecord(b, s) == cudaSuccess) {
            h->pending.push_back({cls, a, b});
        } else {
            cudaGetLastError();
            h->event_pool.push_back(a);
            h->event_pool.push_back(b);
        }
    }
    return e;
}

}  // namespace

namespace pinmpc {
bool solution_trajectory(const mpc_handle* h, const float** xi, int* B, int* N, int* nx, int* device) {
    if (!h || !h->have_solution) return false;
    *xi = h->out_xi;  // [B_solved][N_set][nx]
    *B = h->B_solved;
    *N = h->N_set;
    *nx = h->cfg.nx;
    *device = h->cfg.device;
    return true;
}
}  // namespace pinmpc

static mpc_status fail(mpc_handle* h, mpc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return st;
}

static mpc_status cuda_fail(mpc_handle* h, cudaError_t e, const char* what) {
    return fail(h, MPC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static bool is_host_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// Device (or managed) memory of `device`: what a kernel of this library may
// dereference directly.
static bool is_device_memory(const void* p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == device) || at.type == cudaMemoryTypeManaged;
}

// Host memory the CUDA runtime does not know (not page-locked): a copy into
// it is complete only once the stream has reached it.
static bool is_pageable_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeUnregistered;
}

// Device bytes mpc_create allocates for cfg (records, outputs, factor cache,
// ADMM state, face words, work lists, polish gains); the host-input staging
// buffer is allocated later, on the first set_stages from host memory.
static uint64_t workspace_bytes_of(const mpc_config& c, const Shape& sh) {
    const size_t B = (size_t)c.B_max, N = (size_t)c.N_max;
    const size_t nc = (size_t)c.n_contacts, nu = nc * (size_t)c.contact_dim;
    const size_t irec = (size_t)instance_record_floats(sh.srec, sh.tail, c.N_max);
    const size_t rec_b = B * irec * sizeof(float);
    const size_t xi_b = B * N * c.nx * sizeof(float), u_b = B * N * nu * sizeof(float);
    const size_t small_b = B * (4 * sizeof(int) + sizeof(float)) + B * N * sizeof(unsigned long long);
    const size_t cache_b = B * (size_t)sh.cache_floats(c.N_max) * sizeof(float);
    const size_t state_b = B * (size_t)sh.state_floats(c.N_max) * sizeof(float);
    const size_t modes_b = B * N * nc * sizeof(uint32_t);
    const size_t kst_b = B * N * (nu + kNCB) * (c.nx + 1) * sizeof(float);  // gains + bound multiplier gains
    const size_t round_b = cache_b + state_b + 2 * modes_b + (2 + 2 * kMaxClasses) * B * sizeof(int) +
                           3 * kMaxClasses * sizeof(int) + kst_b;
    const size_t box_b = B * N * (2 * (size_t)c.nx * sizeof(float) + 2 * sizeof(uint32_t));
    return rec_b + xi_b + u_b + small_b + round_b + box_b;
}

extern "C" {

mpc_status mpc_workspace_estimate(const mpc_config* cfg, uint64_t* bytes) {
    if (!cfg || !bytes) return MPC_ERR_INVALID_ARG;
    Shape sh;
    if (cfg->contact_dim != 3 && cfg->contact_dim != 6) return MPC_ERR_INVALID_ARG;
    if (!pick_shape(cfg->nx, cfg->n_contacts, cfg->contact_dim, &sh)) return MPC_ERR_UNSUPPORTED;
    if (cfg->B_max < 1 || cfg->N_max < 1) return MPC_ERR_INVALID_ARG;
    if (cfg->N_max > kClusterMaxN) return MPC_ERR_UNSUPPORTED;
    *bytes = workspace_bytes_of(*cfg, sh);
    return MPC_OK;
}

mpc_status mpc_default_config(mpc_config* cfg, int32_t nx, int32_t n_contacts, int32_t contact_dim,
                              int32_t B_max, int32_t N_max) {
    if (!cfg) return MPC_ERR_INVALID_ARG;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->nx = nx;
    cfg->n_contacts = n_contacts;
    cfg->contact_dim = contact_dim;
    cfg->B_max = B_max;
    cfg->N_max = N_max;
    cfg->rho = 100.0f;
    cfg->u_scale = 300.0f;
    cfg->max_iter = 1000;
    cfg->kkt_tol = 2e-6f;
    cfg->check_start = 12;
    cfg->check_every = 20;
    cfg->check_growth = 2.0f;
    cfg->polish = 1;
    cfg->accel = 1;
    cfg->restart_eta = 0.999f;
    cfg->refine_steps = 3;
    cfg->refine_alpha = 0.01f;
    cfg->foot_half_length = 0.10f;
    cfg->foot_half_width = 0.05f;
    cfg->mem_budget = 0;
    cfg->device = 0;
    cfg->precision = MPC_PREC_FP32;
    cfg->kkt_tol_abs = 0.0f;
    if (nx == 13 && contact_dim == 6) {
        // foot wrenches on the 13-state model: a stiffer penalty, a later
        // first check and finer, longer refinement (measured: 2.3-6x faster,
        // as many instances certified); the 9-state model keeps the above
        cfg->rho = 300.0f;
        cfg->check_start = 32;
        cfg->refine_steps = 4;
        cfg->refine_alpha = 0.001f;
    }
    return MPC_OK;
}

int32_t mpc_max_horizon(int32_t nx, int32_t nu) {
    Shape sh;
    const int cd = (nu == 24) ? 3 : 6;
    if (nu % cd != 0 || !pick_shape(nx, nu / cd, cd, &sh)) return 0;
    // one warp per stage (32 stages per CTA, CTA pairs above 32) and each
    // kernel's shared memory
    int best = 0;
    for (int N = 1; N <= kClusterMaxN; ++N)
        if (sh.round_smem(N, false) <= kSmemLimit && sh.polish_smem(N) <= kSmemLimit) best = N;
    return best;
}

mpc_status mpc_create(const mpc_config* cfg, mpc_handle** out) {
    g_create_error.clear();
    if (!cfg || !out) return fail(nullptr, MPC_ERR_INVALID_ARG, "null config or output pointer");
    *out = nullptr;
    const mpc_config& c = *cfg;
    Shape sh;
    if (c.contact_dim != 3 && c.contact_dim != 6)
        return fail(nullptr, MPC_ERR_INVALID_ARG, "contact_dim must be 3 or 6 (got %d)", c.contact_dim);
    if (!pick_shape(c.nx, c.n_contacts, c.contact_dim, &sh))
        return fail(nullptr, MPC_ERR_UNSUPPORTED,
                    "shape nx=%d n_contacts=%d contact_dim=%d not built (built: nx 13 or 9 with 8/3 or 2/6)", c.nx,
                    c.n_contacts, c.contact_dim);
    if (c.B_max < 1 || c.N_max < 1) return fail(nullptr, MPC_ERR_INVALID_ARG, "B_max and N_max must be >= 1");
    if (!(c.rho > 0.0f) || !(c.u_scale > 0.0f) || !(c.kkt_tol > 0.0f) || c.max_iter < 1 ||
        c.check_every < 1 || c.check_start < 1 || !(c.check_growth >= 1.0f) || !(c.restart_eta > 0.0f && c.restart_eta < 1.0f) ||
        !(c.foot_half_length >= 0.0f) || !(c.foot_half_width >= 0.0f) || c.refine_steps < 0 ||
        !(c.refine_alpha > 0.0f) || c.precision < MPC_PREC_FP32 || c.precision > MPC_PREC_BF16 ||
        !(c.kkt_tol_abs >= 0.0f))
        return fail(nullptr, MPC_ERR_INVALID_ARG, "invalid solver parameter");
    if (c.N_max > kClusterMaxN)
        return fail(nullptr, MPC_ERR_UNSUPPORTED, "N_max=%d exceeds %d stages (one warp per stage, two CTAs)",
                    c.N_max, kClusterMaxN);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, MPC_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (c.device < 0 || c.device >= ndev) return fail(nullptr, MPC_ERR_INVALID_ARG, "bad device ordinal %d", c.device);
    if ((e = cudaSetDevice(c.device)) != cudaSuccess) return fail(nullptr, MPC_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    if (sh.polish_smem(c.N_max) > max_optin_smem(c.device))
        return fail(nullptr, MPC_ERR_UNSUPPORTED, "N_max=%d: polish needs %d B shared memory", c.N_max,
                    sh.polish_smem(c.N_max));
    if (sh.round_smem(c.N_max, false) > max_optin_smem(c.device))
        return fail(nullptr, MPC_ERR_UNSUPPORTED, "N_max=%d: ADMM rounds need %d B shared memory", c.N_max,
                    sh.round_smem(c.N_max, false));
    if ((e = sh.set_round_attrs(sh.round_smem(c.N_max, false), sh.polish_smem(c.N_max))) != cudaSuccess)
        return fail(nullptr, MPC_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));

    mpc_handle* h = new (std::nothrow) mpc_handle();
    if (!h) return fail(nullptr, MPC_ERR_OOM, "host allocation failed");
    h->cfg = c;
    if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess || h->sms < 1) {
        cudaGetLastError();
        h->sms = 1;
    }
    h->optin_smem = max_optin_smem(c.device);
    h->round_attr = sh.round_smem(c.N_max, false);
    h->shape = sh;
    h->nc = c.n_contacts;
    h->nu = c.n_contacts * c.contact_dim;
    h->irec = instance_record_floats(sh.srec, sh.tail, c.N_max);
    const size_t B = (size_t)c.B_max, N = (size_t)c.N_max;
    const size_t rec_b = B * h->irec * sizeof(float);
    const size_t xi_b = B * N * c.nx * sizeof(float), u_b = B * N * h->nu * sizeof(float);
    const size_t cache_b = B * (size_t)sh.cache_floats(c.N_max) * sizeof(float);
    const size_t state_b = B * (size_t)sh.state_floats(c.N_max) * sizeof(float);
    const size_t modes_b = B * N * h->nc * sizeof(uint32_t);
    const size_t kst_b = B * N * (h->nu + kNCB) * (c.nx + 1) * sizeof(float);  // gains + bound multiplier gains
    h->bytes = workspace_bytes_of(c, sh);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = (size_t)-1; }
    if ((c.mem_budget && h->bytes > c.mem_budget) || h->bytes > free_b) {
        mpc_status st = fail(nullptr, MPC_ERR_OOM, "workspace %llu B exceeds budget %llu B / free %llu B",
                             (unsigned long long)h->bytes, (unsigned long long)c.mem_budget,
                             (unsigned long long)free_b);
        delete h;
        return st;
    }
    bool ok = cudaMalloc(&h->rec, rec_b) == cudaSuccess && cudaMalloc(&h->out_xi, xi_b) == cudaSuccess &&
              cudaMalloc(&h->out_u, u_b) == cudaSuccess && cudaMalloc(&h->out_status, B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->out_iters, B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->out_kkt, B * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&h->out_bits, B * N * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&h->out_npol, B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->out_piv, B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->cache, cache_b) == cudaSuccess && cudaMalloc(&h->state, state_b) == cudaSuccess &&
              cudaMalloc(&h->modes, modes_b) == cudaSuccess && cudaMalloc(&h->lastm, modes_b) == cudaSuccess &&
              cudaMalloc(&h->done, B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->flags, B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->lists, 2 * kMaxClasses * B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&h->work, 3 * kMaxClasses * sizeof(int)) == cudaSuccess && cudaMalloc(&h->Kst, kst_b) == cudaSuccess &&
              cudaMalloc(&h->xbox, B * N * 2 * c.nx * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&h->smodes, B * N * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&h->slast, B * N * sizeof(uint32_t)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        const unsigned long long want = h->bytes;
        mpc_destroy(h);
        return fail(nullptr, MPC_ERR_OOM, "cudaMalloc of the %llu B workspace failed", want);
    }
    *out = h;
    return MPC_OK;
}

mpc_status mpc_set_stages(mpc_handle* h, const mpc_stage_view* v, void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!v) return fail(h, MPC_ERR_INVALID_ARG, "null stage view");
    const mpc_config& c = h->cfg;
    if (v->B < 1 || v->B > c.B_max) return fail(h, MPC_ERR_INVALID_ARG, "B=%d outside [1, B_max=%d]", v->B, c.B_max);
    if (v->N < 1 || v->N > c.N_max) return fail(h, MPC_ERR_INVALID_ARG, "N=%d outside [1, N_max=%d]", v->N, c.N_max);
    if (!v->A || !v->Bm || !v->Q || !v->R || !v->ry || !v->mu || !v->fmax || !v->mask || !v->xi0)
        return fail(h, MPC_ERR_INVALID_ARG, "a required stage array is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (v->stage_stride != 0 && v->stage_stride < v->N)
        return fail(h, MPC_ERR_INVALID_ARG, "stage_stride=%d below N=%d", v->stage_stride, v->N);
    const size_t B = v->B, N = v->N, nx = c.nx, nu = h->nu, nc = h->nc;
    const size_t S = v->stage_stride ? (size_t)v->stage_stride : N;
    // stage arrays span (B - 1) S + N stages (the last instance needs only N)
    const size_t ST = (B - 1) * S + N;
    constexpr int NA = 17;
    const void* src[NA] = {v->A,  v->Bm,   v->e,      v->Q,    v->R,       v->ry, v->ru, v->mu,    v->fmax,
                           v->xi0, v->u_prev, v->mask, v->horizon, v->C, v->nu, v->xlo, v->xhi};
    const size_t cnt[NA] = {ST * nx * nx, ST * nx * nu, ST * nx, ST * nx, ST * nu, ST * nx, ST * nu, ST * nc, ST * nc,
                            B * nx,       B * nu,       ST,      B,       ST * nx, B,       ST * nx, ST * nx};
    const void* dev[NA];
    bool any_host = false;
    for (int i = 0; i < NA; ++i) any_host |= is_host_pointer(src[i]);
    if (any_host) {
        size_t need = 0;
        for (int i = 0; i < NA; ++i) need += src[i] ? ((cnt[i] + 63) & ~size_t(63)) : 0;
        if (need > h->staging_floats) {
            if (h->staging) {
                cudaFree(h->staging);
                h->bytes -= h->staging_floats * 4;
                h->staging = nullptr;
                h->staging_floats = 0;
            }
            if (c.mem_budget && h->bytes + need * 4 > c.mem_budget)
                return fail(h, MPC_ERR_OOM, "host-input staging of %llu B exceeds the memory budget",
                            (unsigned long long)(need * 4));
            if ((e = cudaMalloc(&h->staging, need * 4)) != cudaSuccess) {
                cudaGetLastError();
                return fail(h, MPC_ERR_OOM, "staging cudaMalloc failed");
            }
            h->staging_floats = need;
            h->bytes += need * 4;
        }
        if (!h->copy_stream) {
            if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->staged, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->consumed, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return fail(h, MPC_ERR_CUDA, "copy stream or event creation failed");
            }
        }
        if (h->consumed_valid && (e = cudaStreamWaitEvent(h->copy_stream, h->consumed, 0)) != cudaSuccess)
            return cuda_fail(h, e, "cudaStreamWaitEvent");
        size_t off = 0;
        for (int i = 0; i < NA; ++i) {
            if (!src[i]) { dev[i] = nullptr; continue; }
            if (is_host_pointer(src[i])) {
                float* d = h->staging + off;
                if ((e = cudaMemcpyAsync(d, src[i], cnt[i] * 4, cudaMemcpyHostToDevice, h->copy_stream)) != cudaSuccess)
                    return cuda_fail(h, e, "cudaMemcpyAsync (stage data)");
                dev[i] = d;
            } else {
                dev[i] = src[i];
            }
            off += (cnt[i] + 63) & ~size_t(63);
        }
        if ((e = cudaEventRecord(h->staged, h->copy_stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, h->staged, 0)) != cudaSuccess)
            return cuda_fail(h, e, "staging event");
    } else {
        for (int i = 0; i < NA; ++i) dev[i] = src[i];
    }
    PackArgs a{};
    a.A = (const float*)dev[0]; a.Bm = (const float*)dev[1]; a.e = (const float*)dev[2];
    a.Q = (const float*)dev[3]; a.R = (const float*)dev[4]; a.ry = (const float*)dev[5];
    a.ru = (const float*)dev[6]; a.mu = (const float*)dev[7]; a.fmax = (const float*)dev[8];
    a.xi0 = (const float*)dev[9]; a.u_prev = (const float*)dev[10];
    a.mask = (const uint32_t*)dev[11]; a.horizon = (const int32_t*)dev[12];
    a.C = (const float*)dev[13]; a.nu = (const int32_t*)dev[14];
    a.xlo = (const float*)dev[15]; a.xhi = (const float*)dev[16];
    a.xbox = (v->xlo || v->xhi) ? h->xbox : nullptr;
    a.N = (int)N;
    a.S = (int)S;
    a.n_rec = c.N_max;
    a.irec = h->irec;
    a.sigma = c.u_scale;
    a.rec = h->rec;
    if ((e = timed_launch(h, kClassPack, s, [&] { h->shape.launch_pack(a, (int)B, s); })) != cudaSuccess)
        return cuda_fail(h, e, "pack kernel launch");
    if (any_host) {
        if ((e = cudaEventRecord(h->consumed, s)) != cudaSuccess) return cuda_fail(h, e, "staging event");
        h->consumed_valid = true;
    }
    h->B_set = (int)B;
    h->N_set = (int)N;
    h->box_set = a.xbox != nullptr;
    h->have_stages = true;
    h->have_solution = false;
    return MPC_OK;
}

// Launch form of each horizon class's round kernel: stage capacity, TMA
// double buffering, dynamic shared memory, persistent workers.
struct SolvePlan {
    int ncls;
    struct { int cap, dbl, smem, grid; } cls[kMaxClasses];
};

// The classes of a solve: the requested caps below N, then N itself; each
// class's CTAs hold cap stages (CTA pairs above 32).  Raises the round
// kernels' shared-memory attribute when a class needs more than it allows.
static mpc_status plan_solve(mpc_handle* h, int B, SolvePlan* p) {
    const int N = h->N_set;
    p->ncls = 0;
    for (int i = 0; i < h->ncls_req; ++i)
        if (h->cls_req[i] < N) p->cls[p->ncls++].cap = h->cls_req[i];
    p->cls[p->ncls++].cap = N;
    int need = 0;
    for (int k = 0; k < p->ncls; ++k) {
        auto& q = p->cls[k];
        if (q.cap > 32) {
            q.dbl = 0;
            q.smem = h->shape.round_smem(q.cap, false);
            q.grid = h->sms * h->shape.resident_per_sm(0, q.cap, q.smem) / 2;
        } else {
            const int sd = h->shape.round_smem(q.cap, true);
            q.dbl = sd <= h->optin_smem;
            q.smem = q.dbl ? sd : h->shape.round_smem(q.cap, false);
            q.grid = h->sms * h->shape.resident_per_sm(0, q.cap, q.smem);
        }
        q.grid = std::max(1, std::min(B, q.grid));
        need = std::max(need, q.smem);
    }
    if (need > h->round_attr) {
        cudaError_t e = h->shape.set_round_attrs(need, h->shape.polish_smem(h->cfg.N_max));
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
        h->round_attr = need;
    }
    return MPC_OK;
}

// The solve's device work for instances [0, B) on stream st: flag resets,
// the factor kernel and the whole round schedule (no host synchronisation).
static mpc_status enqueue_solve(mpc_handle* h, int32_t B, RoundArgs r, cudaStream_t st, const SolvePlan& plan) {
    const mpc_config& c = h->cfg;
    cudaError_t e;
    const int polish_smem = h->shape.polish_smem(h->N_set);
    if ((e = cudaMemsetAsync(h->done, 0, (size_t)B * sizeof(int), st)) != cudaSuccess)
        return cuda_fail(h, e, "cudaMemsetAsync");
    if ((e = cudaMemsetAsync(h->flags, 0, (size_t)B * sizeof(int), st)) != cudaSuccess)
        return cuda_fail(h, e, "cudaMemsetAsync");
    // every instance reads MPC_RUNNING (-1) until the round that finishes it
    if ((e = cudaMemsetAsync(h->out_status, 0xff, (size_t)B * sizeof(int), st)) != cudaSuccess)
        return cuda_fail(h, e, "cudaMemsetAsync");
    // the polish keeps its best near-miss point's certificate in kkt (a huge
    // value until there is one: bytes 0x7f are 3.4e38) and a stall count in iters
    if ((e = cudaMemsetAsync(h->out_kkt, 0x7f, (size_t)B * sizeof(float), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(h->out_iters, 0, (size_t)B * sizeof(int), st)) != cudaSuccess)
        return cuda_fail(h, e, "cudaMemsetAsync");
    // per-stage factors and input checks for the whole batch
    {
        FactorArgs fa{};
        fa.rec = h->rec; fa.irec = h->irec; fa.n_rec = c.N_max; fa.N = h->N_set; fa.B = B;
        fa.rho = c.rho; fa.cache = h->cache; fa.flags = h->flags; fa.precision = c.precision;
        if ((e = timed_launch(h, kClassFactor, st, [&] { h->shape.launch_factor(fa, st); })) != cudaSuccess)
            return cuda_fail(h, e, "factor kernel launch");
    }
    // rounds of ADMM iterations, each followed by the polish/certify kernel,
    // all enqueued up front (no host synchronisation): the round kernel's
    // persistent CTAs work through the round's list of running instances and
    // the polish kernel's CTAs index it, so a round with few or no instances
    // left costs one short launch of each kernel
    int* cursor = h->work;             // [kMaxClasses]
    int* cnt = h->work + kMaxClasses;  // [2][kMaxClasses]
    const int K = plan.ncls;
    const size_t LS = (size_t)kMaxClasses * c.B_max;  // one parity's lists
    r.ncls = K;
    r.cls_stride = c.B_max;
    for (int k = 0; k < K; ++k) r.cls_cap[k] = plan.cls[k].cap;
    if (K > 1) {
        // round 0's lists: every instance in its horizon class's list
        RoundArgs rb = r;
        rb.list_out = h->lists;
        rb.cnt_out = cnt;
        if ((e = cudaMemsetAsync(cnt, 0, K * sizeof(int), st)) != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
        if ((e = timed_launch(h, kClassRound, st, [&] { h->shape.launch_bin(rb, B, st); })) != cudaSuccess)
            return cuda_fail(h, e, "class binning launch");
    }
    const int polish_grid = B;
    int m0 = 0, round = 0;
    double interval = c.check_every;
    for (;; ++round) {
        int m1;
        if (m0 == 0) {
            m1 = std::min(c.check_start, c.max_iter);
        } else {
            m1 = (int)std::min<double>((double)m0 + interval, (double)c.max_iter);
            interval *= c.check_growth;
        }
        const int in = round & 1, out = in ^ 1;
        r.m0 = m0;
        r.m1 = m1;
        // round 0 of a single class takes every instance without a list
        r.list_in = (round == 0 && K == 1) ? nullptr : h->lists + in * LS;
        r.cnt_in = cnt + in * kMaxClasses;
        r.list_out = h->lists + out * LS;
        r.cnt_out = cnt + out * kMaxClasses;
        r.cursor = cursor;
        r.warm_B = (h->warm_N == h->N_set) ? std::min(h->warm_B, B) : 0;
        // the few instances left after two rounds get more refinement: the
        // allowance doubles per round from round 2 on (up to 32)
        r.refine_steps = std::min(32, c.refine_steps << std::min(std::max(round - 1, 0), 4));
        // and from round 4 on a longer step, which breaks the refinement's
        // active-set cycles (faces flipped in and out again)
        r.refine_alpha = round >= 4 ? kRefineAlphaLate * c.refine_alpha : c.refine_alpha;
        if ((e = cudaMemsetAsync(cursor, 0, K * sizeof(int), st)) != cudaSuccess ||
            (e = cudaMemsetAsync(r.cnt_out, 0, K * sizeof(int), st)) != cudaSuccess)
            return cuda_fail(h, e, "cudaMemsetAsync");
        // one round kernel launch per horizon class, each on its class's list
        for (int k = 0; k < K; ++k) {
            RoundArgs rk = r;
            rk.cap = plan.cls[k].cap;
            rk.dbl = plan.cls[k].dbl;
            rk.cursor = cursor + k;
            if (r.list_in) {
                rk.list_in = r.list_in + (size_t)k * c.B_max;
                rk.cnt_in = r.cnt_in + k;
            }
            const int grid = plan.cls[k].grid, smem = plan.cls[k].smem;
            if ((e = timed_launch(h, kClassRound, st, [&] { h->shape.launch_round(rk, grid, smem, st); })) != cudaSuccess)
                return cuda_fail(h, e, "round kernel launch");
        }
        if ((e = timed_launch(h, kClassPolish, st, [&] { h->shape.launch_polish(r, polish_grid, polish_smem, st); })) != cudaSuccess)
            return cuda_fail(h, e, "polish kernel launch");
        if (round < (int)h->round_events.size() && h->round_events[round] &&
            (e = cudaEventRecord(h->round_events[round], st)) != cudaSuccess)
            return cuda_fail(h, e, "cudaEventRecord");
        if (m1 >= c.max_iter) break;
        m0 = m1;
    }
    return MPC_OK;
}

mpc_status mpc_solve_batch(mpc_handle* h, int32_t B, void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!h->have_stages) return fail(h, MPC_ERR_STATE, "mpc_solve_batch before mpc_set_stages");
    if (B < 1 || B > h->B_set) return fail(h, MPC_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, h->B_set);
    const mpc_config& c = h->cfg;
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RoundArgs r{};
    r.rec = h->rec; r.irec = h->irec; r.n_rec = c.N_max; r.N = h->N_set;
    r.rho = c.rho; r.sigma = c.u_scale; r.kkt_tol = c.kkt_tol; r.eta = c.restart_eta;
    r.kkt_c = c.kkt_tol_abs > 0.0f ? c.kkt_tol_abs / c.kkt_tol : 1.0f;
    r.dx = c.foot_half_length; r.dy = c.foot_half_width;
    r.max_iter = c.max_iter; r.polish = c.polish; r.accel = c.accel;
    r.refine_steps = c.refine_steps; r.refine_alpha = c.refine_alpha;
    r.cache = h->cache; r.state = h->state; r.modes = h->modes; r.lastm = h->lastm;
    r.done = h->done; r.Kst = h->Kst; r.flags = h->flags; r.B = B;
    r.xbox = h->box_set ? h->xbox : nullptr; r.smodes = h->smodes; r.slast = h->slast;
    r.out_xi = h->out_xi; r.out_u = h->out_u; r.out_status = h->out_status; r.out_iters = h->out_iters;
    r.out_kkt = h->out_kkt; r.out_bits = h->out_bits; r.out_npol = h->out_npol; r.out_piv = h->out_piv;
    // each horizon class's launch form (double-buffered records and factors,
    // TMA prefetch, where they fit)
    SolvePlan plan;
    mpc_status ps = plan_solve(h, B, &plan);
    if (ps != MPC_OK) return ps;
    r.dbl = plan.cls[plan.ncls - 1].dbl;
    r.cap = h->N_set;
    r.warm_B = (h->warm_N == h->N_set) ? std::min(h->warm_B, B) : 0;
    mpc_status ms = MPC_OK;
    if (h->graph_mode && !h->timing) {
        // replay the captured sequence for this key, capturing it first if new
        const int key_dbl = r.dbl;
        auto it = std::find_if(h->graphs.begin(), h->graphs.end(), [&](const mpc_handle::SolveGraph& g) {
            return g.B == B && g.N == h->N_set && g.dbl == key_dbl && g.warm_B == r.warm_B && g.box == h->box_set;
        });
        if (it == h->graphs.end()) {
            if (!h->capture_stream &&
                (e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(h, e, "cudaStreamCreateWithFlags");
            if ((e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(h, e, "cudaStreamBeginCapture");
            ms = enqueue_solve(h, B, r, h->capture_stream, plan);
            cudaGraph_t g = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(h->capture_stream, &g);
            if (ms != MPC_OK) {
                if (g) cudaGraphDestroy(g);
                return ms;
            }
            if (ee != cudaSuccess) return cuda_fail(h, ee, "cudaStreamEndCapture");
            cudaGraphExec_t ex = nullptr;
            e = cudaGraphInstantiate(&ex, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
            if (h->graphs.size() >= 4) {
                cudaGraphExecDestroy(h->graphs.front().exec);
                h->graphs.erase(h->graphs.begin());
            }
            h->graphs.push_back({B, h->N_set, key_dbl, r.warm_B, h->box_set, ex});
            ++h->graph_captures;
            it = h->graphs.end() - 1;
        }
        if ((e = cudaGraphLaunch(it->exec, st)) != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
        ++h->graph_replays;
    } else {
        ms = enqueue_solve(h, B, r, st, plan);
        if (ms != MPC_OK) return ms;
    }
    h->have_solution = true;
    h->B_solved = B;
    h->warm_B = 0;  // a warm start is consumed by one solve
    return MPC_OK;
}

mpc_status mpc_get_traj(mpc_handle* h, float* xi, float* u, int32_t* status, int32_t* iters, float* kkt,
                        uint64_t* active_bits, void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!h->have_solution) return fail(h, MPC_ERR_STATE, "mpc_get_traj before mpc_solve_batch");
    const mpc_config& c = h->cfg;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const size_t B = h->B_solved, N = h->N_set;
    struct { void* dst; const void* src; size_t bytes; } cp[6] = {
        {xi, h->out_xi, B * N * c.nx * 4}, {u, h->out_u, B * N * h->nu * 4}, {status, h->out_status, B * 4},
        {iters, h->out_iters, B * 4}, {kkt, h->out_kkt, B * 4}, {active_bits, h->out_bits, B * N * 8}};
    bool host = false;
    for (auto& x : cp) {
        if (!x.dst) continue;
        host |= is_pageable_pointer(x.dst);
        if ((e = cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyDefault, s)) != cudaSuccess)
            return cuda_fail(h, e, "cudaMemcpyAsync (results)");
    }
    if (host && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    return MPC_OK;
}

mpc_status mpc_get_stats(mpc_handle* h, int32_t* polishes, void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!h->have_solution) return fail(h, MPC_ERR_STATE, "mpc_get_stats before mpc_solve_batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(h->cfg.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (polishes) {
        if ((e = cudaMemcpyAsync(polishes, h->out_npol, (size_t)h->B_solved * 4, cudaMemcpyDefault, s)) != cudaSuccess)
            return cuda_fail(h, e, "cudaMemcpyAsync (stats)");
        if (is_pageable_pointer(polishes) && (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(h, e, "cudaStreamSynchronize");
    }
    return MPC_OK;
}

mpc_status mpc_get_pivots(mpc_handle* h, int32_t* pivots, void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!h->have_solution) return fail(h, MPC_ERR_STATE, "mpc_get_pivots before mpc_solve_batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(h->cfg.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (pivots) {
        if ((e = cudaMemcpyAsync(pivots, h->out_piv, (size_t)h->B_solved * 4, cudaMemcpyDefault, s)) != cudaSuccess)
            return cuda_fail(h, e, "cudaMemcpyAsync (pivots)");
        if (is_pageable_pointer(pivots) && (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(h, e, "cudaStreamSynchronize");
    }
    return MPC_OK;
}

mpc_status mpc_warm_start(mpc_handle* h, int32_t shift, void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!h->have_solution) return fail(h, MPC_ERR_STATE, "mpc_warm_start before mpc_solve_batch");
    if (shift < 0 || shift >= h->N_set) return fail(h, MPC_ERR_INVALID_ARG, "shift=%d outside [0, N=%d)", shift, h->N_set);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(h->cfg.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const int smem = h->shape.state_floats(h->N_set) * (int)sizeof(float);
    if (smem > 48 * 1024 && (e = h->shape.set_warm_attr(smem)) != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
    h->shape.launch_warm_shift(h->state, h->rec, h->irec, h->cfg.N_max, h->B_solved, h->N_set, shift, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "warm-start kernel launch");
    h->warm_B = h->B_solved;
    h->warm_N = h->N_set;
    return MPC_OK;
}

int64_t mpc_state_floats(mpc_handle* h, int32_t N) {
    if (!h || N < 1 || N > h->cfg.N_max) return 0;
    return h->shape.state_floats(N);
}

int64_t mpc_state_floats_estimate(const mpc_config* cfg, int32_t N) {
    Shape sh;
    if (!cfg || N < 1 || N > kClusterMaxN || !pick_shape(cfg->nx, cfg->n_contacts, cfg->contact_dim, &sh)) return 0;
    return sh.state_floats(N);
}

mpc_status mpc_save_state(mpc_handle* h, float* store, const int32_t* idx, int32_t rows, int32_t B, int32_t shift,
                          void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!h->have_solution) return fail(h, MPC_ERR_STATE, "mpc_save_state before mpc_solve_batch");
    if (!store || rows < 1) return fail(h, MPC_ERR_INVALID_ARG, "null store or rows < 1");
    if (B < 1 || B > h->B_solved) return fail(h, MPC_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, h->B_solved);
    if (shift < 0 || shift >= h->N_set) return fail(h, MPC_ERR_INVALID_ARG, "shift=%d outside [0, N=%d)", shift, h->N_set);
    cudaError_t e = cudaSetDevice(h->cfg.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (!is_device_memory(store, h->cfg.device) || (idx && !is_device_memory(idx, h->cfg.device)))
        return fail(h, MPC_ERR_INVALID_ARG, "store and idx must be device memory of the handle's device");
    const int smem = h->shape.state_floats(h->N_set) * (int)sizeof(float);
    if (smem > 48 * 1024 && (e = h->shape.set_state_copy_attr(smem)) != cudaSuccess)
        return cuda_fail(h, e, "cudaFuncSetAttribute");
    h->shape.launch_state_copy(h->state, nullptr, h->B_solved, store, idx, rows, h->rec, h->irec, h->cfg.N_max, B,
                               h->N_set, shift, static_cast<cudaStream_t>(stream));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "state copy launch");
    return MPC_OK;
}

mpc_status mpc_load_state(mpc_handle* h, const float* store, const int32_t* idx, int32_t rows, int32_t B,
                          void* stream) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (!h->have_stages) return fail(h, MPC_ERR_STATE, "mpc_load_state before mpc_set_stages");
    if (!store || rows < 1) return fail(h, MPC_ERR_INVALID_ARG, "null store or rows < 1");
    if (B < 1 || B > h->B_set) return fail(h, MPC_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, h->B_set);
    cudaError_t e = cudaSetDevice(h->cfg.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if (!is_device_memory(store, h->cfg.device) || (idx && !is_device_memory(idx, h->cfg.device)))
        return fail(h, MPC_ERR_INVALID_ARG, "store and idx must be device memory of the handle's device");
    const int smem = h->shape.state_floats(h->N_set) * (int)sizeof(float);
    if (smem > 48 * 1024 && (e = h->shape.set_state_copy_attr(smem)) != cudaSuccess)
        return cuda_fail(h, e, "cudaFuncSetAttribute");
    h->shape.launch_state_copy(store, idx, rows, h->state, nullptr, h->B_set, nullptr, 0, 0, B, h->N_set, 0,
                               static_cast<cudaStream_t>(stream));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "state copy launch");
    h->warm_B = B;
    h->warm_N = h->N_set;
    return MPC_OK;
}

static void drop_graphs(mpc_handle* h) {
    for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

mpc_status mpc_set_round_events(mpc_handle* h, void* const* events, int32_t n) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (n < 0 || n > 64 || (n > 0 && !events)) return fail(h, MPC_ERR_INVALID_ARG, "n=%d outside [0, 64] or null events", n);
    h->round_events.assign(n, nullptr);
    for (int i = 0; i < n; ++i) h->round_events[i] = static_cast<cudaEvent_t>(events[i]);
    cudaSetDevice(h->cfg.device);
    drop_graphs(h);  // captured solves hold the previous events
    return MPC_OK;
}

mpc_status mpc_set_horizon_classes(mpc_handle* h, const int32_t* caps, int32_t n) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (n < 0 || n > kMaxClasses - 1 || (n > 0 && !caps))
        return fail(h, MPC_ERR_INVALID_ARG, "n=%d horizon classes (0..%d, caps required)", n, kMaxClasses - 1);
    for (int i = 0; i < n; ++i)
        if (caps[i] < 1 || caps[i] > h->cfg.N_max || (i > 0 && caps[i] <= caps[i - 1]))
            return fail(h, MPC_ERR_INVALID_ARG, "class caps must ascend within [1, N_max=%d]", h->cfg.N_max);
    h->ncls_req = n;
    for (int i = 0; i < n; ++i) h->cls_req[i] = caps[i];
    drop_graphs(h);  // captured solves hold the previous launch sequence
    return MPC_OK;
}

mpc_status mpc_set_graph_mode(mpc_handle* h, int32_t enable) {
    if (!h) return MPC_ERR_INVALID_ARG;
    h->graph_mode = enable != 0;
    if (!h->graph_mode) {
        cudaSetDevice(h->cfg.device);
        drop_graphs(h);
    }
    return MPC_OK;
}

mpc_status mpc_get_graph_stats(mpc_handle* h, int64_t* captures, int64_t* replays) {
    if (!h) return MPC_ERR_INVALID_ARG;
    if (captures) *captures = h->graph_captures;
    if (replays) *replays = h->graph_replays;
    return MPC_OK;
}

mpc_status mpc_set_kernel_timing(mpc_handle* h, int32_t enable) {
    if (!h) return MPC_ERR_INVALID_ARG;
    h->timing = enable != 0;
    return MPC_OK;
}

mpc_status mpc_get_kernel_times(mpc_handle* h, double* ms, int64_t* launches, int32_t reset) {
    if (!h) return MPC_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->cfg.device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    resolve_timed(h);
    for (int i = 0; i < MPC_KERNEL_CLASSES; ++i) {
        if (ms) ms[i] = h->kernel_ms[i];
        if (launches) launches[i] = h->kernel_launches[i];
        if (reset) {
            h->kernel_ms[i] = 0.0;
            h->kernel_launches[i] = 0;
        }
    }
    return MPC_OK;
}

void mpc_destroy(mpc_handle* h) {
    if (!h) return;
    cudaSetDevice(h->cfg.device);
    cudaDeviceSynchronize();
    for (const auto& t : h->pending) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (cudaEvent_t ev : h->event_pool) cudaEventDestroy(ev);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    drop_graphs(h);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    if (h->staged) cudaEventDestroy(h->staged);
    if (h->consumed) cudaEventDestroy(h->consumed);
    cudaFree(h->out_piv);
    cudaFree(h->rec);
    cudaFree(h->out_xi);
    cudaFree(h->out_u);
    cudaFree(h->out_status);
    cudaFree(h->out_iters);
    cudaFree(h->out_kkt);
    cudaFree(h->out_bits);
    cudaFree(h->out_npol);
    cudaFree(h->cache);
    cudaFree(h->state);
    cudaFree(h->modes);
    cudaFree(h->lastm);
    cudaFree(h->done);
    cudaFree(h->flags);
    cudaFree(h->lists);
    cudaFree(h->work);
    cudaFree(h->Kst);
    cudaFree(h->xbox);
    cudaFree(h->smodes);
    cudaFree(h->slast);
    cudaFree(h->staging);
    cudaGetLastError();
    delete h;
}

const char* mpc_last_error(mpc_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

uint64_t mpc_workspace_bytes(mpc_handle* h) { return h ? h->bytes : 0; }

}  // extern "C"
