// mpc_solve_noalloc: the pack + solve path with its scratch in a fixed,
// library-owned device array, for callers that must not allocate.
//
// Who needs this: code that runs where device allocation is off limits --
// inside a captured CUDA graph replayed by someone else, inside an RL
// simulator step that owns a fixed memory pool and forbids cudaMalloc on its
// hot path, or a real-time control loop that has to avoid the allocator's
// locks and page mapping.  Such callers still own and pass every input and
// output buffer; only the solver's internal scratch (the packed per-instance
// records, the active-face bits and the polish counters) is needed, and that
// lives here in a static __device__ array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/pinmpc.h"
#include "solve.cuh"

using namespace pinmpc;

namespace {

// 8 MiB of scratch, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchFloats = size_t(2) << 20;
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device
bool g_attr_done[kMaxDevices][2] = {};    // dynamic shared-memory opt-in done, per device and shape
thread_local std::string g_noalloc_error;

mpc_status fail(mpc_status st, const std::string& msg) {
    g_noalloc_error = msg;
    return st;
}

// Device memory of `device` (or managed memory): a buffer of another GPU
// would be read across the interconnect, or fault without peer access.
bool is_device_pointer(const void* p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == device) || at.type == cudaMemoryTypeManaged;
}

template <class D>
mpc_status run(const mpc_config& c, const mpc_stage_view& v, float* xi, float* u, int32_t* status,
               int32_t* iters, float* kkt, cudaStream_t s, int shape_index) {
    const int N = v.N, B = v.B;
    const size_t irec = (size_t)instance_record_floats(D::SREC, D::TAIL, N);
    // scratch layout: records [B][irec] | active bits [B][N] (2 floats each) | polish counts [B]
    const size_t need = (size_t)B * irec + (size_t)B * N * 2 + (size_t)B;
    if (need > kScratchFloats)
        return fail(MPC_ERR_UNSUPPORTED,
                    "batch needs " + std::to_string(need * 4) + " B of scratch; the fixed scratch holds " +
                        std::to_string(kScratchFloats * 4) + " B (about " +
                        std::to_string(kScratchFloats / (irec + 2 * N + 1)) + " instances at N=" + std::to_string(N) + ")");
    const int smem = Smem<D>(N).bytes();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MPC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(MPC_ERR_UNSUPPORTED, "device ordinal beyond 63");
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MPC_ERR_CUDA, "cudaDeviceGetAttribute failed");
    }
    if (smem > optin)
        return fail(MPC_ERR_UNSUPPORTED, "N=" + std::to_string(N) + " needs " + std::to_string(smem) +
                                             " B of shared memory per CTA (limit " + std::to_string(optin) + ")");
    float* scratch = nullptr;
    {
        // one-time set-up per device, with that device current: the device
        // address of the static array (host code only has a host-side stand-in
        // for its name) and the kernel's shared-memory opt-in
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(MPC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<float*>(p);
        }
        if (!g_attr_done[dev][shape_index]) {
            e = cudaFuncSetAttribute(solve_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Smem<D>(32).bytes() < optin ? Smem<D>(32).bytes() : optin);
            if (e != cudaSuccess)
                return fail(MPC_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
            g_attr_done[dev][shape_index] = true;
        }
        scratch = g_scratch_ptr[dev];
    }
    float* rec = scratch;
    unsigned long long* bits = reinterpret_cast<unsigned long long*>(scratch + (size_t)B * irec);
    int* npol = reinterpret_cast<int*>(scratch + (size_t)B * irec + (size_t)B * N * 2);

    PackArgs pa{};
    pa.A = v.A; pa.Bm = v.Bm; pa.e = v.e; pa.Q = v.Q; pa.R = v.R; pa.ry = v.ry; pa.ru = v.ru;
    pa.mu = v.mu; pa.fmax = v.fmax; pa.xi0 = v.xi0; pa.u_prev = v.u_prev; pa.mask = v.mask;
    pa.horizon = v.horizon;
    pa.C = v.C;
    pa.N = N;
    pa.S = v.stage_stride ? v.stage_stride : N;
    pa.n_rec = N;
    pa.irec = (int)irec;
    pa.sigma = c.u_scale;
    pa.rec = rec;
    pack_kernel<D><<<B, 256, 0, s>>>(pa);  // rewrites every record word the solve reads
    SolveArgs a{};
    a.rec = rec; a.irec = (int)irec; a.N = N;
    a.rho = c.rho; a.sigma = c.u_scale; a.kkt_tol = c.kkt_tol; a.eta = c.restart_eta;
    a.dx = c.foot_half_length; a.dy = c.foot_half_width;
    a.max_iter = c.max_iter; a.check_start = c.check_start; a.check_every = c.check_every;
    a.polish = c.polish; a.accel = c.accel; a.refine_steps = c.refine_steps; a.refine_alpha = c.refine_alpha;
    a.out_xi = xi; a.out_u = u; a.out_status = status; a.out_iters = iters; a.out_kkt = kkt;
    a.out_bits = bits; a.out_npol = npol;
    solve_kernel<D><<<B, 32 * N, smem, s>>>(a, N);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MPC_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return MPC_OK;
}

}  // namespace

extern "C" {

mpc_status mpc_solve_noalloc(const mpc_config* cfg, const mpc_stage_view* v, float* xi, float* u,
                             int32_t* status, int32_t* iters, float* kkt, void* stream) {
    g_noalloc_error.clear();
    if (!cfg || !v || !xi || !u || !status || !iters || !kkt)
        return fail(MPC_ERR_INVALID_ARG, "null config, view or output pointer");
    const mpc_config& c = *cfg;
    if (!(c.rho > 0.0f) || !(c.u_scale > 0.0f) || !(c.kkt_tol > 0.0f) || c.max_iter < 1 || c.check_every < 1 ||
        c.check_start < 1 || !(c.restart_eta > 0.0f && c.restart_eta < 1.0f) || c.refine_steps < 0 ||
        !(c.refine_alpha > 0.0f))
        return fail(MPC_ERR_INVALID_ARG, "invalid solver parameter");
    if (v->nu) return fail(MPC_ERR_UNSUPPORTED, "the no-allocation solver takes every input (nu must be NULL)");
    if (v->xlo || v->xhi) return fail(MPC_ERR_UNSUPPORTED, "the no-allocation solver takes no state boxes");
    if (v->stage_stride != 0 && v->stage_stride < v->N)
        return fail(MPC_ERR_INVALID_ARG, "stage_stride below N");
    if (c.kkt_tol_abs != 0.0f && c.kkt_tol_abs != c.kkt_tol)
        return fail(MPC_ERR_UNSUPPORTED, "the no-allocation solver certifies with kkt_tol_abs = kkt_tol only");
    if (c.precision != MPC_PREC_FP32)
        return fail(MPC_ERR_UNSUPPORTED, "the no-allocation solver runs FP32 only (precision must be MPC_PREC_FP32)");
    if (v->B < 1 || v->N < 1 || v->N > 32) return fail(MPC_ERR_INVALID_ARG, "B must be >= 1 and N in [1, 32]");
    if (!v->A || !v->Bm || !v->Q || !v->R || !v->ry || !v->mu || !v->fmax || !v->mask || !v->xi0)
        return fail(MPC_ERR_INVALID_ARG, "a required stage array is NULL");
    const void* ptrs[] = {v->A, v->Bm, v->e, v->Q, v->R, v->ry, v->ru, v->mu, v->fmax, v->mask, v->xi0,
                          v->u_prev, v->horizon, v->C, xi, u, status, iters, kkt};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MPC_ERR_CUDA, "no current CUDA device");
    }
    for (const void* p : ptrs)
        if (p && !is_device_pointer(p, dev))
            return fail(MPC_ERR_INVALID_ARG,
                        "every buffer must be device memory of the current device (staging host data would allocate)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c.nx == 13 && c.contact_dim == 3 && c.n_contacts == 8)
        return run<Dims<13, 24, 3>>(c, *v, xi, u, status, iters, kkt, s, 0);
    if (c.nx == 13 && c.contact_dim == 6 && c.n_contacts == 2)
        return run<Dims<13, 12, 6>>(c, *v, xi, u, status, iters, kkt, s, 1);
    return fail(MPC_ERR_UNSUPPORTED, "shape not built (built: 13/8/3, 13/2/6)");
}

const char* mpc_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

}  // extern "C"
