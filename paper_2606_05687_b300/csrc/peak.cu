// FP32 FMA throughput of the device (mpc_measure_fma_peak): the measured
// denominator beside the derived SMs x 128 lanes x 2 x clock figure of the
// roofline.  A measurement utility, not part of the solver.
#include <cuda_runtime.h>

#include "../../include/pinmpc.h"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

// Each thread runs kChains independent chains x <- x m + c (|m| < 1 keeps x
// bounded), `iters` steps each, and writes their sum so nothing is dropped.
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(float* out, int iters, float m, float c) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1e-3f * (threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" mpc_status mpc_measure_fma_peak(int32_t device, int32_t iters, double* tflops) {
    if (!tflops || iters < 1) return MPC_ERR_INVALID_ARG;
    *tflops = 0.0;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MPC_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return MPC_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) return MPC_ERR_CUDA;
    const int blocks = sms * kBlocksPerSM;
    float* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mpc_status st = MPC_ERR_CUDA;
    float ms = 0.0f;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return MPC_ERR_OOM;
    }
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        fma_peak_kernel<<<blocks, kThreads>>>(out, iters, 0.9999f, 1e-4f);  // warm-up
        cudaEventRecord(e0);
        fma_peak_kernel<<<blocks, kThreads>>>(out, iters, 0.9999f, 1e-4f);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.0f) {
            const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
            *tflops = flops / (ms * 1e-3) / 1e12;
            st = MPC_OK;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}
