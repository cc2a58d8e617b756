// Per-instance solver state between a handle's slots and a caller-owned
// store (the receding-horizon warm start of one environment across batches
// that place it in different slots).  The state is RoundState<D>: both
// buffers of the ADMM iterate (z, v, theta, beta, lambda), stage-major, then
// the acceleration scalars and the current-buffer index.
#pragma once
#include "polish.cuh"

namespace pinmpc {

// One CTA per row: row didx[b] (b when didx is null) of dst receives row
// sidx[b] (b) of src with its stages moved `shift` towards the start of the
// horizon Nh (the last stage repeated into the freed tail; Nh from slot b's
// record when rec is given, else N) and the acceleration restarted (alpha 1,
// no previous residual).  A row with a non-finite entry (its solve failed)
// arrives as zeros: that instance starts cold.  The current-buffer index is
// copied as 0 or 1 whatever the source holds.
// Indices are checked against the row counts: a source row outside
// [0, src_rows) arrives as a cold start, a destination row outside
// [0, dst_rows) is not written.
template <class D>
__global__ void state_copy_kernel(const float* src, const int* sidx, int src_rows, float* dst, const int* didx,
                                  int dst_rows, const float* rec, int irec, int n_rec, int N, int shift) {
    extern __shared__ __align__(16) float csm[];
    const int b = blockIdx.x;
    const int si = sidx ? sidx[b] : b, di = didx ? didx[b] : b;
    if (di < 0 || di >= dst_rows) return;
    const size_t stride = RoundState<D>::floats(N);
    const bool have_src = si >= 0 && si < src_rows;
    const float* s = src + (size_t)(have_src ? si : 0) * stride;
    float* d = dst + (size_t)di * stride;
    const int nvar = RoundState<D>::var_floats(N);
    int Nh = N;
    if (rec) {
        const int Nh0 = __float_as_int(__ldg(rec + (size_t)b * irec + (size_t)n_rec * D::SREC + D::tH));
        Nh = (Nh0 >= 1 && Nh0 <= N) ? Nh0 : N;
    }
    bool bad = !have_src;
    for (int e = threadIdx.x; e < nvar; e += blockDim.x) {
        csm[e] = have_src ? s[e] : 0.0f;
        bad |= !isfinite(csm[e]);
    }
    const bool cold = __syncthreads_or(bad);
    constexpr int SV = 5 * D::NBP;  // floats of one stage in one buffer
    for (int e = threadIdx.x; e < nvar; e += blockDim.x) {
        const int buf = e / (N * SV), r = e % (N * SV), j = r / SV, o = r % SV;
        const int from = min(j + shift, Nh - 1);
        d[e] = cold ? 0.0f : (j < Nh ? csm[(buf * N + from) * SV + o] : csm[e]);
    }
    if (threadIdx.x == 0) {
        const float* ss = s + nvar;
        float* sd = d + nvar;
        for (int i = 0; i < (int)(stride - nvar); ++i) sd[i] = have_src ? ss[i] : 0.0f;
        // the current-buffer index selects one of two buffers: anything but 1 reads as 0
        sd[RoundState<D>::sCb] = __int_as_float(have_src && __float_as_int(ss[RoundState<D>::sCb]) == 1 ? 1 : 0);
        sd[RoundState<D>::sAlpha] = 1.0f;
        sd[RoundState<D>::sCprev] = INFINITY;
        sd[RoundState<D>::sWgt] = 0.0f;
        sd[RoundState<D>::sRestart] = 0.0f;
    }
}

}  // namespace pinmpc
