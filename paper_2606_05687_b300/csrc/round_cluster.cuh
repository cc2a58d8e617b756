// ADMM round for horizons above 32 stages: a thread-block cluster of two
// CTAs per instance, one warp per stage in each.  The iteration is the one
// of round2_kernel (Sec. III's three blocks in the factored form, fast ADMM
// with restart); only the placement differs.  CTA r of the pair holds the
// global stages [k0, k0 + nloc) of the instance's horizon Nh (the first
// ceil(Nh/2) in CTA 0, the rest in CTA 1) with their records, factors and
// iterate in its own shared memory.  The horizon coupling crosses the split
// at one place in each block:
//   block 1 of CTA 1's first stage reads the iterate of stage k0 - 1,
//   block 2 of CTA 0's last stage reads xibar of stage k0,
// both from the other CTA's shared memory (distributed shared memory), and
// the combined residual of the acceleration sums both CTAs' stage shares.
// The two CTA barriers of each iteration become cluster barriers, which
// order those shared-memory accesses across the pair.
//
// Every cluster barrier is reached by all threads of both CTAs: the pair
// takes the same instances in the same order (CTA 0 draws each from the
// round's cursor and writes it, with the action to take, into both CTAs'
// shared memory), and every branch around a barrier depends only on values
// both CTAs read identically.
#pragma once
#include "admm.cuh"

namespace pinmpc {

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Barrier over every thread of the cluster; shared-memory writes before it
// (release) are visible to the other CTA after it (acquire).
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Generic address of the same shared-memory location in CTA `rank` of the cluster.
template <class T>
__device__ __forceinline__ T* cluster_peer(T* p, uint32_t rank) {
    uint64_t out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
    return reinterpret_cast<T*>(out);
}

// Largest horizon of the two-CTA form: 32 stages per CTA.
constexpr int kClusterMaxN = 64;

// One round (a.m0, a.m1] of one instance by CTA `rank` of the pair; NL is the
// local stage capacity ceil(cap / 2).  The instance's horizon Nh (1..cap)
// was checked by the caller.
template <class D, int MAXT, bool BOX>
__device__ __forceinline__ void round_instance_cl(const RoundArgs& a, int b, float* smem, uint32_t rank, int NL) {
    constexpr int NX = D::NX, NU = D::NU, NB = D::NB, NBP = D::NBP, FR = RoundSmem<D>::FR;
    constexpr bool TWO = RegT<D>::kTwo;
    const RoundSmem<D> L(NL, false);
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const float* rec = a.rec + (size_t)b * a.irec;
    const float* tail = rec + (size_t)a.n_rec * D::SREC;
    const int Nh = __float_as_int(__ldg(tail + D::tH));
    const int n0 = (Nh + 1) / 2;  // stages of CTA 0
    const int k0 = rank ? n0 : 0, nloc = rank ? Nh - n0 : n0;
    RCtx<D> c;
    c.var = smem + L.var; c.xb = smem + L.xb; c.tmp = smem + L.tmp; c.pre = smem + L.pre;
    c.fac = smem + L.fac; c.part = smem + L.part;
    c.N = NL; c.Nh = Nh; c.rho = a.rho;
    c.k0 = k0; c.nloc = nloc; c.pjl = n0 - 1;
    c.pvar = cluster_peer(c.var, rank ^ 1u);
    c.pxb = cluster_peer(c.xb, rank ^ 1u);
    const float* ppre = cluster_peer(c.pre, rank ^ 1u);
    const float* ppart = cluster_peer(c.part, rank ^ 1u);
    float* sd = smem + L.sd;
    {
        const float4* src = reinterpret_cast<const float4*>(rec + (size_t)k0 * D::SREC);
        float4* dst = reinterpret_cast<float4*>(sd);
        for (int e = tid; e < nloc * D::SREC / 4; e += nthr) dst[e] = __ldg(src + e);
    }
    // xibar_0 (fixed) belongs to CTA 0; CTA 1's xb[0] is xibar_{k0}, written by block 1
    for (int i = tid; i < NBP; i += nthr)
        c.xb[i] = (rank == 0 && i < NB) ? (i < NX ? __ldg(tail + D::tXI0 + i) : __ldg(tail + D::tUP + i - NX)) : 0.0f;
    for (int e = NBP + tid; e < (NL + 1) * NBP; e += nthr) c.xb[e] = 0.0f;
    for (int e = tid; e < NL * RoundSmem<D>::kTmp * NBP; e += nthr) c.tmp[e] = 0.0f;
    __syncthreads();
    auto stage = [&](int k) { return sd + k * D::SREC; };
    auto mask = [&](int k) { return __float_as_uint(stage(k)[D::oMASK]); };
    float* gcache = a.cache + (size_t)b * RoundSmem<D>::cache_floats(a.N);
    float* gstate = a.state + (size_t)b * RoundState<D>::floats(a.N);
    const int nvar = RoundState<D>::var_floats(a.N);
    for (int e = tid; e < nloc * NBP; e += nthr) {
        const int k = e / NBP, i = e % NBP;
        const float* sk = stage(k);
        float qb = 0.0f, idp = 0.0f, idn = 0.0f;
        if (i < NX) {
            qb = sk[D::oQ + i] * sk[D::oRY + i];
            idp = idn = 1.0f / (sk[D::oQ + i] + a.rho);
        } else if (i < NB) {
            qb = sk[D::oR + i - NX] * sk[D::oRU + i - NX];
            idp = 1.0f / (sk[D::oR + i - NX] + 2.0f * a.rho);
            idn = 1.0f / (sk[D::oR + i - NX] + a.rho);
        }
        c.pre[(k * 3 + PQB) * NBP + i] = qb;
        c.pre[(k * 3 + PID) * NBP + i] = idp;
        c.pre[(k * 3 + PIDN) * NBP + i] = idn;
    }
    {
        const float4* fs = reinterpret_cast<const float4*>(gcache + (size_t)k0 * 2 * NX * FR);
        float4* fd = reinterpret_cast<float4*>(c.fac);
        for (int e = tid; e < nloc * 2 * NX * FR / 4; e += nthr) fd[e] = fs[e];
    }
    const bool warm = a.m0 == 0 && b < a.warm_B;
    const int lvar = 5 * NBP * nloc;  // floats of this CTA's stages in one buffer
    if (a.m0 == 0) {
        if (!warm) {
            for (int e = tid; e < RoundState<D>::var_floats(NL); e += nthr) c.var[e] = 0.0f;
            // stages past the horizon start (and stay) zero, as in the one-CTA form
            for (int e = tid; rank == 0 && e < 2 * (a.N - Nh) * 5 * NBP; e += nthr) {
                const int bf = e / ((a.N - Nh) * 5 * NBP), r = e % ((a.N - Nh) * 5 * NBP);
                gstate[RoundState<D>::at(a.N, bf, Nh, 0) + r] = 0.0f;
            }
        }
        if (rank == 0) {
            for (int e = tid; e < a.N * D::NC; e += nthr) a.lastm[(size_t)b * a.N * D::NC + e] = 0xffffffffu;
            if constexpr (BOX)
                for (int e = tid; e < a.N; e += nthr) a.slast[(size_t)b * a.N + e] = 0xffffffffu;
            if (tid == 0) {
                a.out_npol[b] = 0;
                a.out_piv[b] = 0;
            }
        }
    }
    if (a.m0 > 0 || warm) {
        for (int buf = 0; buf < 2; ++buf) {
            const float4* src = reinterpret_cast<const float4*>(gstate + RoundState<D>::at(a.N, buf, k0, 0));
            float4* dst = reinterpret_cast<float4*>(c.var + RoundState<D>::at(NL, buf, 0, 0));
            for (int e = tid; e < lvar / 4; e += nthr) dst[e] = src[e];
        }
    }
    // both CTAs' constants and iterates are in place
    cluster_barrier();
    const int j = warp < nloc ? warp : 0;
    RegT<D> M;
    StageRegs<D> R;
    {
        const float* sj = stage(j);
        auto Tm = [&](int r, int col) { return col < NX ? sj[D::oA + r * NX + col] : sj[D::oB + r * NU + col - NX]; };
        const int r = lane >> 1, h = lane & 1;
#pragma unroll
        for (int rr = 0; rr < NX; ++rr) {
            M.colA[rr] = (lane < NB) ? Tm(rr, lane) : 0.0f;
            if constexpr (TWO) M.colB[rr] = (32 + lane < NB) ? Tm(rr, 32 + lane) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < D::CS; ++q) {
            const int col = h * D::CS + q;
            M.rowT[q] = (r < NX && col < NB) ? Tm(r, col) : 0.0f;
        }
        R.e0 = lane < NX ? sj[D::oE + lane] : 0.0f;
        // constants of global stage k0 + j - 1 (the other CTA's last stage for CTA 1's first)
        const bool remote = rank == 1 && j == 0;
        const float* pb = remote ? ppre : c.pre;
        const int jp = remote ? c.pjl : (j >= 1 ? j - 1 : 0);
        const float* pq = pb + (jp * 3 + PQB) * NBP;
        const float* pd = pb + (jp * 3 + PID) * NBP;
        R.qbp[0] = lane < NB ? pq[lane] : 0.0f;
        R.idp[0] = lane < NB ? pd[lane] : 0.0f;
        R.qbp[1] = (TWO && lane < NB - 32) ? pq[32 + lane] : 0.0f;
        R.idp[1] = (TWO && lane < NB - 32) ? pd[32 + lane] : 0.0f;
        const int q = lane < D::NC ? lane : 0;
        R.mu = sj[D::oMU + q];
        R.fmx = sj[D::oFM + q];
        R.ir1 = 1.0f / (1.0f + R.mu * R.mu);
        R.ir2 = 1.0f / (1.0f + 2.0f * R.mu * R.mu);
        R.stance = (mask(j) >> q) & 1u;
        R.mw = 0u;
        if constexpr (BOX) load_box<D>(a, b, k0 + j, lane, R);
    }
    __syncthreads();
    // Abar_0 xibar_0 is constant (global stage 0); the other stages form theirs every iteration
    {
        const float ar = prod_T<D>(M, c.xb, lane);
        const float axs = __shfl_sync(0xffffffffu, ar, (2 * lane) & 31);
        R.ax[0] = lane < NX ? axs : (lane < NB ? c.xb[lane] : 0.0f);
        R.ax[1] = (TWO && lane < NB - 32) ? c.xb[32 + lane] : 0.0f;
    }
    float alpha = 1.0f, cprev = INFINITY, wgt = 0.0f;
    bool restart = false;
    int cb = 0;
    if (a.m0 > 0 || warm) {
        const float* sc = gstate + nvar;
        alpha = sc[RoundState<D>::sAlpha];
        cprev = sc[RoundState<D>::sCprev];
        wgt = sc[RoundState<D>::sWgt];
        restart = sc[RoundState<D>::sRestart] != 0.0f;
        cb = __float_as_int(sc[RoundState<D>::sCb]);
    }
    const bool active = warp < nloc;
    // the stage shares of CTA 0 and CTA 1, summed in that order by both CTAs
    const float* part0 = rank == 0 ? c.part : ppart;
    const float* part1 = rank == 0 ? ppart : c.part;
    const int nl1 = Nh - n0;
    for (int m = a.m0 + 1; m <= a.m1; ++m) {
        const float wa = restart ? 0.0f : 1.0f + wgt, wb = restart ? 1.0f : -wgt;
        if (active) {
            load_hats<D>(c, R, cb, j, lane, wa, wb);
            block1_r<D, true>(c, M, R, cb, j, lane, wa, wb);
        }
        cluster_barrier();
        if (active) {
            const float cm = block2_r<D, true, BOX>(c, R, cb, j, lane, a.dx, a.dy);
            if (lane == 0) c.part[j] = cm;
        }
        cluster_barrier();
        const float t0 = warp_sum(lane < n0 ? part0[lane] : 0.0f);
        const float t1 = warp_sum(lane < nl1 ? part1[lane] : 0.0f);
        const float tot = (t0 + t1) * a.rho;
        if (a.accel) {
            if (tot < a.eta * cprev) {
                const float an = 0.5f * (1.0f + sqrtf(1.0f + 4.0f * alpha * alpha));
                wgt = (alpha - 1.0f) / an;
                alpha = an;
                cprev = tot;
                restart = false;
            } else {
                alpha = 1.0f;
                wgt = 0.0f;
                restart = true;
                cprev = cprev / a.eta;
            }
        }
        cb = 1 - cb;
    }
    for (int buf = 0; buf < 2; ++buf) {
        const float4* src = reinterpret_cast<const float4*>(c.var + RoundState<D>::at(NL, buf, 0, 0));
        float4* dst = reinterpret_cast<float4*>(gstate + RoundState<D>::at(a.N, buf, k0, 0));
        for (int e = tid; e < lvar / 4; e += nthr) dst[e] = src[e];
    }
    if (active && lane < D::NC && a.m1 > a.m0) a.modes[((size_t)b * a.N + k0 + j) * D::NC + lane] = R.mw;
    if constexpr (BOX)
        if (active && a.m1 > a.m0) store_box_bits<D>(a, b, k0 + j, lane, R, c.var + RoundState<D>::at(NL, cb, j, VZ));
    if (rank == 0 && tid == 0) {
        float* sc = gstate + nvar;
        sc[RoundState<D>::sAlpha] = alpha;
        sc[RoundState<D>::sCprev] = cprev;
        sc[RoundState<D>::sWgt] = wgt;
        sc[RoundState<D>::sRestart] = restart ? 1.0f : 0.0f;
        sc[RoundState<D>::sCb] = __int_as_float(cb);
    }
}

// Persistent pairs: grid = 2 x pairs, block = 32 ceil(cap / 2) threads
// (MAXT at least that), dynamic shared memory RoundSmem<D>(ceil(cap / 2)),
// cap = a.cap: the longest horizon the launch takes.
template <class D, int MAXT, bool BOX = false>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(MAXT, 1) round_cl_kernel(RoundArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int item[2];  // instance (or -1: no work left) and the action for it
    const uint32_t rank = cluster_rank();
    const int cap = a.cap;
    const int NL = (cap + 1) / 2;
    int* peer_item = cluster_peer(item, rank ^ 1u);
    for (;;) {
        // both CTAs are done with the previous instance, including each
        // other's shared memory
        cluster_barrier();
        if (rank == 0 && threadIdx.x == 0) {
            const int i = atomicAdd(a.cursor, 1);
            const int n = a.list_in ? *a.cnt_in : a.B;
            const int b = (i < n) ? (a.list_in ? a.list_in[i] : i) : -1;
            // 0 iterate, 1 skip (already final), else the failure status to report
            int act = 0;
            if (b >= 0) {
                const float* tail = a.rec + (size_t)b * a.irec + (size_t)a.n_rec * D::SREC;
                const int Nh = __float_as_int(tail[D::tH]);
                if (a.done[b]) {
                    act = 1;
                } else if (Nh < 1 || Nh > cap) {
                    act = 2 + kBadHorizon;
                } else if (a.m0 == 0 && a.flags[b]) {
                    act = 2 + ((a.flags[b] & 1) ? kNonFinite : ((a.flags[b] & 4) ? kBadDim : kBadSet));
                }
            }
            item[0] = b;
            item[1] = act;
            peer_item[0] = b;
            peer_item[1] = act;
        }
        cluster_barrier();
        const int b = item[0], act = item[1];
        if (b < 0) break;
        if (act == 0) round_instance_cl<D, MAXT, BOX>(a, b, smem, rank, NL);
        else if (act >= 2 && rank == 0) round_fail<D>(a, b, act - 2);
    }
}

}  // namespace pinmpc
