// ADMM round kernel with register-resident stage matrices.
//
// Same iteration as block1/block2 in solve.cuh (Sec. III, the closed-form
// horizon-parallel updates in the factored form described there), one CTA
// per instance and one warp per stage, but each warp keeps its stage's
// T_j = [A_j B_j], S_j and W_j in registers in two layouts:
//   column layout: lane c holds column c (and 32 + c) of T   -> T' x products
//   row layout:    lanes 2r, 2r+1 hold halves of row r of T,
//                  S and W                                   -> T x, S x, W x
// so every product is a short register dot product over vectors read from
// shared memory as broadcast float4, plus one shuffle for the row halves.
// The Nesterov-extrapolated values are formed where they are read.
#pragma once
#include "polish.cuh"

namespace pinmpc {

template <class D>
struct RegT {
    static constexpr int NX = D::NX, NB = D::NB, CS = D::CS, SS = 8;
    float colA[NX];  // column lane of T
    float colB[NX];  // column 32 + lane of T (0 where it does not exist)
    float rowT[CS];  // row lane/2 of T, columns [(lane&1) CS, (lane&1) CS + CS)
    float rowS[SS];  // row lane/2 of S_j, columns [(lane&1) 8, ... + 8)
    float rowW[SS];  // row lane/2 of W_j
    static_assert(NX <= 16, "row split of S and W assumes nx <= 16");
};

// y_r = sum_c T[r][c] x[c]; x has finite padding up to 2 CS.  Valid in lanes 2r, 2r+1.
template <class D>
__device__ __forceinline__ float prod_T(const RegT<D>& M, const float* x, int lane) {
    const float4* x4 = reinterpret_cast<const float4*>(x + (lane & 1) * D::CS);
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int q = 0; q < D::CS / 4; ++q) {
        const float4 v = x4[q];
        a0 = fmaf(M.rowT[4 * q + 0], v.x, a0);
        a1 = fmaf(M.rowT[4 * q + 1], v.y, a1);
        a0 = fmaf(M.rowT[4 * q + 2], v.z, a0);
        a1 = fmaf(M.rowT[4 * q + 3], v.w, a1);
    }
    const float acc = a0 + a1;
    return acc + __shfl_xor_sync(0xffffffffu, acc, 1);
}

// y_r = sum_c R[r][c] x[c] for R = S_j or W_j (rows split 8 + 8); x has finite padding to 16.
__device__ __forceinline__ float prod_R(const float (&row)[8], const float* x, int lane) {
    const float4* x4 = reinterpret_cast<const float4*>(x + (lane & 1) * 8);
    const float4 v0 = x4[0], v1 = x4[1];
    float a0 = row[0] * v0.x, a1 = row[1] * v0.y;
    a0 = fmaf(row[2], v0.z, a0);
    a1 = fmaf(row[3], v0.w, a1);
    a0 = fmaf(row[4], v1.x, a0);
    a1 = fmaf(row[5], v1.y, a1);
    a0 = fmaf(row[6], v1.z, a0);
    a1 = fmaf(row[7], v1.w, a1);
    const float acc = a0 + a1;
    return acc + __shfl_xor_sync(0xffffffffu, acc, 1);
}

// (y_lane, y_{32+lane}) with y_c = sum_r T[r][c] x[r]; x holds NX entries.
template <class D>
__device__ __forceinline__ float2 prod_Tt(const RegT<D>& M, const float* x) {
    constexpr int NX = D::NX;
    const float4* x4 = reinterpret_cast<const float4*>(x);
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int q = 0; q < (NX + 3) / 4; ++q) {
        const float4 v = x4[q];
        const float xv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int r = 4 * q + t;
            if (r < NX) {
                a0 = fmaf(M.colA[r], xv[t], a0);
                a1 = fmaf(M.colB[r], xv[t], a1);
            }
        }
    }
    return make_float2(a0, a1);
}

// per-stage constant vectors kept in shared memory: qbar, 1/D' (k < N-1 form), 1/D (last stage form)
enum : int { PQB = 0, PID = 1, PIDN = 2 };

template <class D>
struct Ctx2 {
    float *var, *xb, *ax, *bdu, *tmp, *pre, *sd, *part;
    uint32_t* modes;
    int N, Nh;
    float rho, dx, dy, wgt;
    bool restart;
    int cb;
    __device__ const float* stage(int k) const { return sd + k * D::SREC; }
    __device__ float* V(int buf, int which, int j) const { return var + ((buf * 5 + which) * N + j) * D::NBP; }
    __device__ float* T(int j, int t) const { return tmp + (j * Smem<D>::kTmpVecs + t) * D::NBP; }
    __device__ float* P(int j, int t) const { return pre + (j * 3 + t) * D::NBP; }
    __device__ uint32_t mask(int k) const { return __float_as_uint(stage(k)[D::oMASK]); }
    // extrapolated (hatted) value of variable `which` of stage j, element i
    __device__ float hat(int which, int j, int i) const {
        const float c = V(cb, which, j)[i], p = V(1 - cb, which, j)[i];
        return restart ? p : fmaf(wgt, c - p, c);
    }
};

// Block 1 of stage j (warp j): du_j (B du into bdu[0, NX), du into bdu[NX, NB)),
// xibar_j = H_{j-1} htilde_{j-1} (factored), Abar_j xibar_j, and xibar_N for the last stage.
template <class D>
__device__ void block1_reg(const Ctx2<D>& c, const RegT<D>& M, int j, int lane) {
    constexpr int NX = D::NX, NB = D::NB;
    const float rho = c.rho;
    const int r = lane >> 1, h = lane & 1;
    const bool rowlane = (r < NX) && (h == 0);
    float* om = c.T(j, 0);
    float* gv = c.T(j, 1);
    float* pv = c.T(j, 2);
    float* sv = c.T(j, 3);
    float* bdu = c.bdu + j * D::NBP;
    const int c0 = lane, c1 = 32 + lane;
    // omega = vhat - betahat
    for (int i = lane; i < NB; i += 32) om[i] = c.hat(VV, j, i) - c.hat(VBE, j, i);
    __syncwarp();
    // g = B' omega_x + omega_u on the input columns (0 on the state columns)
    const float2 tg = prod_Tt<D>(M, om);
    const float g0 = (c0 >= NX && c0 < NB) ? tg.x + om[c0] : 0.0f;
    const float g1 = (c1 < NB) ? tg.y + om[c1] : 0.0f;
    if (c0 < NB) gv[c0] = g0;
    if (c1 < NB) gv[c1] = g1;
    __syncwarp();
    // p = B g ; s = S p (= B du)
    const float pr = prod_T<D>(M, gv, lane);
    if (rowlane) pv[r] = pr;
    __syncwarp();
    const float sr = prod_R(M.rowS, pv, lane);
    if (rowlane) {
        sv[r] = sr;
        bdu[r] = sr;
    }
    __syncwarp();
    // du = g - B' s
    const float2 bs = prod_Tt<D>(M, sv);
    if (c0 >= NX && c0 < NB) bdu[c0] = g0 - bs.x;
    if (c1 < NB) bdu[c1] = g1 - bs.y;
    if (j >= 1) {
        float* wx = c.T(j, 4);
        float* cp = c.T(j, 5);
        const float* sj = c.stage(j);
        const float* qb = c.P(j - 1, PQB);
        const float* idp = c.P(j - 1, PID);
        // w = zhat_{j+1} - vhat_j - ebar_j + lambdahat_j ; c' = D'^{-1}(qbar + rho(zhat_j - thetahat_{j-1}) + rho [0; w_u])
        for (int i = lane; i < NB; i += 32) {
            const float wi = c.hat(VZ, j, i) - c.hat(VV, j, i) - (i < NX ? sj[D::oE + i] : 0.0f) + c.hat(VLA, j, i);
            float cc = qb[i] + rho * (c.hat(VZ, j - 1, i) - c.hat(VTH, j - 1, i));
            if (i >= NX) cc = fmaf(rho, wi, cc);
            else wx[i] = wi;
            cp[i] = cc * idp[i];
        }
        __syncwarp();
        // t = T c' - w_x ; sigma = W t
        const float tr = prod_T<D>(M, cp, lane) - ((r < NX) ? wx[r] : 0.0f);
        __syncwarp();
        if (rowlane) pv[r] = tr;
        __syncwarp();
        const float sg = prod_R(M.rowW, pv, lane);
        __syncwarp();
        if (rowlane) om[r] = sg;
        __syncwarp();
        // xibar_j = c' - D'^{-1} T' sigma
        const float2 ts = prod_Tt<D>(M, om);
        float* xbj = c.xb + j * D::NBP;
        if (c0 < NB) xbj[c0] = fmaf(-idp[c0], ts.x, cp[c0]);
        if (c1 < NB) xbj[c1] = fmaf(-idp[c1], ts.y, cp[c1]);
        __syncwarp();
        // Abar_j xibar_j
        const float ar = prod_T<D>(M, xbj, lane);
        float* axj = c.ax + j * D::NBP;
        if (rowlane) axj[r] = ar;
        if (c0 >= NX && c0 < NB) axj[c0] = xbj[c0];
        if (c1 < NB) axj[c1] = xbj[c1];
    }
    if (j == c.Nh - 1) {
        float* xbN = c.xb + c.Nh * D::NBP;
        const float* qb = c.P(j, PQB);
        const float* idn = c.P(j, PIDN);
        for (int i = lane; i < NB; i += 32)
            xbN[i] = (qb[i] + rho * (c.hat(VZ, j, i) - c.hat(VTH, j, i))) * idn[i];
    }
    __syncwarp();
}

// Block 2 and the dual ascents of stage j; new values go to buffer 1 - cb.
template <class D>
__device__ void block2_reg(const Ctx2<D>& c, int j, int lane) {
    constexpr int NX = D::NX, NB = D::NB, CD = D::CD;
    const int nb = 1 - c.cb;
    const float* sj = c.stage(j);
    const float* xbn = c.xb + (j + 1) * D::NBP;
    const float* axj = c.ax + j * D::NBP;
    const float* bdu = c.bdu + j * D::NBP;
    float* arg = c.T(j, 0);
    float* zp = c.T(j, 1);
    float zh[2], vh[2], th[2], bh[2], lh[2], gam[2];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
        const int i = lane + 32 * s2;
        if (i < NB) {
            zh[s2] = c.hat(VZ, j, i);
            vh[s2] = c.hat(VV, j, i);
            th[s2] = c.hat(VTH, j, i);
            bh[s2] = c.hat(VBE, j, i);
            lh[s2] = c.hat(VLA, j, i);
            const float eb = i < NX ? sj[D::oE + i] : 0.0f;
            const float g_ = bdu[i] + bh[s2] - axj[i] - eb + lh[s2];
            const float gt_ = xbn[i] + th[s2] + axj[i] + eb - lh[s2];
            arg[i] = (2.0f * gt_ + g_) * (1.0f / 3.0f);
            gam[s2] = g_;
        } else {
            zh[s2] = vh[s2] = th[s2] = bh[s2] = lh[s2] = gam[s2] = 0.0f;
        }
    }
    __syncwarp();
    if (lane < NX) zp[lane] = arg[lane];
    if (lane < D::NC) {
        const int q = lane;
        uint32_t mw;
        if ((c.mask(j) >> q) & 1u) {
            mw = project_contact<CD>(arg + NX + q * CD, zp + NX + q * CD, sj[D::oMU + q], sj[D::oFM + q], c.dx, c.dy);
        } else {
            for (int i = 0; i < CD; ++i) zp[NX + q * CD + i] = 0.0f;
            mw = kSwingBit;
        }
        c.modes[j * D::NC + q] = mw;
    }
    __syncwarp();
    float* zn = c.V(nb, VZ, j);
    float* vn = c.V(nb, VV, j);
    float* tn = c.V(nb, VTH, j);
    float* bn = c.V(nb, VBE, j);
    float* ln = c.V(nb, VLA, j);
    float cm = 0.0f;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
        const int i = lane + 32 * s2;
        if (i < NB) {
            const float eb = i < NX ? sj[D::oE + i] : 0.0f;
            const float z = zp[i];
            const float v = 0.5f * (z + gam[s2]);
            const float th_ = th[s2] + xbn[i] - z;
            const float be_ = bh[s2] + bdu[i] - v;
            const float la_ = lh[s2] + z - axj[i] - v - eb;
            zn[i] = z;
            vn[i] = v;
            tn[i] = th_;
            bn[i] = be_;
            ln[i] = la_;
            const float d1 = th_ - th[s2], d2 = be_ - bh[s2], d3 = la_ - lh[s2];
            const float d4 = z - zh[s2], d5 = v - vh[s2], d6 = d4 - d5;
            cm += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
        }
    }
    cm = warp_sum(cm);
    if (lane == 0) c.part[j] = cm;
}

// One round of ADMM iterations (CTA per instance, warp per stage) with the
// caches and the iterate kept in global memory between rounds.
template <class D, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) round2_kernel(RoundArgs a) {
    extern __shared__ __align__(16) float smem[];
    constexpr int NX = D::NX, NU = D::NU, NB = D::NB;
    const int b = blockIdx.x;
    if (a.done[b]) return;
    const Smem<D> L(a.N);
    Ctx<D> c;  // setup helpers (records, caches)
    c.sd = smem + L.sd; c.Sm = smem + L.Sm; c.Wm = smem + L.Wm; c.var = smem + L.var;
    c.hat = smem + L.hat; c.xb = smem + L.xb; c.ax = smem + L.ax; c.bdu = smem + L.bdu;
    c.tmp = smem + L.tmp; c.Kst = smem + L.Kst; c.wk = smem + L.wk; c.xr = smem + L.xr;
    c.ur = smem + L.ur; c.y = smem + L.y; c.wv = smem + L.wv; c.red = smem + L.red;
    c.part = smem + L.part; c.res = smem + L.res;
    c.modes = reinterpret_cast<uint32_t*>(smem + L.modes);
    c.lastm = reinterpret_cast<uint32_t*>(smem + L.lastm);
    c.N = a.N;
    c.rho = a.rho; c.sigma = a.sigma; c.dx = a.dx; c.dy = a.dy;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const float* rec = a.rec + (size_t)b * a.irec;
    const float* tail = rec + (size_t)a.n_rec * D::SREC;
    const int Nh = __float_as_int(tail[D::tH]);
    c.Nh = (Nh >= 1 && Nh <= a.N) ? Nh : 0;
    SolveArgs wa{};
    wa.N = a.N; wa.out_xi = a.out_xi; wa.out_u = a.out_u; wa.out_status = a.out_status;
    wa.out_iters = a.out_iters; wa.out_kkt = a.out_kkt; wa.out_bits = a.out_bits; wa.out_npol = a.out_npol;
    if (c.Nh == 0) {
        write_output<D>(c, wa, b, kBadHorizon, 0, 0.0f, 0);
        if (tid == 0) a.done[b] = 1;
        return;
    }
    {
        const float4* src = reinterpret_cast<const float4*>(rec);
        float4* dst = reinterpret_cast<float4*>(c.sd);
        const int n4 = c.Nh * D::SREC / 4;
        for (int e = tid; e < n4; e += nthr) dst[e] = src[e];
    }
    float* x0 = c.xb;
    for (int i = tid; i < D::NBP; i += nthr) x0[i] = i < NX ? tail[D::tXI0 + i] : (i < NB ? tail[D::tUP + i - NX] : 0.0f);
    float* gcache = a.cache + (size_t)b * a.N * 2 * NX * NX;
    float* gstate = a.state + (size_t)b * RoundState<D>::floats(a.N);
    const int nvar = RoundState<D>::var_floats(a.N);
    // vectors read as float4 must have finite padding: clear the scratch, xb, ax, bdu areas
    for (int e = tid; e < a.N * Smem<D>::kTmpVecs * D::NBP; e += nthr) c.tmp[e] = 0.0f;
    for (int e = D::NBP + tid; e < (a.N + 1) * D::NBP; e += nthr) c.xb[e] = 0.0f;
    for (int e = tid; e < a.N * D::NBP; e += nthr) { c.ax[e] = 0.0f; c.bdu[e] = 0.0f; }
    __syncthreads();
    if (a.m0 == 0) {
        bool bad = false, badset = false;
        for (int e = tid; e < c.Nh * D::SREC; e += nthr) {
            const int off = e % D::SREC;
            if (off < D::oMASK && !isfinite(c.sd[e])) bad = true;
        }
        for (int i = tid; i < NB; i += nthr) if (!isfinite(x0[i])) bad = true;
        for (int e = tid; e < c.Nh * D::NC; e += nthr) {
            const int k = e / D::NC, q = e % D::NC;
            if (((c.mask(k) >> q) & 1u) && (c.stage(k)[D::oMU + q] < 0.0f || c.stage(k)[D::oFM + q] < 0.0f)) badset = true;
        }
        const bool any_bad = __syncthreads_or(bad);
        const bool any_badset = __syncthreads_or(badset);
        if (any_bad || any_badset) {
            write_output<D>(c, wa, b, any_bad ? kNonFinite : kBadSet, 0, 0.0f, 0);
            if (tid == 0) a.done[b] = 1;
            return;
        }
        if (warp < c.Nh) {
            const int j = warp;
            const float* sj = c.stage(j);
            float* Sj = c.Sm + j * NX * NX;
            for (int e = lane; e < NX * NX; e += 32) {
                const int r = e / NX, cc = e % NX;
                float acc = (r == cc) ? 1.0f : 0.0f;
                for (int i = 0; i < NU; ++i) acc = fmaf(sj[D::oB + r * NU + i], sj[D::oB + cc * NU + i], acc);
                Sj[e] = acc;
            }
            __syncwarp();
            warp_inverse_spd(Sj, NX, lane);
            if (j >= 1) {
                const float* sp = c.stage(j - 1);
                float* Wj = c.Wm + j * NX * NX;
                for (int e = lane; e < NX * NX; e += 32) {
                    const int r = e / NX, cc = e % NX;
                    float acc = (r == cc) ? 1.0f / a.rho : 0.0f;
                    for (int i = 0; i < NX; ++i)
                        acc = fmaf(sj[D::oA + r * NX + i] * sj[D::oA + cc * NX + i], 1.0f / (sp[D::oQ + i] + a.rho), acc);
                    for (int i = 0; i < NU; ++i)
                        acc = fmaf(sj[D::oB + r * NU + i] * sj[D::oB + cc * NU + i], 1.0f / (sp[D::oR + i] + 2.0f * a.rho), acc);
                    Wj[e] = acc;
                }
                __syncwarp();
                warp_inverse_spd(Wj, NX, lane);
            }
            for (int e = lane; e < NX * NX; e += 32) {
                gcache[(j * 2 + 0) * NX * NX + e] = Sj[e];
                if (j >= 1) gcache[(j * 2 + 1) * NX * NX + e] = c.Wm[j * NX * NX + e];
            }
        }
        for (int e = tid; e < nvar; e += nthr) c.var[e] = 0.0f;
        for (int e = tid; e < a.N * D::NC; e += nthr) {
            a.lastm[(size_t)b * a.N * D::NC + e] = 0xffffffffu;
            c.modes[e] = 0u;
        }
        if (tid == 0) a.out_npol[b] = 0;
    } else {
        for (int e = tid; e < c.Nh * 2 * NX * NX; e += nthr) {
            const int j = e / (2 * NX * NX), r = e % (2 * NX * NX);
            (r < NX * NX ? c.Sm + j * NX * NX + r : c.Wm + j * NX * NX + (r - NX * NX))[0] = gcache[e];
        }
        const float4* src = reinterpret_cast<const float4*>(gstate);
        float4* dst = reinterpret_cast<float4*>(c.var);
        for (int e = tid; e < nvar / 4; e += nthr) dst[e] = src[e];
    }
    // per-stage constants: qbar, 1/D' = 1/(Q+rho | R+2rho), 1/D = 1/(Q+rho | R+rho)
    float* pre = c.hat;  // the hat area is free: extrapolated values are formed where read
    for (int e = tid; e < c.Nh * D::NBP; e += nthr) {
        const int k = e / D::NBP, i = e % D::NBP;
        const float* sk = c.stage(k);
        float qb = 0.0f, idp = 0.0f, idn = 0.0f;
        if (i < NX) {
            qb = sk[D::oQ + i] * sk[D::oRY + i];
            idp = idn = 1.0f / (sk[D::oQ + i] + a.rho);
        } else if (i < NB) {
            qb = sk[D::oR + i - NX] * sk[D::oRU + i - NX];
            idp = 1.0f / (sk[D::oR + i - NX] + 2.0f * a.rho);
            idn = 1.0f / (sk[D::oR + i - NX] + a.rho);
        }
        pre[(k * 3 + PQB) * D::NBP + i] = qb;
        pre[(k * 3 + PID) * D::NBP + i] = idp;
        pre[(k * 3 + PIDN) * D::NBP + i] = idn;
    }
    // Abar_0 xibar_0 (constant)
    if (warp == 0) {
        const float* s0 = c.stage(0);
        if (lane < NX) {
            float acc = 0.0f;
            for (int cc = 0; cc < NX; ++cc) acc = fmaf(s0[D::oA + lane * NX + cc], x0[cc], acc);
            for (int i = 0; i < NU; ++i) acc = fmaf(s0[D::oB + lane * NU + i], x0[NX + i], acc);
            c.ax[lane] = acc;
        }
        for (int i = NX + lane; i < NB; i += 32) c.ax[i] = x0[i];
    }
    __syncthreads();
    // stage matrices into registers
    RegT<D> M;
    {
        const int j = warp < c.Nh ? warp : 0;
        const float* sj = c.stage(j);
        auto Tm = [&](int r, int col) { return col < NX ? sj[D::oA + r * NX + col] : sj[D::oB + r * NU + col - NX]; };
        const int r = lane >> 1, h = lane & 1;
#pragma unroll
        for (int rr = 0; rr < NX; ++rr) {
            M.colA[rr] = (lane < NB) ? Tm(rr, lane) : 0.0f;
            M.colB[rr] = (32 + lane < NB) ? Tm(rr, 32 + lane) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < D::CS; ++q) {
            const int col = h * D::CS + q;
            M.rowT[q] = (r < NX && col < NB) ? Tm(r, col) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int col = h * 8 + q;
            M.rowS[q] = (r < NX && col < NX) ? c.Sm[j * NX * NX + r * NX + col] : 0.0f;
            M.rowW[q] = (r < NX && col < NX && j >= 1) ? c.Wm[j * NX * NX + r * NX + col] : 0.0f;
        }
    }
    Ctx2<D> c2;
    c2.var = c.var; c2.xb = c.xb; c2.ax = c.ax; c2.bdu = c.bdu; c2.tmp = c.tmp; c2.pre = pre;
    c2.sd = c.sd; c2.part = c.part; c2.modes = c.modes;
    c2.N = a.N; c2.Nh = c.Nh; c2.rho = a.rho; c2.dx = a.dx; c2.dy = a.dy;
    float alpha = 1.0f, cprev = INFINITY;
    c2.wgt = 0.0f;
    c2.restart = false;
    c2.cb = 0;
    if (a.m0 > 0) {
        const float* sc = gstate + nvar;
        alpha = sc[RoundState<D>::sAlpha];
        cprev = sc[RoundState<D>::sCprev];
        c2.wgt = sc[RoundState<D>::sWgt];
        c2.restart = sc[RoundState<D>::sRestart] != 0.0f;
        c2.cb = __float_as_int(sc[RoundState<D>::sCb]);
    }
    for (int m = a.m0 + 1; m <= a.m1; ++m) {
        if (warp < c.Nh) block1_reg<D>(c2, M, warp, lane);
        __syncthreads();
        if (warp < c.Nh) block2_reg<D>(c2, warp, lane);
        __syncthreads();
        float tot = 0.0f;
        for (int j = 0; j < c.Nh; ++j) tot += c.part[j];
        tot *= a.rho;
        if (a.accel) {
            if (tot < a.eta * cprev) {
                const float an = 0.5f * (1.0f + sqrtf(1.0f + 4.0f * alpha * alpha));
                c2.wgt = (alpha - 1.0f) / an;
                alpha = an;
                cprev = tot;
                c2.restart = false;
            } else {
                alpha = 1.0f;
                c2.wgt = 0.0f;
                c2.restart = true;
                cprev = cprev / a.eta;
            }
        }
        c2.cb = 1 - c2.cb;
    }
    __syncthreads();
    {
        const float4* src = reinterpret_cast<const float4*>(c.var);
        float4* dst = reinterpret_cast<float4*>(gstate);
        for (int e = tid; e < nvar / 4; e += nthr) dst[e] = src[e];
    }
    for (int e = tid; e < c.Nh * D::NC; e += nthr) a.modes[(size_t)b * a.N * D::NC + e] = c.modes[e];
    if (tid == 0) {
        float* sc = gstate + nvar;
        sc[RoundState<D>::sAlpha] = alpha;
        sc[RoundState<D>::sCprev] = cprev;
        sc[RoundState<D>::sWgt] = c2.wgt;
        sc[RoundState<D>::sRestart] = c2.restart ? 1.0f : 0.0f;
        sc[RoundState<D>::sCb] = __int_as_float(c2.cb);
    }
}

}  // namespace pinmpc
