// Warp-per-instance polish, certificate and active-set refinement.
//
// After a round of ADMM iterations (the round kernel below), every instance
// whose active faces changed is polished by ONE warp: the backward Riccati
// scan of the equality-constrained LQR on those faces (reduced inputs
// u = T ut + o, the same algebra as `polish` in solve.cuh), the forward
// rollout, the KKT certificate, and up to `refine_steps` projected-gradient
// face updates.  A warp needs only __syncwarp, so many instances are in
// flight per SM; the 24x24 Cholesky factor and both triangular solves live in
// registers (lane = row) and move data by shuffles.
#pragma once
#include "solve.cuh"

namespace pinmpc {

constexpr int kPolishWarps = 4;  // warps (instances) per CTA of the polish kernel

// Global-memory state of an instance between rounds.
template <class D>
struct RoundState {
    // [2 buffers][5 vars][N][NBP] ADMM variables, then scalars
    __host__ __device__ static int var_floats(int N) { return 2 * 5 * N * D::NBP; }
    __host__ __device__ static int floats(int N) { return var_floats(N) + 8; }
    // scalar slots after the variables
    static constexpr int sAlpha = 0, sCprev = 1, sWgt = 2, sRestart = 3, sCb = 4;
};

struct RoundArgs {
    const float* rec;
    int irec, n_rec, N;
    float rho, sigma, kkt_tol, eta, dx, dy;
    int max_iter, polish, accel, refine_steps;
    float refine_alpha;
    int m0, m1;              // this round runs iterations m0+1 .. m1
    float* cache;            // [B][N][2][NX*NX]  S_j, W_j
    float* state;            // [B][RoundState::floats(N)]
    uint32_t* modes;         // [B][N][NC] faces of the latest z
    uint32_t* lastm;         // [B][N][NC] faces of the last polished z
    int* done;               // [B] 1 once the instance has its final output
    int* active;             // count of instances still running after this round
    float* Kst;              // [B][N][NU][NX+1] polish gains
    float* out_xi;
    float* out_u;
    int* out_status;
    int* out_iters;
    float* out_kkt;
    unsigned long long* out_bits;
    int* out_npol;
};

// per-warp shared memory of the polish kernel (floats)
template <class D>
struct WarpSmem {
    static constexpr int NX = D::NX, NU = D::NU, NK = NX + 1;
    // every region starts on a 16-byte boundary (float4 traffic goes to oK and the stage buffers)
    static constexpr int al(int x) { return (x + 3) & ~3; }
    static constexpr int oP = 0, op = al(oP + NX * NX), oS = al(op + NX), osv = al(oS + NX * NX),
                         oSA = al(osv + NX), oSB = al(oSA + NX * NX), oSe = al(oSB + NX * NU), oet = al(oSe + NX),
                         oot = al(oet + NX), og2 = al(oot + NU), oL = al(og2 + NX),
                         oK = al(oL + NU * NU), out = al(oK + NU * NK), obuf0 = al(out + NU),
                         obuf1 = al(obuf0 + D::SREC), oFixed = al(obuf1 + D::SREC);
    static_assert(oK % 4 == 0 && obuf0 % 4 == 0 && obuf1 % 4 == 0 && oFixed % 4 == 0, "16-byte regions");
    static_assert((NU * NK) % 4 == 0 && D::SREC % 4 == 0, "float4 transfers");
    int xr, ur, y, wv, modes, cmu, cfm, cmask, total;
    __host__ __device__ explicit WarpSmem(int N) {
        int o = oFixed;
        auto take = [&o](int n) { int r = o; o += (n + 3) & ~3; return r; };
        xr = take((N + 1) * NX);
        ur = take(N * NU);
        // the certificate runs after the Riccati scan: its costates reuse the
        // factor buffer and its gradient the S/SA/SB area when they fit
        y = (N * NX <= NU * NU) ? oL : take(N * NX);
        wv = (N * NU <= oSe - oS) ? oS : take(N * NU);
        modes = take(N * D::NC);
        cmu = take(N * D::NC);
        cfm = take(N * D::NC);
        cmask = take(N);
        total = o;
    }
};

// Register prefetch of FLOATS consecutive floats (multiple of 4, 16-byte
// aligned) by one warp, stored to shared memory later: the next stage's data
// is in flight while the current stage computes.
template <int FLOATS, bool READONLY>
struct Prefetch {
    static constexpr int V4 = FLOATS / 4;
    static constexpr int PER = (V4 + 31) / 32;
    float4 r[PER];
    __device__ __forceinline__ void load(const float* src, int lane) {
        const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int idx = lane + 32 * t;
            if (idx < V4) r[t] = READONLY ? __ldg(s + idx) : s[idx];
        }
    }
    __device__ __forceinline__ void store(float* dst, int lane) const {
        float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int idx = lane + 32 * t;
            if (idx < V4) d[idx] = r[t];
        }
    }
};

template <class D>
struct WCtx {
    const float* rec;  // instance record in global memory
    float* sm;         // this warp's shared memory
    WarpSmem<D> L;
    uint32_t* modes;   // shared copy of the mode words
    float* K;          // global gains of this instance [N][NU][NK]
    int Nh, lane;
    float sigma, dx, dy;
    __device__ WCtx(int N) : L(N) {}
    __device__ const float* grec(int k) const { return rec + (size_t)k * D::SREC; }
    __device__ float* buf(int k) const { return sm + ((k & 1) ? WarpSmem<D>::obuf1 : WarpSmem<D>::obuf0); }
    __device__ float* xr() const { return sm + L.xr; }
    __device__ float* ur() const { return sm + L.ur; }
    __device__ float* y() const { return sm + L.y; }
    __device__ float* wv() const { return sm + L.wv; }
    __device__ float mu(int k, int q) const { return sm[L.cmu + k * D::NC + q]; }
    __device__ float fms(int k, int q) const { return sm[L.cfm + k * D::NC + q]; }
    __device__ uint32_t mask(int k) const { return __float_as_uint(sm[L.cmask + k]); }
};

// Column i of the reduced input map of one stage (lane i < NU), from the
// stage's record s in shared memory:
// bt = Bs T e_i, rt = (T'RsT)_ii (1 for an eliminated column), gt = (T'Rs(o - rus))_i, ot = o_i.
template <class D, class C>
__device__ __forceinline__ void reduced_column(const C& w, const float* s, uint32_t mw, int i, float* bt,
                                               float& rt, float& gt, float& ot) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD;
    const int q = i / CD, j = i % CD, base = q * CD;
    const bool swing = (mw & kSwingBit) != 0;
    const bool apex = (mw >> (2 * D::M)) & 1u;
    const bool top = (mw >> (2 * D::M + 1)) & 1u;
    const float fms = s[D::oFM + q];
    const float mu = s[D::oMU + q];
#pragma unroll
    for (int r = 0; r < NX; ++r) bt[r] = 0.0f;
    rt = 1.0f;
    gt = 0.0f;
    ot = 0.0f;
    if (swing || apex) return;
    if (j == D::NRM) {
        if (top) { ot = fms; return; }
        rt = s[D::oR + i];
        gt = -rt * s[D::oRU + i];
#pragma unroll
        for (int r = 0; r < NX; ++r) bt[r] = s[D::oB + r * NU + i];
        for (int jj = 0; jj < D::M; ++jj) {
            const int sg = face_sign(mw, jj);
            if (sg == 0) continue;
            const int tj = base + Cone<CD>::tang(jj);
            const float cj = sg * cone_coef<CD>(jj, mu, w.dx, w.dy);
            const float rtj = s[D::oR + tj];
            rt += cj * cj * rtj;
            gt -= cj * rtj * s[D::oRU + tj];
#pragma unroll
            for (int r = 0; r < NX; ++r) bt[r] = fmaf(cj, s[D::oB + r * NU + tj], bt[r]);
        }
        return;
    }
    const int jj = j < 2 ? j : j - 1;  // tangential index of component j
    const int sg = face_sign(mw, jj);
    if (sg != 0) {
        if (top) ot = sg * cone_coef<CD>(jj, mu, w.dx, w.dy) * fms;
        return;
    }
    rt = s[D::oR + i];
    gt = -rt * s[D::oRU + i];
#pragma unroll
    for (int r = 0; r < NX; ++r) bt[r] = s[D::oB + r * NU + i];
}

// x_{k+1} = A x_k + Bs u_k + e_k for lanes < NX (stage record s in shared memory)
template <class D>
__device__ __forceinline__ void rollout_step(const WCtx<D>& w, const float* s, int k) {
    constexpr int NX = D::NX, NU = D::NU;
    if (w.lane < NX) {
        const float* xk = w.xr() + k * NX;
        const float* u = w.ur() + k * NU;
        float acc = s[D::oE + w.lane];
#pragma unroll
        for (int c = 0; c < NX; ++c) acc = fmaf(s[D::oA + w.lane * NX + c], xk[c], acc);
#pragma unroll
        for (int i = 0; i < NU; ++i) acc = fmaf(s[D::oB + w.lane * NU + i], u[i], acc);
        w.xr()[(k + 1) * NX + w.lane] = acc;
    }
    __syncwarp();
}

// Backward Riccati scan + forward rollout of one instance by one warp.
template <class D>
__device__ void warp_polish(const WCtx<D>& w) {
    constexpr int NX = D::NX, NU = D::NU, NK = NX + 1;
    using WS = WarpSmem<D>;
    const int lane = w.lane;
    float* sm = w.sm;
    float* P = sm + WS::oP;
    float* p = sm + WS::op;
    float* S = sm + WS::oS;
    float* sv = sm + WS::osv;
    float* SA = sm + WS::oSA;
    float* SB = sm + WS::oSB;
    float* Se = sm + WS::oSe;
    float* et = sm + WS::oet;
    float* ot_s = sm + WS::oot;
    float* g2 = sm + WS::og2;
    float* Ls = sm + WS::oL;
    float* Ks = sm + WS::oK;
    for (int e = lane; e < NX * NX + NX; e += 32) {
        if (e < NX * NX) P[e] = 0.0f; else p[e - NX * NX] = 0.0f;
    }
    Prefetch<D::SREC, true> pf;
    pf.load(w.grec(w.Nh - 1), lane);
    for (int k = w.Nh - 1; k >= 0; --k) {
        float* s = w.buf(k);
        pf.store(s, lane);
        __syncwarp();
        if (k > 0) pf.load(w.grec(k - 1), lane);
        float bt[NX], rt = 1.0f, gt = 0.0f, ot = 0.0f;
        if (lane < NU) {
            reduced_column<D>(w, s, w.modes[k * D::NC + lane / D::CD], lane, bt, rt, gt, ot);
            ot_s[lane] = ot;
        } else {
#pragma unroll
            for (int r = 0; r < NX; ++r) bt[r] = 0.0f;
        }
        __syncwarp();
        // et = e + Bs ot ; S = diag(Q) + P ; s = Q ry + p
        if (lane < NX) {
            float acc = s[D::oE + lane];
#pragma unroll
            for (int i = 0; i < NU; ++i) acc = fmaf(s[D::oB + lane * NU + i], ot_s[i], acc);
            et[lane] = acc;
            sv[lane] = fmaf(s[D::oQ + lane], s[D::oRY + lane], p[lane]);
        }
        for (int e = lane; e < NX * NX; e += 32) {
            const int r = e / NX, c = e % NX;
            S[e] = P[e] + (r == c ? s[D::oQ + r] : 0.0f);
        }
        __syncwarp();
        // SB column lane = S bt ; SA column / Se by lanes 0..NX
        if (lane < NU) {
#pragma unroll 1
            for (int r = 0; r < NX; ++r) {
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < NX; ++c) acc = fmaf(S[r * NX + c], bt[c], acc);
                SB[r * NU + lane] = acc;
            }
        }
        if (lane <= NX) {
            float a[NX];
#pragma unroll
            for (int r = 0; r < NX; ++r) a[r] = (lane < NX) ? s[D::oA + r * NX + lane] : et[r];
#pragma unroll 1
            for (int r = 0; r < NX; ++r) {
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < NX; ++c) acc = fmaf(S[r * NX + c], a[c], acc);
                if (lane < NX) SA[r * NX + lane] = acc; else Se[r] = acc;
            }
        }
        __syncwarp();
        // row lane of M = Rt + Bt' S Bt (to shared memory, then registers) and of
        // RHS = [-Bt' S A | Bt'(s - S et) - gt] (registers)
        float m[NU], x[NK];
        if (lane < NU) {
#pragma unroll 1
            for (int j = 0; j < NU; ++j) {
                float acc = (j == lane) ? rt : 0.0f;
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(bt[r], SB[r * NU + j], acc);
                Ls[lane * NU + j] = acc;
            }
#pragma unroll 1
            for (int c = 0; c < NX; ++c) {
                float acc = 0.0f;
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(bt[r], SA[r * NX + c], acc);
                Ks[lane * NK + c] = -acc;
            }
            float acc = -gt;
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(bt[r], sv[r] - Se[r], acc);
            Ks[lane * NK + NX] = acc;
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NU; ++j) m[j] = (lane < NU) ? Ls[lane * NU + j] : 0.0f;
#pragma unroll
        for (int q = 0; q < NK; ++q) x[q] = (lane < NU) ? Ks[lane * NK + q] : 0.0f;
        __syncwarp();
        // Cholesky M = L L' (lane = row).  The row is kept shifted so that the
        // current pivot column is m[0]: step p uses m[cc] = M[lane][p + cc], and
        // column p of L is written to shared memory.
#pragma unroll 1
        for (int pp = 0; pp < NU; ++pp) {
            const float d = sqrtf(fmaxf(__shfl_sync(0xffffffffu, m[0], pp), 1e-30f));
            const float l = (lane == pp) ? d : ((lane > pp) ? m[0] / d : 0.0f);
            if (lane < NU) Ls[lane * NU + pp] = l;
#pragma unroll
            for (int cc = 1; cc < NU; ++cc) {
                const int c = pp + cc;
                const float lc = __shfl_sync(0xffffffffu, l, c & 31);
                if (c < NU && lane >= c) m[cc] = fmaf(-l, lc, m[cc]);
            }
#pragma unroll
            for (int cc = 0; cc + 1 < NU; ++cc) m[cc] = m[cc + 1];
            m[NU - 1] = 0.0f;
        }
        __syncwarp();
        // forward substitution L y = RHS (rows in registers)
#pragma unroll 1
        for (int i = 0; i < NU; ++i) {
            const float li = (lane < NU) ? Ls[lane * NU + i] : 0.0f;  // L[lane][i]
            if (lane == i) {
                const float inv = 1.0f / li;
#pragma unroll
                for (int q = 0; q < NK; ++q) x[q] *= inv;
            }
#pragma unroll
            for (int q = 0; q < NK; ++q) {
                const float xi = __shfl_sync(0xffffffffu, x[q], i);
                if (lane > i) x[q] = fmaf(-li, xi, x[q]);
            }
        }
        // backward substitution L' x = y
#pragma unroll 1
        for (int i = NU - 1; i >= 0; --i) {
            if (lane == i) {
                const float inv = 1.0f / Ls[i * NU + i];
#pragma unroll
                for (int q = 0; q < NK; ++q) x[q] *= inv;
            }
            const float lir = (lane < i) ? Ls[i * NU + lane] : 0.0f;  // L[i][lane]
#pragma unroll
            for (int q = 0; q < NK; ++q) {
                const float xi = __shfl_sync(0xffffffffu, x[q], i);
                if (lane < i) x[q] = fmaf(-lir, xi, x[q]);
            }
        }
        __syncwarp();
        if (lane < NU) {
            float* Kg = w.K + (size_t)k * NU * NK + lane * NK;
#pragma unroll
            for (int q = 0; q < NK; ++q) {
                Ks[lane * NK + q] = x[q];
                Kg[q] = x[q];
            }
        }
        __syncwarp();
        // G = SA + SB K (in place over SA), g2 = s - Se - SB kappa
#pragma unroll 1
        for (int e = lane; e < NX * NX + NX; e += 32) {
            if (e < NX * NX) {
                const int r = e / NX, c = e % NX;
                float acc = SA[e];
#pragma unroll
                for (int i = 0; i < NU; ++i) acc = fmaf(SB[r * NU + i], Ks[i * NK + c], acc);
                SA[e] = acc;
            } else {
                const int r = e - NX * NX;
                float acc = sv[r] - Se[r];
#pragma unroll
                for (int i = 0; i < NU; ++i) acc = fmaf(-SB[r * NU + i], Ks[i * NK + NX], acc);
                g2[r] = acc;
            }
        }
        __syncwarp();
        // P = sym(A' G), p = A' g2
#pragma unroll 1
        for (int e = lane; e < NX * NX + NX; e += 32) {
            if (e < NX * NX) {
                const int r = e / NX, c = e % NX;
                float a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    a1 = fmaf(s[D::oA + i * NX + r], SA[i * NX + c], a1);
                    a2 = fmaf(s[D::oA + i * NX + c], SA[i * NX + r], a2);
                }
                P[e] = 0.5f * (a1 + a2);
            } else {
                const int r = e - NX * NX;
                float acc = 0.0f;
#pragma unroll
                for (int i = 0; i < NX; ++i) acc = fmaf(s[D::oA + i * NX + r], g2[i], acc);
                p[r] = acc;
            }
        }
        __syncwarp();
    }
    // forward rollout: ut = K x + kappa, u = T ut + o, x' = A x + Bs u + e
    float* ut = sm + WS::out;
    Prefetch<D::NU * NK, false> pk;
    pf.load(w.grec(0), lane);
    pk.load(w.K, lane);
    for (int k = 0; k < w.Nh; ++k) {
        float* s = w.buf(k);
        pf.store(s, lane);
        pk.store(Ks, lane);
        __syncwarp();
        if (k + 1 < w.Nh) {
            pf.load(w.grec(k + 1), lane);
            pk.load(w.K + (size_t)(k + 1) * NU * NK, lane);
        }
        const float* xk = w.xr() + k * NX;
        if (lane < NU) {
            float acc = Ks[lane * NK + NX];
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(Ks[lane * NK + r], xk[r], acc);
            ut[lane] = acc;
        }
        __syncwarp();
        if (lane < D::NC) {
            const int q = lane, base = q * D::CD;
            const uint32_t mw = w.modes[k * D::NC + q];
            float* u = w.ur() + k * NU;
            const bool swing = (mw & kSwingBit) != 0;
            const bool apex = (mw >> (2 * D::M)) & 1u;
            const bool top = (mw >> (2 * D::M + 1)) & 1u;
            if (swing || apex) {
                for (int i = 0; i < D::CD; ++i) u[base + i] = 0.0f;
            } else {
                const float mu = s[D::oMU + q];
                const float n = top ? s[D::oFM + q] : ut[base + D::NRM];
                u[base + D::NRM] = n;
                for (int jj = 0; jj < D::M; ++jj) {
                    const int tj = base + Cone<D::CD>::tang(jj);
                    const int sg = face_sign(mw, jj);
                    u[tj] = (sg == 0) ? ut[tj] : sg * cone_coef<D::CD>(jj, mu, w.dx, w.dy) * n;
                }
            }
        }
        __syncwarp();
        rollout_step<D>(w, s, k);
    }
}

// Forward rollout of given (scaled) inputs ur (one warp).
template <class D>
__device__ void warp_rollout(const WCtx<D>& w) {
    Prefetch<D::SREC, true> pf;
    pf.load(w.grec(0), w.lane);
    for (int k = 0; k < w.Nh; ++k) {
        float* s = w.buf(k);
        pf.store(s, w.lane);
        __syncwarp();
        if (k + 1 < w.Nh) pf.load(w.grec(k + 1), w.lane);
        rollout_step<D>(w, s, k);
    }
}

// KKT certificate (same terms as `certificate` in solve.cuh), one warp.
template <class D>
__device__ float warp_certificate(const WCtx<D>& w) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int lane = w.lane;
    const float sig = w.sigma, isig = 1.0f / w.sigma;
    float den = 0.0f, uinf = 0.0f;
    // costates and the reduced gradient, stage by stage from the end
    Prefetch<D::SREC, true> pf;
    pf.load(w.grec(w.Nh - 1), lane);
    for (int k = w.Nh - 1; k >= 0; --k) {
        float* s = w.buf(k);
        pf.store(s, lane);
        __syncwarp();
        if (k > 0) pf.load(w.grec(k - 1), lane);
        if (lane < NX) {
            float acc = s[D::oQ + lane] * (w.xr()[(k + 1) * NX + lane] - s[D::oRY + lane]);
            if (k + 1 < w.Nh) {
                const float* An = w.buf(k + 1) + D::oA;  // stage k+1, kept from the previous step
#pragma unroll
                for (int i = 0; i < NX; ++i) acc = fmaf(An[i * NX + lane], w.y()[(k + 1) * NX + i], acc);
            }
            w.y()[k * NX + lane] = acc;
        }
        __syncwarp();
        if (lane < NU) {
            const int e = k * NU + lane;
            const float rdu = s[D::oR + lane] * (w.ur()[e] - s[D::oRU + lane]) * isig;
            float bty = 0.0f;
#pragma unroll
            for (int r = 0; r < NX; ++r) bty = fmaf(s[D::oB + r * NU + lane], w.y()[k * NX + r], bty);
            bty *= isig;
            w.wv()[e] = rdu + bty;
            den = fmaxf(den, fmaxf(fabsf(rdu), fabsf(bty)));
            uinf = fmaxf(uinf, fabsf(w.ur()[e]) * sig);
        }
        __syncwarp();
    }
    den = warp_max(den);
    uinf = warp_max(uinf);
    float feas = 0.0f, stat = 0.0f, comp = 0.0f;
    for (int e = lane; e < w.Nh * D::NC; e += 32) {
        const int k = e / D::NC, q = e % D::NC;
        const float fmax = w.fms(k, q) * sig;
        const float* us = w.ur() + k * NU + q * CD;
        float u[CD], r[CD];
#pragma unroll
        for (int i = 0; i < CD; ++i) { u[i] = us[i] * sig; r[i] = w.wv()[k * NU + q * CD + i]; }
        if (!((w.mask(k) >> q) & 1u)) {
            float mm = 0.0f;
#pragma unroll
            for (int i = 0; i < CD; ++i) mm = fmaxf(mm, fabsf(u[i]));
            feas = fmaxf(feas, mm / (1.0f + fmax));
            continue;
        }
        const float mu = w.mu(k, q);
        float cf[M], g[F], lam[F], nrm2[F];
        const float n = u[D::NRM];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            cf[j] = cone_coef<CD>(j, mu, w.dx, w.dy);
            const float t = u[Cone<CD>::tang(j)];
            g[2 * j] = t - cf[j] * n;
            g[2 * j + 1] = -t - cf[j] * n;
            nrm2[2 * j] = nrm2[2 * j + 1] = 1.0f + cf[j] * cf[j];
        }
        g[2 * M] = -n;
        g[2 * M + 1] = n - fmax;
        nrm2[2 * M] = nrm2[2 * M + 1] = 1.0f;
        float gmax = -INFINITY, wmax = 0.0f;
#pragma unroll
        for (int f = 0; f < F; ++f) { lam[f] = 0.0f; gmax = fmaxf(gmax, g[f]); }
#pragma unroll
        for (int i = 0; i < CD; ++i) wmax = fmaxf(wmax, fabsf(r[i]));
        feas = fmaxf(feas, fmaxf(gmax, 0.0f) / (1.0f + fmax));
        for (int sweep = 0; sweep < 100; ++sweep) {
            float change = 0.0f;
#pragma unroll
            for (int f = 0; f < F; ++f) {
                // G_f . r for face f (tangential pair j = f/2, or the two normal faces)
                float gr;
                if (f < 2 * M) {
                    const int tj = Cone<CD>::tang(f >> 1);
                    gr = ((f & 1) ? -r[tj] : r[tj]) - cf[f >> 1] * r[D::NRM];
                } else {
                    gr = (f == 2 * M) ? -r[D::NRM] : r[D::NRM];
                }
                const float num = gr + g[f] * g[f] * lam[f];
                const float dd = nrm2[f] + g[f] * g[f];
                const float nl = fmaxf(0.0f, lam[f] - num / dd);
                const float dl = nl - lam[f];
                if (f < 2 * M) {
                    const int tj = Cone<CD>::tang(f >> 1);
                    r[tj] += (f & 1) ? -dl : dl;
                    r[D::NRM] -= cf[f >> 1] * dl;
                } else {
                    r[D::NRM] += (f == 2 * M) ? -dl : dl;
                }
                lam[f] = nl;
                change = fmaxf(change, fabsf(dl) * sqrtf(dd));
            }
            // stop once a sweep moves no multiplier by more than 1e-9 (absolute,
            // far below the 1e-6-level residuals certified) or 1e-7 relative
            if (change <= 1e-9f + 1e-7f * wmax) break;
        }
        float rs = 0.0f, rc = 0.0f;
#pragma unroll
        for (int i = 0; i < CD; ++i) rs = fmaxf(rs, fabsf(r[i]));
#pragma unroll
        for (int f = 0; f < F; ++f) rc = fmaxf(rc, fabsf(lam[f] * g[f]));
        stat = fmaxf(stat, rs);
        comp = fmaxf(comp, rc);
    }
    feas = warp_max(feas);
    stat = warp_max(stat);
    comp = warp_max(comp);
    return fmaxf(feas, fmaxf(stat / (1.0f + den), comp / (1.0f + uinf)));
}

// Faces re-read off Proj(u - alpha sigma w) (see refine_modes in solve.cuh).
template <class D>
__device__ bool warp_refine_modes(const WCtx<D>& w, float alpha) {
    constexpr int NU = D::NU, CD = D::CD;
    bool changed = false;
    for (int e = w.lane; e < w.Nh * D::NC; e += 32) {
        const int k = e / D::NC, q = e % D::NC;
        if (!((w.mask(k) >> q) & 1u)) continue;
        float a[CD], out[CD];
#pragma unroll
        for (int i = 0; i < CD; ++i)
            a[i] = w.ur()[k * NU + q * CD + i] - alpha * w.sigma * w.wv()[k * NU + q * CD + i];
        const uint32_t mw = project_contact<CD>(a, out, w.mu(k, q), w.fms(k, q), w.dx, w.dy);
        if (mw != w.modes[e]) {
            changed = true;
            w.modes[e] = mw;
        }
    }
    __syncwarp();
    return __any_sync(0xffffffffu, changed);
}

// Outputs of one instance (one warp); stages beyond the horizon are 0.
template <class D>
__device__ void warp_write_output(const WCtx<D>& w, const RoundArgs& a, int b, int status, int iters, float kkt,
                                  int npol) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int Nv = a.N;
    const bool ok = status == kConverged || status == kMaxIter;
    float* oxi = a.out_xi + (size_t)b * Nv * NX;
    float* ou = a.out_u + (size_t)b * Nv * NU;
    for (int e = w.lane; e < Nv * NX; e += 32) {
        const int k = e / NX;
        oxi[e] = (ok && k < w.Nh) ? w.xr()[(k + 1) * NX + (e % NX)] : 0.0f;
    }
    for (int e = w.lane; e < Nv * NU; e += 32) {
        const int k = e / NU;
        ou[e] = (ok && k < w.Nh) ? w.ur()[e] * w.sigma : 0.0f;
    }
    for (int k = w.lane; k < Nv; k += 32) {
        unsigned long long bits = 0ull;
        if (ok && k < w.Nh) {
            for (int q = 0; q < D::NC; ++q) {
                if (!((w.mask(k) >> q) & 1u)) continue;
                const float fmax = w.fms(k, q) * w.sigma;
                const float mu = w.mu(k, q);
                const float* us = w.ur() + k * NU + q * CD;
                const float n = us[D::NRM] * w.sigma;
                const float thr = -1e-5f * (1.0f + fmax);
                float g[F];
                for (int j = 0; j < M; ++j) {
                    const float cj = cone_coef<CD>(j, mu, w.dx, w.dy);
                    const float t = us[Cone<CD>::tang(j)] * w.sigma;
                    g[2 * j] = t - cj * n;
                    g[2 * j + 1] = -t - cj * n;
                }
                g[2 * M] = -n;
                g[2 * M + 1] = n - fmax;
                for (int f = 0; f < F; ++f)
                    if (g[f] >= thr) bits |= 1ull << (q * F + f);
            }
        }
        a.out_bits[(size_t)b * Nv + k] = bits;
    }
    if (w.lane == 0) {
        a.out_status[b] = status;
        a.out_iters[b] = iters;
        a.out_kkt[b] = ok ? kkt : INFINITY;
        a.out_npol[b] = npol;
        a.done[b] = 1;
    }
}

// Polish / certify / refine after a round (one warp per instance).
template <class D>
__global__ void __launch_bounds__(32 * kPolishWarps) polish_kernel(RoundArgs a, int B) {
    extern __shared__ __align__(16) float psm[];
    constexpr int NX = D::NX, NU = D::NU;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * kPolishWarps + warp;
    if (b >= B) return;
    if (a.done[b]) return;
    WCtx<D> w(a.N);
    w.sm = psm + warp * w.L.total;
    w.rec = a.rec + (size_t)b * a.irec;
    w.modes = reinterpret_cast<uint32_t*>(w.sm + w.L.modes);
    w.K = a.Kst + (size_t)b * a.N * NU * (NX + 1);
    w.lane = lane;
    w.sigma = a.sigma;
    w.dx = a.dx;
    w.dy = a.dy;
    const float* tail = w.rec + (size_t)a.n_rec * D::SREC;
    w.Nh = __float_as_int(__ldg(tail + D::tH));
    const bool final_round = a.m1 >= a.max_iter;
    uint32_t* gmodes = a.modes + (size_t)b * a.N * D::NC;
    uint32_t* glast = a.lastm + (size_t)b * a.N * D::NC;
    bool changed = false;
    for (int e = lane; e < w.Nh * D::NC; e += 32) {
        const uint32_t mw = gmodes[e];
        w.modes[e] = mw;
        changed |= (mw != glast[e]);
        const int k = e / D::NC, q = e % D::NC;
        w.sm[w.L.cmu + e] = __ldg(w.grec(k) + D::oMU + q);
        w.sm[w.L.cfm + e] = __ldg(w.grec(k) + D::oFM + q);
    }
    for (int k = lane; k < w.Nh; k += 32) w.sm[w.L.cmask + k] = __ldg(w.grec(k) + D::oMASK);
    changed = __any_sync(0xffffffffu, changed);
    for (int i = lane; i < NX; i += 32) w.xr()[i] = __ldg(tail + D::tXI0 + i);
    int npol = a.out_npol[b];
    __syncwarp();
    float kkt = INFINITY;
    if (a.polish && changed) {
        for (int e = lane; e < w.Nh * D::NC; e += 32) glast[e] = w.modes[e];
        warp_polish<D>(w);
        ++npol;
        kkt = warp_certificate<D>(w);
        for (int r = 0; kkt > a.kkt_tol && r < a.refine_steps; ++r) {
            if (!warp_refine_modes<D>(w, a.refine_alpha)) break;
            warp_polish<D>(w);
            ++npol;
            kkt = warp_certificate<D>(w);
        }
        if (kkt <= a.kkt_tol) {
            warp_write_output<D>(w, a, b, kConverged, a.m1, kkt, npol);
            return;
        }
    }
    if (!a.polish || final_round) {
        // certify the ADMM iterate itself: u from z of the current buffer
        const float* st = a.state + (size_t)b * RoundState<D>::floats(a.N);
        const int cb = __float_as_int(st[RoundState<D>::var_floats(a.N) + RoundState<D>::sCb]);
        for (int e = lane; e < w.Nh * NU; e += 32) {
            const int k = e / NU, i = e % NU;
            w.ur()[e] = st[((cb * 5 + VZ) * a.N + k) * D::NBP + NX + i];
        }
        __syncwarp();
        warp_rollout<D>(w);
        kkt = warp_certificate<D>(w);
        if (kkt <= a.kkt_tol || final_round) {
            warp_write_output<D>(w, a, b, kkt <= a.kkt_tol ? kConverged : kMaxIter, a.m1, kkt, npol);
            return;
        }
    }
    if (lane == 0) {
        a.out_npol[b] = npol;
        atomicAdd(a.active, 1);
    }
}

// ---------------------------------------------------------------------------
// One round of ADMM iterations (CTA per instance, warp per stage): the
// iteration body of solve_kernel, with the caches and the iterate kept in
// global memory between rounds.  The first round packs the caches.
template <class D>
__global__ void __launch_bounds__(1024, 1) round_kernel(RoundArgs a) {
    extern __shared__ __align__(16) float smem[];
    constexpr int NX = D::NX, NU = D::NU, NB = D::NB;
    const int b = blockIdx.x;
    if (a.done[b]) return;
    const Smem<D> L(a.N);
    Ctx<D> c;
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
    for (int i = tid; i < NB; i += nthr) x0[i] = i < NX ? tail[D::tXI0 + i] : tail[D::tUP + i - NX];
    float* gcache = a.cache + (size_t)b * a.N * 2 * NX * NX;
    float* gstate = a.state + (size_t)b * RoundState<D>::floats(a.N);
    const int nvar = RoundState<D>::var_floats(a.N);
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
    float alpha = 1.0f, cprev = INFINITY, wgt = 0.0f;
    bool restart = false;
    int cb = 0;
    if (a.m0 > 0) {
        const float* sc = gstate + nvar;
        alpha = sc[RoundState<D>::sAlpha];
        cprev = sc[RoundState<D>::sCprev];
        wgt = sc[RoundState<D>::sWgt];
        restart = sc[RoundState<D>::sRestart] != 0.0f;
        cb = __float_as_int(sc[RoundState<D>::sCb]);
    }
    __syncthreads();
    for (int m = a.m0 + 1; m <= a.m1; ++m) {
        if (warp < c.Nh) {
            for (int which = 0; which < 5; ++which) {
                const float* cur = c.V(cb, which, warp);
                const float* prv = c.V(1 - cb, which, warp);
                float* h = c.Hh(which, warp);
                for (int i = lane; i < NB; i += 32) h[i] = restart ? prv[i] : fmaf(wgt, cur[i] - prv[i], cur[i]);
            }
        }
        __syncthreads();
        if (warp < c.Nh) block1<D>(c, warp, lane);
        __syncthreads();
        if (warp < c.Nh) block2<D>(c, warp, lane, 1 - cb);
        __syncthreads();
        float tot = 0.0f;
        for (int j = 0; j < c.Nh; ++j) tot += c.part[j];
        tot *= a.rho;
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
    // save the iterate and the faces of z for the polish kernel
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
        sc[RoundState<D>::sWgt] = wgt;
        sc[RoundState<D>::sRestart] = restart ? 1.0f : 0.0f;
        sc[RoundState<D>::sCb] = __int_as_float(cb);
    }
}

}  // namespace pinmpc
