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
    static constexpr int oP = 0, op = oP + NX * NX, oS = op + NX, osv = oS + NX * NX, oSA = osv + NX,
                         oSB = oSA + NX * NX, oSe = oSB + NX * NU, oet = oSe + NX, oot = oet + NX,
                         oG = oot + NU, og2 = oG + NX * NX, oL = og2 + NX, oK = oL + NU * NU,
                         out = oK + NU * NK, oFixed = ((out + NU) + 3) & ~3;
    int xr, ur, y, wv, modes, red, total;
    __host__ __device__ explicit WarpSmem(int N) {
        int o = oFixed;
        auto take = [&o](int n) { int r = o; o += (n + 3) & ~3; return r; };
        xr = take((N + 1) * NX);
        ur = take(N * NU);
        y = take(N * NX);
        wv = take(N * NU);
        modes = take(N * D::NC);
        red = take(4);
        total = o;
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
    __device__ const float* stage(int k) const { return rec + (size_t)k * D::SREC; }
    __device__ float* xr() const { return sm + L.xr; }
    __device__ float* ur() const { return sm + L.ur; }
    __device__ float* y() const { return sm + L.y; }
    __device__ float* wv() const { return sm + L.wv; }
    __device__ uint32_t mask(int k) const { return __float_as_uint(__ldg(stage(k) + D::oMASK)); }
};

// Column i of the reduced input map of stage k (lane i < NU):
// bt = Bs T e_i, rt = (T'RsT)_ii (1 for an eliminated column), gt = (T'Rs(o - rus))_i, ot = o_i.
template <class D>
__device__ __forceinline__ void reduced_column(const WCtx<D>& w, int k, int i, float* bt, float& rt, float& gt,
                                               float& ot) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD;
    const float* s = w.stage(k);
    const int q = i / CD, j = i % CD, base = q * CD;
    const uint32_t mw = w.modes[k * D::NC + q];
    const bool swing = (mw & kSwingBit) != 0;
    const bool apex = (mw >> (2 * D::M)) & 1u;
    const bool top = (mw >> (2 * D::M + 1)) & 1u;
    const float fms = __ldg(s + D::oFM + q);
    const float mu = __ldg(s + D::oMU + q);
#pragma unroll
    for (int r = 0; r < NX; ++r) bt[r] = 0.0f;
    rt = 1.0f;
    gt = 0.0f;
    ot = 0.0f;
    if (swing || apex) return;
    if (j == D::NRM) {
        if (top) { ot = fms; return; }
        rt = __ldg(s + D::oR + i);
        gt = -rt * __ldg(s + D::oRU + i);
#pragma unroll
        for (int r = 0; r < NX; ++r) bt[r] = __ldg(s + D::oB + r * NU + i);
        for (int jj = 0; jj < D::M; ++jj) {
            const int sg = face_sign(mw, jj);
            if (sg == 0) continue;
            const int tj = base + Cone<CD>::tang(jj);
            const float cj = sg * cone_coef<CD>(jj, mu, w.dx, w.dy);
            const float rtj = __ldg(s + D::oR + tj);
            rt += cj * cj * rtj;
            gt -= cj * rtj * __ldg(s + D::oRU + tj);
#pragma unroll
            for (int r = 0; r < NX; ++r) bt[r] = fmaf(cj, __ldg(s + D::oB + r * NU + tj), bt[r]);
        }
        return;
    }
    const int jj = j < 2 ? j : j - 1;  // tangential index of component j
    const int sg = face_sign(mw, jj);
    if (sg != 0) {
        if (top) ot = sg * cone_coef<CD>(jj, mu, w.dx, w.dy) * fms;
        return;
    }
    rt = __ldg(s + D::oR + i);
    gt = -rt * __ldg(s + D::oRU + i);
#pragma unroll
    for (int r = 0; r < NX; ++r) bt[r] = __ldg(s + D::oB + r * NU + i);
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
    float* G = sm + WS::oG;
    float* g2 = sm + WS::og2;
    float* Ls = sm + WS::oL;
    float* Ks = sm + WS::oK;
    for (int e = lane; e < NX * NX + NX; e += 32) {
        if (e < NX * NX) P[e] = 0.0f; else p[e - NX * NX] = 0.0f;
    }
    __syncwarp();
    for (int k = w.Nh - 1; k >= 0; --k) {
        const float* s = w.stage(k);
        float bt[NX], rt = 1.0f, gt = 0.0f, ot = 0.0f;
        if (lane < NU) reduced_column<D>(w, k, lane, bt, rt, gt, ot);
        else {
#pragma unroll
            for (int r = 0; r < NX; ++r) bt[r] = 0.0f;
        }
        if (lane < NU) ot_s[lane] = ot;
        __syncwarp();
        // et = e + Bs ot ; S = diag(Q) + P ; s = Q ry + p
        if (lane < NX) {
            float acc = __ldg(s + D::oE + lane);
            for (int i = 0; i < NU; ++i) acc = fmaf(__ldg(s + D::oB + lane * NU + i), ot_s[i], acc);
            et[lane] = acc;
            sv[lane] = fmaf(__ldg(s + D::oQ + lane), __ldg(s + D::oRY + lane), p[lane]);
        }
        for (int e = lane; e < NX * NX; e += 32) {
            const int r = e / NX, c = e % NX;
            S[e] = P[e] + (r == c ? __ldg(s + D::oQ + r) : 0.0f);
        }
        __syncwarp();
        // SB column lane = S bt ; SA and Se
        if (lane < NU) {
#pragma unroll
            for (int r = 0; r < NX; ++r) {
                float acc = 0.0f;
#pragma unroll
                for (int c = 0; c < NX; ++c) acc = fmaf(S[r * NX + c], bt[c], acc);
                SB[r * NU + lane] = acc;
            }
        }
        for (int cidx = lane; cidx < NX + 1; cidx += 32) {
            if (cidx < NX) {
                float a[NX];
#pragma unroll
                for (int r = 0; r < NX; ++r) a[r] = __ldg(s + D::oA + r * NX + cidx);
#pragma unroll
                for (int r = 0; r < NX; ++r) {
                    float acc = 0.0f;
#pragma unroll
                    for (int c = 0; c < NX; ++c) acc = fmaf(S[r * NX + c], a[c], acc);
                    SA[r * NX + cidx] = acc;
                }
            } else {
#pragma unroll
                for (int r = 0; r < NX; ++r) {
                    float acc = 0.0f;
#pragma unroll
                    for (int c = 0; c < NX; ++c) acc = fmaf(S[r * NX + c], et[c], acc);
                    Se[r] = acc;
                }
            }
        }
        __syncwarp();
        // row lane of M = Rt + Bt' S Bt and of RHS = [-Bt' S A | Bt'(s - S et) - gt]
        float m[NU], x[NK];
#pragma unroll
        for (int j = 0; j < NU; ++j) {
            float acc = (j == lane) ? rt : 0.0f;
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(bt[r], SB[r * NU + j], acc);
            m[j] = acc;
        }
#pragma unroll
        for (int c = 0; c < NX; ++c) {
            float acc = 0.0f;
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(bt[r], SA[r * NX + c], acc);
            x[c] = -acc;
        }
        {
            float acc = -gt;
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(bt[r], sv[r] - Se[r], acc);
            x[NX] = acc;
        }
        // Cholesky M = L L' in registers (lane = row)
#pragma unroll
        for (int pp = 0; pp < NU; ++pp) {
            const float d = sqrtf(fmaxf(__shfl_sync(0xffffffffu, m[pp], pp), 1e-30f));
            if (lane == pp) m[pp] = d;
            else if (lane > pp) m[pp] = m[pp] / d;
            const float lp = m[pp];
#pragma unroll
            for (int c = pp + 1; c < NU; ++c) {
                const float lcp = __shfl_sync(0xffffffffu, lp, c);
                if (lane >= c) m[c] = fmaf(-lp, lcp, m[c]);
            }
        }
        // forward substitution L y = RHS (rows in registers)
#pragma unroll
        for (int i = 0; i < NU; ++i) {
            if (lane == i) {
#pragma unroll
                for (int q = 0; q < NK; ++q) x[q] = x[q] / m[i];
            }
#pragma unroll
            for (int q = 0; q < NK; ++q) {
                const float xi = __shfl_sync(0xffffffffu, x[q], i);
                if (lane > i) x[q] = fmaf(-m[i], xi, x[q]);
            }
        }
        // L to shared memory for the transposed solve
        if (lane < NU) {
#pragma unroll
            for (int c = 0; c < NU; ++c) Ls[lane * NU + c] = (c <= lane) ? m[c] : 0.0f;
        }
        __syncwarp();
        // backward substitution L' x = y
#pragma unroll
        for (int i = NU - 1; i >= 0; --i) {
            if (lane == i) {
#pragma unroll
                for (int q = 0; q < NK; ++q) x[q] = x[q] / m[i];
            }
            const float lir = (lane < i) ? Ls[i * NU + lane] : 0.0f;
#pragma unroll
            for (int q = 0; q < NK; ++q) {
                const float xi = __shfl_sync(0xffffffffu, x[q], i);
                if (lane < i) x[q] = fmaf(-lir, xi, x[q]);
            }
        }
        if (lane < NU) {
            float* Kg = w.K + (size_t)k * NU * NK + lane * NK;
#pragma unroll
            for (int q = 0; q < NK; ++q) {
                Ks[lane * NK + q] = x[q];
                Kg[q] = x[q];
            }
        }
        __syncwarp();
        // G = SA + SB K, g2 = s - Se - SB kappa
        for (int e = lane; e < NX * NX + NX; e += 32) {
            if (e < NX * NX) {
                const int r = e / NX, c = e % NX;
                float acc = SA[e];
#pragma unroll
                for (int i = 0; i < NU; ++i) acc = fmaf(SB[r * NU + i], Ks[i * NK + c], acc);
                G[e] = acc;
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
        for (int e = lane; e < NX * NX + NX; e += 32) {
            if (e < NX * NX) {
                const int r = e / NX, c = e % NX;
                float a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    a1 = fmaf(__ldg(s + D::oA + i * NX + r), G[i * NX + c], a1);
                    a2 = fmaf(__ldg(s + D::oA + i * NX + c), G[i * NX + r], a2);
                }
                P[e] = 0.5f * (a1 + a2);
            } else {
                const int r = e - NX * NX;
                float acc = 0.0f;
#pragma unroll
                for (int i = 0; i < NX; ++i) acc = fmaf(__ldg(s + D::oA + i * NX + r), g2[i], acc);
                p[r] = acc;
            }
        }
        __syncwarp();
    }
    // forward rollout: ut = K x + kappa, u = T ut + o, x' = A x + Bs u + e
    float* ut = sm + WS::out;
    for (int k = 0; k < w.Nh; ++k) {
        const float* s = w.stage(k);
        const float* xk = w.xr() + k * NX;
        if (lane < NU) {
            const float* Kg = w.K + (size_t)k * NU * NK + lane * NK;
            float acc = Kg[NX];
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(Kg[r], xk[r], acc);
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
                const float mu = __ldg(s + D::oMU + q);
                const float n = top ? __ldg(s + D::oFM + q) : ut[base + D::NRM];
                u[base + D::NRM] = n;
                for (int jj = 0; jj < D::M; ++jj) {
                    const int tj = base + Cone<D::CD>::tang(jj);
                    const int sg = face_sign(mw, jj);
                    u[tj] = (sg == 0) ? ut[tj] : sg * cone_coef<D::CD>(jj, mu, w.dx, w.dy) * n;
                }
            }
        }
        __syncwarp();
        if (lane < NX) {
            const float* u = w.ur() + k * NU;
            float acc = __ldg(s + D::oE + lane);
#pragma unroll
            for (int c = 0; c < NX; ++c) acc = fmaf(__ldg(s + D::oA + lane * NX + c), xk[c], acc);
#pragma unroll
            for (int i = 0; i < NU; ++i) acc = fmaf(__ldg(s + D::oB + lane * NU + i), u[i], acc);
            w.xr()[(k + 1) * NX + lane] = acc;
        }
        __syncwarp();
    }
}

// Forward rollout of given (scaled) inputs ur (one warp).
template <class D>
__device__ void warp_rollout(const WCtx<D>& w) {
    constexpr int NX = D::NX, NU = D::NU;
    for (int k = 0; k < w.Nh; ++k) {
        const float* s = w.stage(k);
        const float* xk = w.xr() + k * NX;
        if (w.lane < NX) {
            const float* u = w.ur() + k * NU;
            float acc = __ldg(s + D::oE + w.lane);
            for (int c = 0; c < NX; ++c) acc = fmaf(__ldg(s + D::oA + w.lane * NX + c), xk[c], acc);
            for (int i = 0; i < NU; ++i) acc = fmaf(__ldg(s + D::oB + w.lane * NU + i), u[i], acc);
            w.xr()[(k + 1) * NX + w.lane] = acc;
        }
        __syncwarp();
    }
}

// KKT certificate (same terms as `certificate` in solve.cuh), one warp.
template <class D>
__device__ float warp_certificate(const WCtx<D>& w) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int lane = w.lane;
    const float sig = w.sigma, isig = 1.0f / w.sigma;
    for (int k = w.Nh - 1; k >= 0; --k) {
        const float* s = w.stage(k);
        if (lane < NX) {
            float acc = __ldg(s + D::oQ + lane) * (w.xr()[(k + 1) * NX + lane] - __ldg(s + D::oRY + lane));
            if (k + 1 < w.Nh) {
                const float* An = w.stage(k + 1) + D::oA;
                for (int i = 0; i < NX; ++i) acc = fmaf(__ldg(An + i * NX + lane), w.y()[(k + 1) * NX + i], acc);
            }
            w.y()[k * NX + lane] = acc;
        }
        __syncwarp();
    }
    float den = 0.0f, uinf = 0.0f;
    for (int e = lane; e < w.Nh * NU; e += 32) {
        const int k = e / NU, i = e % NU;
        const float* s = w.stage(k);
        const float rdu = __ldg(s + D::oR + i) * (w.ur()[e] - __ldg(s + D::oRU + i)) * isig;
        float bty = 0.0f;
        for (int r = 0; r < NX; ++r) bty = fmaf(__ldg(s + D::oB + r * NU + i), w.y()[k * NX + r], bty);
        bty *= isig;
        w.wv()[e] = rdu + bty;
        den = fmaxf(den, fmaxf(fabsf(rdu), fabsf(bty)));
        uinf = fmaxf(uinf, fabsf(w.ur()[e]) * sig);
    }
    __syncwarp();
    den = warp_max(den);
    uinf = warp_max(uinf);
    float feas = 0.0f, stat = 0.0f, comp = 0.0f;
    for (int e = lane; e < w.Nh * D::NC; e += 32) {
        const int k = e / D::NC, q = e % D::NC;
        const float* s = w.stage(k);
        const float fmax = __ldg(s + D::oFM + q) * sig;
        const float* us = w.ur() + k * NU + q * CD;
        float u[CD], r[CD];
        for (int i = 0; i < CD; ++i) { u[i] = us[i] * sig; r[i] = w.wv()[k * NU + q * CD + i]; }
        if (!((w.mask(k) >> q) & 1u)) {
            float mm = 0.0f;
            for (int i = 0; i < CD; ++i) mm = fmaxf(mm, fabsf(u[i]));
            feas = fmaxf(feas, mm / (1.0f + fmax));
            continue;
        }
        const float mu = __ldg(s + D::oMU + q);
        float cf[M], g[F], lam[F], nrm2[F];
        const float n = u[D::NRM];
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
        for (int f = 0; f < F; ++f) { lam[f] = 0.0f; gmax = fmaxf(gmax, g[f]); }
        for (int i = 0; i < CD; ++i) wmax = fmaxf(wmax, fabsf(r[i]));
        feas = fmaxf(feas, fmaxf(gmax, 0.0f) / (1.0f + fmax));
        for (int sweep = 0; sweep < 200; ++sweep) {
            float change = 0.0f;
            for (int f = 0; f < F; ++f) {
                float gr;
                int tj = 0;
                float cj = 0.0f, sgn = 0.0f;
                if (f < 2 * M) {
                    tj = Cone<CD>::tang(f >> 1);
                    cj = cf[f >> 1];
                    sgn = (f & 1) ? -1.0f : 1.0f;
                    gr = sgn * r[tj] - cj * r[D::NRM];
                } else {
                    gr = (f == 2 * M) ? -r[D::NRM] : r[D::NRM];
                }
                const float num = gr + g[f] * g[f] * lam[f];
                const float dd = nrm2[f] + g[f] * g[f];
                const float nl = fmaxf(0.0f, lam[f] - num / dd);
                const float dl = nl - lam[f];
                if (dl != 0.0f) {
                    if (f < 2 * M) {
                        r[tj] += sgn * dl;
                        r[D::NRM] -= cj * dl;
                    } else {
                        r[D::NRM] += (f == 2 * M) ? -dl : dl;
                    }
                    lam[f] = nl;
                    change = fmaxf(change, fabsf(dl) * sqrtf(dd));
                }
            }
            if (change <= 1e-7f * wmax) break;
        }
        float rs = 0.0f, rc = 0.0f;
        for (int i = 0; i < CD; ++i) rs = fmaxf(rs, fabsf(r[i]));
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
        const float* s = w.stage(k);
        float a[CD], out[CD];
        for (int i = 0; i < CD; ++i)
            a[i] = w.ur()[k * NU + q * CD + i] - alpha * w.sigma * w.wv()[k * NU + q * CD + i];
        const uint32_t mw = project_contact<CD>(a, out, __ldg(s + D::oMU + q), __ldg(s + D::oFM + q), w.dx, w.dy);
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
            const float* s = w.stage(k);
            for (int q = 0; q < D::NC; ++q) {
                if (!((w.mask(k) >> q) & 1u)) continue;
                const float fmax = __ldg(s + D::oFM + q) * w.sigma;
                const float mu = __ldg(s + D::oMU + q);
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
    }
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
