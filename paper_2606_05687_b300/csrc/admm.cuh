// ADMM round kernel: one CTA per instance, one warp per stage.
//
// The iteration is the three-block ADMM of Sec. III with its closed-form,
// horizon-parallel updates, in the factored form
//   J_j g = g - B_j' S_j B_j g,            S_j = (I + B_j B_j')^{-1}
//   H h   = D'^{-1}(h - T' W_j T D'^{-1} h), W_j = (I/rho + T D'^{-1} T')^{-1}
// with T = T_j = [A_j B_j] and D' the diagonal of the previous stage's cost
// plus the penalties.  Warp j keeps T_j in registers in two layouts:
//   column layout: lane c holds column c (and 32 + c) of T   -> T' x products
//   row layout:    lanes 2r, 2r+1 hold halves of row r of T  -> T x products
// S_j and W_j stay in shared memory as 16-float padded rows.  Everything
// that only stage j reads (its extrapolated iterate, B du_j, Abar_j xibar_j,
// its constants) lives in the registers of element lanes i and 32 + i, so a
// stage-iteration touches shared memory only for the vectors other lanes or
// other stages read.
#pragma once
#include <cuda_bf16.h>

#include "polish.cuh"
#include "tma.cuh"

namespace pinmpc {

template <class D>
struct RoundSmem {
    static constexpr int kTmp = 5;  // per-warp scratch vectors
    static constexpr int FR = 16;   // padded row length of S_j and W_j
    int sd, var, xb, tmp, pre, fac, part, sd2, fac2, total;
    // dbl: a second record and factor buffer, which TMA fills for the next
    // instance while the current one iterates
    __host__ __device__ explicit RoundSmem(int N, bool dbl = false) {
        int o = 0;
        auto take = [&o](int n) { int r = o; o += (n + 3) & ~3; return r; };
        sd = take(N * D::SREC);
        var = take(RoundState<D>::var_floats(N));
        xb = take((N + 1) * D::NBP);
        tmp = take(N * kTmp * D::NBP);
        pre = take(N * 3 * D::NBP);
        fac = take(N * 2 * D::NX * FR);
        part = take(32);
        sd2 = dbl ? take(N * D::SREC) : sd;
        fac2 = dbl ? take(N * 2 * D::NX * FR) : fac;
        total = o;
    }
    __host__ __device__ int bytes() const { return total * 4; }
    // floats of the per-instance factor cache (S_j, W_j for every stage)
    __host__ __device__ static int cache_floats(int N) { return N * 2 * D::NX * FR; }
};

template <class D>
struct RegT {
    static constexpr int NX = D::NX, NB = D::NB, CS = D::CS;
    static constexpr bool kTwo = NB > 32;  // some columns live in a second lane slot
    float colA[NX];                        // column lane of T
    float colB[kTwo ? NX : 1];             // column 32 + lane of T (0 where it does not exist)
    float rowT[CS];                        // row lane/2 of T, columns [(lane&1) CS, (lane&1) CS + CS)
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

// y_r = sum_c R[r][c] x[c] for a 16-float padded row (R = S_j or W_j); x has finite padding to 16.
__device__ __forceinline__ float prod_R(const float* row, const float* x, int lane) {
    const float4* m4 = reinterpret_cast<const float4*>(row + (lane & 1) * 8);
    const float4* x4 = reinterpret_cast<const float4*>(x + (lane & 1) * 8);
    const float4 r0 = m4[0], r1 = m4[1], v0 = x4[0], v1 = x4[1];
    float a0 = r0.x * v0.x, a1 = r0.y * v0.y;
    a0 = fmaf(r0.z, v0.z, a0);
    a1 = fmaf(r0.w, v0.w, a1);
    a0 = fmaf(r1.x, v1.x, a0);
    a1 = fmaf(r1.y, v1.y, a1);
    a0 = fmaf(r1.z, v1.z, a0);
    a1 = fmaf(r1.w, v1.w, a1);
    const float acc = a0 + a1;
    return acc + __shfl_xor_sync(0xffffffffu, acc, 1);
}

// (y_lane, y_{32+lane}) with y_c = sum_r T[r][c] x[r]; x holds NX entries (finite padding to 4).
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
                if constexpr (RegT<D>::kTwo) a1 = fmaf(M.colB[r], xv[t], a1);
            }
        }
    }
    return make_float2(a0, a1);
}

// Exact projection onto the point-contact pyramid {|t_x|, |t_y| <= mu n,
// 0 <= n <= nmax}: project_contact for contact_dim 3, where both cone
// coefficients equal mu.  The candidate pieces of phi are then the empty set,
// the larger tangential component and both, n = (a_n + mu sum_S |a_j|) /
// (1 + |S| mu^2), so with ir1 = 1/(1 + mu^2) and ir2 = 1/(1 + 2 mu^2)
// precomputed there is no division.  Any extra feasible candidate cannot
// beat the unique minimiser of the strictly convex phi.
__device__ __forceinline__ uint32_t project_point(const float* a, float* out, float mu, float nmax, float ir1,
                                                  float ir2) {
    const float ax = a[0], ay = a[1], an = a[2];
    const float tx = fabsf(ax), ty = fabsf(ay);
    // the pieces in breakpoint order (b = |t| / mu): the minimiser over the
    // reals is the first candidate whose n is not below the next breakpoint
    // (none clipped: n = a_n >= b_max; the larger clipped: n_1 >= b_min;
    // else both), clamped to [0, nmax]
    const float tmax = fmaxf(tx, ty), tmin = fminf(tx, ty);
    const float u1 = fmaf(mu, tmax, an) * ir1, u2 = fmaf(mu, tx + ty, an) * ir2;
    const float nu = (mu * an >= tmax) ? an : ((mu * u1 >= tmin) ? u1 : u2);
    const float n = fminf(fmaxf(nu, 0.0f), nmax);
    uint32_t mode = 0;
    if (n <= 0.0f) mode |= 1u << 4;
    if (n >= nmax) mode |= 1u << 5;
    const float lim = mu * n;
    float t0 = ax, t1 = ay;
    if (ax >= lim) { t0 = lim; mode |= 1u << 0; }
    if (ax <= -lim) { t0 = -lim; mode |= 1u << 1; }
    if (ay >= lim) { t1 = lim; mode |= 1u << 2; }
    if (ay <= -lim) { t1 = -lim; mode |= 1u << 3; }
    out[0] = t0;
    out[1] = t1;
    out[2] = n;
    return mode;
}

// per-stage constant vectors kept in shared memory: qbar, 1/D' (k < N-1 form), 1/D (last stage form)
enum : int { PQB = 0, PID = 1, PIDN = 2 };

template <class D>
struct RCtx {
    float *var, *xb, *tmp, *pre, *fac, *part;
    int N, Nh;
    float rho;
    // two-CTA form: this CTA holds global stages [k0, k0 + nloc) at local
    // indices 0..nloc-1; pvar/pxb are the other CTA's var/xb (generic
    // addresses into its shared memory) and pjl the local index there of
    // global stage k0 - 1
    const float *pvar, *pxb;
    int k0, nloc, pjl;
    __device__ float* T(int j, int t) const { return tmp + (j * RoundSmem<D>::kTmp + t) * D::NBP; }
    __device__ const float* P(int j, int t) const { return pre + (j * 3 + t) * D::NBP; }
    // padded row min(lane/2, NX-1) of S_j (m = 0) or W_j (m = 1)
    __device__ const float* Frow(int j, int m, int lane) const {
        const int r = min(lane >> 1, D::NX - 1);
        return fac + ((j * 2 + m) * D::NX + r) * RoundSmem<D>::FR;
    }
};

// Registers of warp j: element slots i = lane (s = 0) and i = 32 + lane (s = 1).
template <class D>
struct StageRegs {
    float e0;                 // ebar_j[lane] (0 beyond NX)
    float qbp[2], idp[2];     // qbar_{j-1} and 1/D'_{j-1}
    float mu, fmx;            // contact lane q: friction coefficient and force bound
    float ir1, ir2;           // contact lane q: 1/(1 + mu^2), 1/(1 + 2 mu^2) (point contacts)
    uint32_t stance;          // contact lane q is in stance
    uint32_t mw;              // contact lane q: faces of the latest projection
    float xlo, xhi;           // state lane i < NX: box of component i of xi_{j+1} (+-inf: none)
    float ax[2];              // Abar_j xibar_j
    float bd[2];              // B_j du_j (state rows) and du_j (input rows)
    float zh[2], vh[2], thh[2], beh[2], lah[2];  // extrapolated iterate of stage j
};

// Extrapolated value fma(wa, current, wb * previous) of variable `which`
// at element i: wa = 1 + w, wb = -w for Nesterov weight w; wa = 0, wb = 1 on
// a restart (the previous iterate).
__device__ __forceinline__ float hat_at(const float* cur, const float* prv, int off, float wa, float wb) {
    return fmaf(wa, cur[off], wb * prv[off]);
}

template <class D>
__device__ __forceinline__ void load_hats(const RCtx<D>& c, StageRegs<D>& R, int cb, int j, int lane, float wa,
                                          float wb) {
    constexpr int NBP = D::NBP, NB = D::NB;
    const float* cur = c.var + RoundState<D>::at(c.N, cb, j, 0);
    const float* prv = c.var + RoundState<D>::at(c.N, 1 - cb, j, 0);
    const bool v0 = lane < NB;
    R.zh[0] = v0 ? hat_at(cur, prv, VZ * NBP + lane, wa, wb) : 0.0f;
    R.vh[0] = v0 ? hat_at(cur, prv, VV * NBP + lane, wa, wb) : 0.0f;
    R.thh[0] = v0 ? hat_at(cur, prv, VTH * NBP + lane, wa, wb) : 0.0f;
    R.beh[0] = v0 ? hat_at(cur, prv, VBE * NBP + lane, wa, wb) : 0.0f;
    R.lah[0] = v0 ? hat_at(cur, prv, VLA * NBP + lane, wa, wb) : 0.0f;
    if constexpr (RegT<D>::kTwo) {
        const bool v1 = lane < NB - 32;
        const int i = 32 + lane;
        R.zh[1] = v1 ? hat_at(cur, prv, VZ * NBP + i, wa, wb) : 0.0f;
        R.vh[1] = v1 ? hat_at(cur, prv, VV * NBP + i, wa, wb) : 0.0f;
        R.thh[1] = v1 ? hat_at(cur, prv, VTH * NBP + i, wa, wb) : 0.0f;
        R.beh[1] = v1 ? hat_at(cur, prv, VBE * NBP + i, wa, wb) : 0.0f;
        R.lah[1] = v1 ? hat_at(cur, prv, VLA * NBP + i, wa, wb) : 0.0f;
    } else {
        R.zh[1] = R.vh[1] = R.thh[1] = R.beh[1] = R.lah[1] = 0.0f;
    }
}

// Block 1 of stage j (warp j): du_j, xibar_j = H_{j-1} htilde_{j-1} (factored),
// Abar_j xibar_j, and xibar_N for the last stage.
template <class D, bool CL = false>
__device__ __forceinline__ void block1_r(const RCtx<D>& c, const RegT<D>& M, StageRegs<D>& R, int cb, int j,
                                         int lane, float wa, float wb) {
    constexpr int NX = D::NX, NB = D::NB, NBP = D::NBP;
    constexpr bool TWO = RegT<D>::kTwo;
    const float rho = c.rho;
    const int r = lane >> 1;
    const bool rowlane = (r < NX) && !(lane & 1);
    const bool v0 = lane < NB, v1 = TWO && lane < NB - 32, p1 = TWO && lane < NBP - 32;
    float* om = c.T(j, 0);
    float* gv = c.T(j, 1);
    float* pv = c.T(j, 2);
    float* sv = c.T(j, 3);
    float* cp = c.T(j, 4);
    // omega = vhat - betahat; T' omega reads its first NX (padded to 4) entries
    const float om0 = R.vh[0] - R.beh[0], om1 = R.vh[1] - R.beh[1];
    if (lane < ((NX + 3) & ~3)) om[lane] = om0;
    __syncwarp();
    // g = B' omega_x + omega_u on the input columns (0 on the state columns)
    const float2 tg = prod_Tt<D>(M, om);
    const float g0 = (lane >= NX && v0) ? tg.x + om0 : 0.0f;
    const float g1 = v1 ? tg.y + om1 : 0.0f;
    gv[lane] = g0;
    if (p1) gv[32 + lane] = g1;
    __syncwarp();
    // p = B g ; s = S p (= B du) ; du = g - B' s
    const float pr = prod_T<D>(M, gv, lane);
    if (rowlane) pv[r] = pr;
    __syncwarp();
    const float sr = prod_R(c.Frow(j, 0, lane), pv, lane);
    if (rowlane) sv[r] = sr;
    __syncwarp();
    const float2 bs = prod_Tt<D>(M, sv);
    const float sx = __shfl_sync(0xffffffffu, sr, (2 * lane) & 31);
    R.bd[0] = lane < NX ? sx : g0 - bs.x;
    R.bd[1] = g1 - bs.y;
    // global stage index (j itself except in the two-CTA form)
    const int jg = CL ? c.k0 + j : j;
    if (jg >= 1) {
        // w = zhat_j - vhat_j - ebar_j + lambdahat_j ;
        // c' = D'^{-1}(qbar + rho (zhat_{j-1} - thetahat_{j-1}) + rho [0; w_u])
        // (stage j-1 of the first local stage lives in the other CTA)
        const bool remote = CL && j == 0;
        const float* vb = remote ? c.pvar : c.var;
        const int jp = remote ? c.pjl : j - 1;
        const float* cur = vb + RoundState<D>::at(c.N, cb, jp, 0);
        const float* prv = vb + RoundState<D>::at(c.N, 1 - cb, jp, 0);
        const float w0 = R.zh[0] - R.vh[0] - R.e0 + R.lah[0];
        float cc0 = 0.0f, cc1 = 0.0f;
        if (v0) {
            cc0 = fmaf(rho, hat_at(cur, prv, VZ * NBP + lane, wa, wb) - hat_at(cur, prv, VTH * NBP + lane, wa, wb),
                       R.qbp[0]);
            if (lane >= NX) cc0 = fmaf(rho, w0, cc0);
        }
        if (v1) {
            const float w1 = R.zh[1] - R.vh[1] + R.lah[1];
            cc1 = fmaf(rho, hat_at(cur, prv, VZ * NBP + 32 + lane, wa, wb) - hat_at(cur, prv, VTH * NBP + 32 + lane, wa, wb),
                       R.qbp[1]);
            cc1 = fmaf(rho, w1, cc1);
        }
        const float cp0 = cc0 * R.idp[0], cp1 = cc1 * R.idp[1];
        cp[lane] = cp0;
        if (p1) cp[32 + lane] = cp1;
        __syncwarp();
        // t = T c' - w_x ; sigma = W t
        const float wx = __shfl_sync(0xffffffffu, w0, r & 31);
        const float tr = prod_T<D>(M, cp, lane) - wx;
        if (rowlane) pv[r] = tr;
        __syncwarp();
        const float sg = prod_R(c.Frow(j, 1, lane), pv, lane);
        if (rowlane) om[r] = sg;
        __syncwarp();
        // xibar_j = c' - D'^{-1} T' sigma
        const float2 ts = prod_Tt<D>(M, om);
        const float xb0 = v0 ? fmaf(-R.idp[0], ts.x, cp0) : 0.0f;
        const float xb1 = v1 ? fmaf(-R.idp[1], ts.y, cp1) : 0.0f;
        float* xbj = c.xb + j * NBP;
        xbj[lane] = xb0;
        if (p1) xbj[32 + lane] = xb1;
        __syncwarp();
        // Abar_j xibar_j
        const float ar = prod_T<D>(M, xbj, lane);
        const float axs = __shfl_sync(0xffffffffu, ar, (2 * lane) & 31);
        R.ax[0] = lane < NX ? axs : xb0;
        R.ax[1] = xb1;
    }
    if (jg == c.Nh - 1) {
        float* xbN = c.xb + (CL ? j + 1 : c.Nh) * NBP;
        const float* qb = c.P(j, PQB);
        const float* idn = c.P(j, PIDN);
        xbN[lane] = v0 ? fmaf(rho, R.zh[0] - R.thh[0], qb[lane]) * idn[lane] : 0.0f;
        if (p1) xbN[32 + lane] = v1 ? fmaf(rho, R.zh[1] - R.thh[1], qb[32 + lane]) * idn[32 + lane] : 0.0f;
    }
}

// Block 2 and the dual ascents of stage j; new values go to buffer 1 - cb.
// Returns the stage's share of the combined residual (valid in every lane).
template <class D, bool CL = false, bool BOX = false>
__device__ __forceinline__ float block2_r(const RCtx<D>& c, StageRegs<D>& R, int cb, int j, int lane, float dx,
                                          float dy) {
    constexpr int NX = D::NX, NB = D::NB, NBP = D::NBP, CD = D::CD;
    constexpr bool TWO = RegT<D>::kTwo;
    const bool v0 = lane < NB, v1 = TWO && lane < NB - 32;
    // xibar_{j+1} of the last local stage comes from the other CTA's first
    // stage unless j is the last stage of the horizon
    const float* xbn = (CL && j + 1 == c.nloc && c.k0 + j + 1 < c.Nh) ? c.pxb : c.xb + (j + 1) * NBP;
    float* arg = c.T(j, 0);
    float* zp = c.T(j, 1);
    // gamma = B du + betahat - Abar xibar - ebar + lambdahat ; gammatilde = xibar_{j+1} + thetahat + Abar xibar + ebar - lambdahat
    const float xn0 = v0 ? xbn[lane] : 0.0f;
    const float xn1 = v1 ? xbn[32 + lane] : 0.0f;
    const float ga0 = R.bd[0] + R.beh[0] - R.ax[0] - R.e0 + R.lah[0];
    const float gt0 = xn0 + R.thh[0] + R.ax[0] + R.e0 - R.lah[0];
    const float a0 = (2.0f * gt0 + ga0) * (1.0f / 3.0f);
    const float ga1 = R.bd[1] + R.beh[1] - R.ax[1] + R.lah[1];
    const float gt1 = xn1 + R.thh[1] + R.ax[1] - R.lah[1];
    const float a1 = (2.0f * gt1 + ga1) * (1.0f / 3.0f);
    if (v0) arg[lane] = a0;
    if (v1) arg[32 + lane] = a1;
    __syncwarp();
    if (lane < D::NC) {
        const int q = lane;
        if (R.stance) {
            if constexpr (CD == 3)
                R.mw = project_point(arg + NX + q * CD, zp + NX + q * CD, R.mu, R.fmx, R.ir1, R.ir2);
            else
                R.mw = project_contact<CD>(arg + NX + q * CD, zp + NX + q * CD, R.mu, R.fmx, dx, dy);
        } else {
#pragma unroll
            for (int i = 0; i < CD; ++i) zp[NX + q * CD + i] = 0.0f;
            R.mw = kSwingBit;
        }
    }
    __syncwarp();
    float* nxt = c.var + RoundState<D>::at(c.N, 1 - cb, j, 0);
    float cm = 0.0f;
    if (v0) {
        // z = Proj onto X_j x U_j: the state part clipped to its box (when set)
        const float z = lane < NX ? (BOX ? fminf(fmaxf(a0, R.xlo), R.xhi) : a0) : zp[lane];
        const float v = 0.5f * (z + ga0);
        const float th = R.thh[0] + xn0 - z;
        const float be = R.beh[0] + R.bd[0] - v;
        const float la = R.lah[0] + z - R.ax[0] - v - R.e0;
        nxt[VZ * NBP + lane] = z;
        nxt[VV * NBP + lane] = v;
        nxt[VTH * NBP + lane] = th;
        nxt[VBE * NBP + lane] = be;
        nxt[VLA * NBP + lane] = la;
        const float d1 = th - R.thh[0], d2 = be - R.beh[0], d3 = la - R.lah[0];
        const float d4 = z - R.zh[0], d5 = v - R.vh[0], d6 = d4 - d5;
        cm = d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
    }
    if (v1) {
        const int i = 32 + lane;
        const float z = zp[i];
        const float v = 0.5f * (z + ga1);
        const float th = R.thh[1] + xn1 - z;
        const float be = R.beh[1] + R.bd[1] - v;
        const float la = R.lah[1] + z - R.ax[1] - v;
        nxt[VZ * NBP + i] = z;
        nxt[VV * NBP + i] = v;
        nxt[VTH * NBP + i] = th;
        nxt[VBE * NBP + i] = be;
        nxt[VLA * NBP + i] = la;
        const float d1 = th - R.thh[1], d2 = be - R.beh[1], d3 = la - R.lah[1];
        const float d4 = z - R.zh[1], d5 = v - R.vh[1], d6 = d4 - d5;
        cm += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
    }
    return warp_sum(cm);
}

// In-place Gauss-Jordan inverses (no pivoting: the matrices are SPD) of two
// matrices at once, one per half warp: lane (m, r) = (lane / 16, lane % 16) holds row r of matrix m (rows past
// NX duplicate the last one).  Every pivot row is broadcast within its half.
template <class D>
__device__ __forceinline__ void gj_inverse_two(int lane, float (&row)[D::NX]) {
    constexpr int NX = D::NX;
    const int base = lane & 16, r = min(lane & 15, NX - 1);
#pragma unroll
    for (int p = 0; p < NX; ++p) {
        float prow[NX];
#pragma unroll
        for (int cc = 0; cc < NX; ++cc) prow[cc] = __shfl_sync(0xffffffffu, row[cc], base + p);
        const float piv = 1.0f / prow[p];
        const float fp = row[p] * piv;
        const bool mine = (r == p);
#pragma unroll
        for (int cc = 0; cc < NX; ++cc) {
            const float other = (cc == p) ? -fp : fmaf(-fp, prow[cc], row[cc]);
            const float pivr = (cc == p) ? piv : prow[cc] * piv;
            row[cc] = mine ? pivr : other;
        }
    }
}

// Row r = min(lane % 16, NX - 1) of  dg I + T diag(w) T'  with T = [A B]
// given as its columns tT[i][0..15] (zero-padded), i < NB, and the column
// weights w (0 drops a column).  The terms go into two partial sums by the
// parity of i - i0 (i0 = NX for m = 0, the first column of B; 0 for m = 1),
// added at the end; both halves of the warp run the same loop.
template <class D>
__device__ __forceinline__ void gram_rows(const float* tT, const float* w, float dg, int lane, float (&row)[D::NX]) {
    constexpr int NX = D::NX, NB = D::NB;
    const int r = min(lane & 15, NX - 1);
    const int i_start = (lane < 16) ? (NX & 1) : 0;
    float a0[NX], a1[NX];
#pragma unroll
    for (int cc = 0; cc < NX; ++cc) a0[cc] = a1[cc] = 0.0f;
    auto term = [&](int i, float (&acc)[NX]) {
        const float4* col = reinterpret_cast<const float4*>(tT + i * 16);
        float cv[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 t4 = col[q];
            cv[4 * q] = t4.x;
            cv[4 * q + 1] = t4.y;
            cv[4 * q + 2] = t4.z;
            cv[4 * q + 3] = t4.w;
        }
        const float tri = tT[i * 16 + r] * w[i];
#pragma unroll
        for (int cc = 0; cc < NX; ++cc) acc[cc] = fmaf(tri, cv[cc], acc[cc]);
    };
    for (int t = 0; t < (NB + 1) / 2; ++t) {
        const int i = i_start + 2 * t;
        if (i < NB) term(i, a0);
        if (i + 1 < NB) term(i + 1, a1);
    }
#pragma unroll
    for (int cc = 0; cc < NX; ++cc) {
        row[cc] = a0[cc] + a1[cc];
        if (cc == r) row[cc] += dg;
    }
}


// Precision of the factor kernel's Gram products T diag(d) T' (mpc_config.precision).
enum : int { kPrecFP32 = 0, kPrecTF32 = 1, kPrecBF16 = 2 };

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t to_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo in the low half
    return *reinterpret_cast<const uint32_t*>(&v);
}

// The Gram product of gram_rows (T diag(d) T' over the columns i >= i0) on the tensor cores
// (warp-level mma.sync, FP32 accumulation): TF32 operands (m16n8k8) or BF16
// operands (m16n8k16).  M = the NX rows of T (padded to 16), N = the same 16
// (two 8-column tiles), K = the columns i0 .. NB-1 (padded to the MMA's K);
// A[m][k] = T[m][i0 + k], B[k][n] = d[i0 + k] T[n][i0 + k].  The 16 x 16
// result goes to the warp's scratch `sg` (16 x 17 floats), from which the
// rows of the inversion (FP32) are read.
template <class D, int PREC>
__device__ __forceinline__ void gram_mma(const float* sj, const float* d, int i0, int lane, float* sg) {
    constexpr int NX = D::NX, NU = D::NU, NB = D::NB, GP = 17;
    const int g = lane >> 2, t = lane & 3;
    auto T = [&](int rr, int cc) -> float {
        if (rr >= NX || cc >= NB) return 0.0f;
        return cc < NX ? sj[D::oA + rr * NX + cc] : sj[D::oB + rr * NU + cc - NX];
    };
    auto dT = [&](int rr, int cc) -> float { return (cc < NB && d) ? d[cc] * T(rr, cc) : T(rr, cc); };
    float acc[2][4] = {};
    if constexpr (PREC == kPrecTF32) {
        for (int c0 = i0; c0 < NB; c0 += 8) {
            const uint32_t a0 = to_tf32(T(g, c0 + t)), a1 = to_tf32(T(g + 8, c0 + t));
            const uint32_t a2 = to_tf32(T(g, c0 + t + 4)), a3 = to_tf32(T(g + 8, c0 + t + 4));
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const uint32_t b0 = to_tf32(dT(nt * 8 + g, c0 + t)), b1 = to_tf32(dT(nt * 8 + g, c0 + t + 4));
                asm volatile(
                    "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};"
                    : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        }
    } else {
        for (int c0 = i0; c0 < NB; c0 += 16) {
            const uint32_t a0 = to_bf16x2(T(g, c0 + 2 * t), T(g, c0 + 2 * t + 1));
            const uint32_t a1 = to_bf16x2(T(g + 8, c0 + 2 * t), T(g + 8, c0 + 2 * t + 1));
            const uint32_t a2 = to_bf16x2(T(g, c0 + 2 * t + 8), T(g, c0 + 2 * t + 9));
            const uint32_t a3 = to_bf16x2(T(g + 8, c0 + 2 * t + 8), T(g + 8, c0 + 2 * t + 9));
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int n = nt * 8 + g;
                const uint32_t b0 = to_bf16x2(dT(n, c0 + 2 * t), dT(n, c0 + 2 * t + 1));
                const uint32_t b1 = to_bf16x2(dT(n, c0 + 2 * t + 8), dT(n, c0 + 2 * t + 9));
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};"
                    : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        }
    }
    // accumulator (row g or g + 8, column nt*8 + 2t or + 1) -> sg
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        sg[g * GP + nt * 8 + 2 * t] = acc[nt][0];
        sg[g * GP + nt * 8 + 2 * t + 1] = acc[nt][1];
        sg[(g + 8) * GP + nt * 8 + 2 * t] = acc[nt][2];
        sg[(g + 8) * GP + nt * 8 + 2 * t + 1] = acc[nt][3];
    }
}

// Per-stage factors of the ADMM round, one warp per (instance, stage):
// S_j = (I + B_j B_j')^{-1} and W_j = (I/rho + T_j D'^{-1}_{j-1} T_j')^{-1},
// written to the factor cache as 16-float padded rows, and the input checks
// of the stage (non-finite data; a stance contact with negative friction
// coefficient or force bound) as per-instance flag bits (1, 2).  Runs at
// full occupancy ahead of the first round, which then only loads the cache.
struct FactorArgs {
    const float* rec;
    int irec, n_rec, N, B;
    float rho;
    float* cache;  // [B][N][2][NX][16]
    int* flags;    // [B], zeroed before the launch
    int precision; // kPrecFP32 / kPrecTF32 / kPrecBF16: operands of the Gram products
};
constexpr int kFactorWarps = 8;

// PREC selects the Gram products' operands (FP32 on the FMA pipes, or TF32 /
// BF16 on the tensor cores with FP32 accumulation); the inversions are FP32.
template <class D, int PREC = kPrecFP32>
__global__ void __launch_bounds__(32 * kFactorWarps) factor_kernel(FactorArgs a) {
    constexpr int NX = D::NX, NB = D::NB, NBP = D::NBP, FR = RoundSmem<D>::FR;
    static_assert(D::SREC % 4 == 0, "records are copied as float4");
    static_assert(NX <= 16, "the tensor-core Gram covers 16 rows");
    __shared__ __align__(16) float s_rec[kFactorWarps][D::SREC];
    __shared__ __align__(16) float s_d[kFactorWarps][NBP];
    // FP32: T = [A B] as columns (16-float rows, zero-padded) and the two
    // Grams' column weights; tensor cores: the two 16 x 17 Gram products
    constexpr bool F32 = PREC == kPrecFP32;
    __shared__ __align__(16) float s_t[kFactorWarps][F32 ? NB * 16 + 2 * NBP : 2 * 16 * 17];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kFactorWarps + warp;
    if (gw >= a.B * a.N) return;  // whole warps leave; the kernel has no CTA barrier
    const int b = gw / a.N, j = gw % a.N;
    const float* rec = a.rec + (size_t)b * a.irec;
    const float* tail = rec + (size_t)a.n_rec * D::SREC;
    const int Nh0 = __float_as_int(__ldg(tail + D::tH));
    const int Nh = (Nh0 >= 1 && Nh0 <= a.N) ? Nh0 : 0;
    if (j >= Nh) return;
    float* sr = s_rec[warp];
    float* dd = s_d[warp];
    {
        const float4* src = reinterpret_cast<const float4*>(rec + (size_t)j * D::SREC);
        for (int e = lane; e < D::SREC / 4; e += 32) reinterpret_cast<float4*>(sr)[e] = __ldg(src + e);
    }
    if (j >= 1) {
        const float* sp = rec + (size_t)(j - 1) * D::SREC;
        for (int i = lane; i < NBP; i += 32)
            dd[i] = i < NX ? 1.0f / (__ldg(sp + D::oQ + i) + a.rho)
                           : (i < NB ? 1.0f / (__ldg(sp + D::oR + i - NX) + 2.0f * a.rho) : 0.0f);
    }
    __syncwarp();
    bool bad = false, badset = false;
    for (int e = lane; e < D::oMASK; e += 32) bad |= !isfinite(sr[e]);
    int packbits = 0;
    if (j == 0) {
        for (int i = lane; i < NB; i += 32)
            bad |= !isfinite(__ldg(tail + (i < NX ? D::tXI0 + i : D::tUP + i - NX)));
        packbits = __float_as_int(__ldg(tail + D::tFLAG));  // 4: bad per-instance input count
    }
    const uint32_t mk = __float_as_uint(sr[D::oMASK]);
    if (lane < D::NC && ((mk >> lane) & 1u)) badset = sr[D::oMU + lane] < 0.0f || sr[D::oFM + lane] < 0.0f;
    bad = __any_sync(0xffffffffu, bad);
    badset = __any_sync(0xffffffffu, badset);
    if (lane == 0 && (bad || badset || packbits)) atomicOr(a.flags + b, (bad ? 1 : 0) | (badset ? 2 : 0) | packbits);
    float* gc = a.cache + (size_t)b * RoundSmem<D>::cache_floats(a.N);
    // half warp m computes matrix m: S_j (m = 0, the Gram of B's columns plus
    // I) and W_j (m = 1, the Gram of T D'^{-1} plus I/rho; stage 0 has none),
    // one row per lane, then both are inverted in one pass
    const int m = lane >> 4, r = lane & 15;
    const float dg = m ? 1.0f / a.rho : 1.0f;
    float* st = s_t[warp];
    float row[NX];
    if constexpr (F32) {
        float* w = st + NB * 16;
        for (int e = lane; e < NB * 16; e += 32) {
            const int i = e >> 4, cc = e & 15;
            st[e] = cc < NX ? (i < NX ? sr[D::oA + cc * NX + i] : sr[D::oB + cc * D::NU + i - NX]) : 0.0f;
        }
        for (int i = lane; i < NBP; i += 32) {
            w[i] = (i >= NX && i < NB) ? 1.0f : 0.0f;
            w[NBP + i] = (j >= 1 && i < NB) ? dd[i] : 0.0f;
        }
        __syncwarp();
        gram_rows<D>(st, w + m * NBP, dg, lane, row);
    } else {
        gram_mma<D, PREC>(sr, nullptr, NX, lane, st);
        if (j >= 1) gram_mma<D, PREC>(sr, dd, 0, lane, st + 16 * 17);
        __syncwarp();
        const float* g = st + m * 16 * 17;
        const int rr = min(r, NX - 1);
        const bool none = m == 1 && j == 0;
#pragma unroll
        for (int cc = 0; cc < NX; ++cc) row[cc] = (none ? 0.0f : g[rr * 17 + cc]) + (cc == rr ? dg : 0.0f);
    }
    gj_inverse_two<D>(lane, row);
    if (r < NX && (m == 0 || j >= 1)) {
        float4* dst = reinterpret_cast<float4*>(gc + ((j * 2 + m) * NX + r) * FR);
#pragma unroll
        for (int q = 0; q < FR / 4; ++q) {
            const int c0 = 4 * q;
            dst[q] = make_float4(c0 < NX ? row[c0] : 0.0f, c0 + 1 < NX ? row[c0 + 1] : 0.0f,
                                 c0 + 2 < NX ? row[c0 + 2] : 0.0f, c0 + 3 < NX ? row[c0 + 3] : 0.0f);
        }
    }
}

// State box of global stage jg (the bounds of xi_{jg+1}) into the state lanes' registers.
template <class D>
__device__ __forceinline__ void load_box(const RoundArgs& a, int b, int jg, int lane, StageRegs<D>& R) {
    R.xlo = -INFINITY;
    R.xhi = INFINITY;
    if (a.xbox && lane < D::NX) {
        const float* bx = a.xbox + ((size_t)b * a.n_rec + jg) * 2 * D::NX;
        R.xlo = bx[lane];
        R.xhi = bx[D::NX + lane];
    }
}

// After a round, the state bounds z_{jg+1} sits at (its clip is exact, so
// equality marks an active bound): bit i lower, bit 16 + i upper.  Whole warp.
template <class D>
__device__ __forceinline__ void store_box_bits(const RoundArgs& a, int b, int jg, int lane, const StageRegs<D>& R,
                                               const float* zcur) {
    if (!a.xbox) return;
    const float z = lane < D::NX ? zcur[lane] : 0.0f;
    const unsigned lo = __ballot_sync(0xffffffffu, lane < D::NX && z <= R.xlo);
    const unsigned hi = __ballot_sync(0xffffffffu, lane < D::NX && z >= R.xhi);
    if (lane == 0) a.smodes[(size_t)b * a.N + jg] = (lo & 0xffffu) | (hi << 16);
}

// Writes a failure status for instance b (no iterate): zero trajectory and inputs.
template <class D>
__device__ void round_fail(const RoundArgs& a, int b, int status) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int e = tid; e < a.N * D::NX; e += nthr) a.out_xi[(size_t)b * a.N * D::NX + e] = 0.0f;
    for (int e = tid; e < a.N * D::NU; e += nthr) a.out_u[(size_t)b * a.N * D::NU + e] = 0.0f;
    for (int k = tid; k < a.N; k += nthr) a.out_bits[(size_t)b * a.N + k] = 0ull;
    if (tid == 0) {
        a.out_status[b] = status;
        a.out_iters[b] = 0;
        a.out_kkt[b] = INFINITY;
        a.out_npol[b] = 0;
        a.out_piv[b] = 0;
        a.done[b] = 1;
    }
}

// One round of ADMM iterations (a.m0, a.m1] for one instance per CTA; the
// factor cache and the iterate stay in global memory between rounds.  The
// CTA's shared memory holds cap stages: N, or with CAPPED a.cap < N (the
// launch serves a horizon class whose horizons all fit).  The uncapped form
// is compiled with cap = N throughout.
template <class D, int MAXT, bool CAPPED, bool BOX>
__device__ __forceinline__ void round_instance(const RoundArgs& a, int b, float* smem, int buf) {
    constexpr int NX = D::NX, NU = D::NU, NB = D::NB, NBP = D::NBP, FR = RoundSmem<D>::FR;
    constexpr bool TWO = RegT<D>::kTwo;
    if (a.done[b]) return;
    const int cap = CAPPED ? a.cap : a.N;
    const RoundSmem<D> L(cap, a.dbl != 0);
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const float* rec = a.rec + (size_t)b * a.irec;
    const float* tail = rec + (size_t)a.n_rec * D::SREC;
    const int Nh0 = __float_as_int(__ldg(tail + D::tH));
    const int Nh = (Nh0 >= 1 && Nh0 <= cap) ? Nh0 : 0;
    if (Nh == 0) {
        round_fail<D>(a, b, kBadHorizon);
        return;
    }
    if (a.m0 == 0) {
        const int fl = a.flags[b];  // written by factor_kernel
        if (fl) {
            round_fail<D>(a, b, (fl & 1) ? kNonFinite : ((fl & 4) ? kBadDim : kBadSet));
            return;
        }
    }
    RCtx<D> c;
    c.var = smem + L.var; c.xb = smem + L.xb; c.tmp = smem + L.tmp; c.pre = smem + L.pre;
    c.fac = smem + (buf ? L.fac2 : L.fac); c.part = smem + L.part;
    c.N = cap; c.Nh = Nh; c.rho = a.rho;
    float* sd = smem + (buf ? L.sd2 : L.sd);
    if (!a.dbl) {  // otherwise the records are already there (TMA)
        const float4* src = reinterpret_cast<const float4*>(rec);
        float4* dst = reinterpret_cast<float4*>(sd);
        const int n4 = Nh * D::SREC / 4;
        for (int e = tid; e < n4; e += nthr) dst[e] = __ldg(src + e);
    }
    for (int i = tid; i < NBP; i += nthr)
        c.xb[i] = i < NX ? __ldg(tail + D::tXI0 + i) : (i < NB ? __ldg(tail + D::tUP + i - NX) : 0.0f);
    // vectors read as float4 need finite padding
    for (int e = NBP + tid; e < (cap + 1) * NBP; e += nthr) c.xb[e] = 0.0f;
    for (int e = tid; e < cap * RoundSmem<D>::kTmp * NBP; e += nthr) c.tmp[e] = 0.0f;
    __syncthreads();
    auto stage = [&](int k) { return sd + k * D::SREC; };
    auto mask = [&](int k) { return __float_as_uint(stage(k)[D::oMASK]); };
    float* gcache = a.cache + (size_t)b * RoundSmem<D>::cache_floats(a.N);
    float* gstate = a.state + (size_t)b * RoundState<D>::floats(a.N);
    const int nvar = RoundState<D>::var_floats(a.N);  // global layout: N stages per buffer
    const int lvar = RoundState<D>::var_floats(cap);  // shared-memory layout: cap stages per buffer
    // per-stage constants: qbar, 1/D' = 1/(Q+rho | R+2rho), 1/D = 1/(Q+rho | R+rho)
    for (int e = tid; e < Nh * NBP; e += nthr) {
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
    __syncthreads();
    if (!a.dbl) {
        const float4* fs = reinterpret_cast<const float4*>(gcache);
        float4* fd = reinterpret_cast<float4*>(c.fac);
        for (int e = tid; e < Nh * 2 * NX * FR / 4; e += nthr) fd[e] = fs[e];
    }
    const bool warm = a.m0 == 0 && b < a.warm_B;  // start from the shifted previous iterate
    if (a.m0 == 0) {
        if (!warm) {
            for (int e = tid; e < lvar; e += nthr) c.var[e] = 0.0f;
            // stages past cap start (and stay) zero, as when all N are held
            for (int e = tid; cap < a.N && e < 2 * (a.N - cap) * 5 * NBP; e += nthr) {
                const int bf = e / ((a.N - cap) * 5 * NBP), r = e % ((a.N - cap) * 5 * NBP);
                gstate[RoundState<D>::at(a.N, bf, cap, 0) + r] = 0.0f;
            }
        }
        for (int e = tid; e < a.N * D::NC; e += nthr) a.lastm[(size_t)b * a.N * D::NC + e] = 0xffffffffu;
        if constexpr (BOX)
            for (int e = tid; e < a.N; e += nthr) a.slast[(size_t)b * a.N + e] = 0xffffffffu;
        if (tid == 0) {
            a.out_npol[b] = 0;
            a.out_piv[b] = 0;
        }
    }
    if (a.m0 > 0 || warm) {
        if (cap == a.N) {
            const float4* src = reinterpret_cast<const float4*>(gstate);
            float4* dst = reinterpret_cast<float4*>(c.var);
            for (int e = tid; e < nvar / 4; e += nthr) dst[e] = src[e];
        } else {
            for (int bf = 0; bf < 2; ++bf) {
                const float4* src = reinterpret_cast<const float4*>(gstate + RoundState<D>::at(a.N, bf, 0, 0));
                float4* dst = reinterpret_cast<float4*>(c.var + RoundState<D>::at(cap, bf, 0, 0));
                for (int e = tid; e < lvar / 8; e += nthr) dst[e] = src[e];
            }
        }
    }
    // stage matrix and per-stage constants into registers
    const int j = warp < Nh ? warp : 0;
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
        const int jp = j >= 1 ? j - 1 : 0;
        R.qbp[0] = lane < NB ? c.P(jp, PQB)[lane] : 0.0f;
        R.idp[0] = lane < NB ? c.P(jp, PID)[lane] : 0.0f;
        R.qbp[1] = (TWO && lane < NB - 32) ? c.P(jp, PQB)[32 + lane] : 0.0f;
        R.idp[1] = (TWO && lane < NB - 32) ? c.P(jp, PID)[32 + lane] : 0.0f;
        const int q = lane < D::NC ? lane : 0;
        R.mu = sj[D::oMU + q];
        R.fmx = sj[D::oFM + q];
        R.ir1 = 1.0f / (1.0f + R.mu * R.mu);
        R.ir2 = 1.0f / (1.0f + 2.0f * R.mu * R.mu);
        R.stance = (mask(j) >> q) & 1u;
        R.mw = 0u;
        if constexpr (BOX) load_box<D>(a, b, j, lane, R);
    }
    __syncthreads();
    // Abar_0 xibar_0 is constant; the other stages form theirs every iteration
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
    const bool active = warp < Nh;
    for (int m = a.m0 + 1; m <= a.m1; ++m) {
        const float wa = restart ? 0.0f : 1.0f + wgt, wb = restart ? 1.0f : -wgt;
        if (active) {
            load_hats<D>(c, R, cb, j, lane, wa, wb);
            block1_r<D>(c, M, R, cb, j, lane, wa, wb);
        }
        __syncthreads();
        if (active) {
            const float cm = block2_r<D, false, BOX>(c, R, cb, j, lane, a.dx, a.dy);
            if (lane == 0) c.part[j] = cm;
        }
        __syncthreads();
        float tot = lane < Nh ? c.part[lane] : 0.0f;
        tot = warp_sum(tot) * a.rho;
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
    if (cap == a.N) {
        const float4* src = reinterpret_cast<const float4*>(c.var);
        float4* dst = reinterpret_cast<float4*>(gstate);
        for (int e = tid; e < nvar / 4; e += nthr) dst[e] = src[e];
    } else {
        for (int bf = 0; bf < 2; ++bf) {
            const float4* src = reinterpret_cast<const float4*>(c.var + RoundState<D>::at(cap, bf, 0, 0));
            float4* dst = reinterpret_cast<float4*>(gstate + RoundState<D>::at(a.N, bf, 0, 0));
            for (int e = tid; e < lvar / 8; e += nthr) dst[e] = src[e];
        }
    }
    if (active && lane < D::NC && a.m1 > a.m0) a.modes[((size_t)b * a.N + j) * D::NC + lane] = R.mw;
    if constexpr (BOX)
        if (active && a.m1 > a.m0) store_box_bits<D>(a, b, j, lane, R, c.var + RoundState<D>::at(cap, cb, j, VZ));
    if (tid == 0) {
        float* sc = gstate + nvar;
        sc[RoundState<D>::sAlpha] = alpha;
        sc[RoundState<D>::sCprev] = cprev;
        sc[RoundState<D>::sWgt] = wgt;
        sc[RoundState<D>::sRestart] = restart ? 1.0f : 0.0f;
        sc[RoundState<D>::sCb] = __int_as_float(cb);
    }
}

// Receding-horizon warm start: the final
// ADMM iterate of instance b -- both buffers of (z, v, theta, beta, lambda) --
// moves `shift` stages towards the start of its horizon Nh, the last stage
// repeated into the freed tail, and the acceleration restarts (alpha 1, no
// previous residual).  One CTA per instance, through shared memory.
template <class D>
__global__ void warm_shift_kernel(float* state, const float* rec, int irec, int n_rec, int N, int shift) {
    extern __shared__ __align__(16) float wsm[];
    const int b = blockIdx.x;
    float* st = state + (size_t)b * RoundState<D>::floats(N);
    const int nvar = RoundState<D>::var_floats(N);
    const float* tail = rec + (size_t)b * irec + (size_t)n_rec * D::SREC;
    const int Nh0 = __float_as_int(__ldg(tail + D::tH));
    const int Nh = (Nh0 >= 1 && Nh0 <= N) ? Nh0 : N;
    bool bad = false;
    for (int e = threadIdx.x; e < nvar; e += blockDim.x) {
        wsm[e] = st[e];
        bad |= !isfinite(wsm[e]);
    }
    // an instance without a usable iterate (its previous solve failed) starts cold
    const bool cold = __syncthreads_or(bad);
    constexpr int SV = 5 * D::NBP;  // floats of one stage in one buffer
    for (int e = threadIdx.x; e < nvar; e += blockDim.x) {
        const int buf = e / (N * SV), r = e % (N * SV), j = r / SV, o = r % SV;
        const int src = min(j + shift, Nh - 1);
        st[e] = cold ? 0.0f : (j < Nh ? wsm[(buf * N + src) * SV + o] : wsm[e]);
    }
    if (threadIdx.x == 0) {
        float* sc = st + nvar;
        sc[RoundState<D>::sAlpha] = 1.0f;
        sc[RoundState<D>::sCprev] = INFINITY;
        sc[RoundState<D>::sWgt] = 0.0f;
        sc[RoundState<D>::sRestart] = 0.0f;
    }
}

// One round of ADMM iterations (a.m0, a.m1]: persistent CTAs (one per SM), each
// taking instances of the round's list until it is exhausted.
// Thread 0: start the TMA copies of instance b's records (the first cap
// stages) and factors into buffer buf, completing on bar[buf].
template <class D, bool CAPPED>
__device__ __noinline__ void round_fetch(const RoundArgs& a, float* smem, uint64_t* bar, int b, int buf) {
    const int cap = CAPPED ? a.cap : a.N;
    const RoundSmem<D> L(cap, true);
    const uint32_t rec_bytes = (uint32_t)(cap * D::SREC * sizeof(float));
    const uint32_t fac_bytes = (uint32_t)(RoundSmem<D>::cache_floats(cap) * sizeof(float));
    mbar_arrive_expect_tx(&bar[buf], rec_bytes + fac_bytes);
    bulk_copy_g2s(smem + (buf ? L.sd2 : L.sd), a.rec + (size_t)b * a.irec, rec_bytes, &bar[buf]);
    bulk_copy_g2s(smem + (buf ? L.fac2 : L.fac), a.cache + (size_t)b * RoundSmem<D>::cache_floats(a.N), fac_bytes,
                  &bar[buf]);
}

// With a.dbl, thread 0 starts the TMA copies of the next instance's records
// and factors into the other buffer as soon as it knows that instance, so
// they arrive while the current instance iterates.
template <class D, int MAXT, bool CAPPED = false, bool BOX = false>
__global__ void __launch_bounds__(MAXT, 1) round2_kernel(RoundArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int item;
    __shared__ __align__(8) uint64_t bar[2];
    const bool dbl = a.dbl != 0;
    if (dbl && threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    int b = next_instance(a, 0, &item);  // starts with a barrier: the initialisation is visible
    if (b < 0) return;
    if (dbl && threadIdx.x == 0) round_fetch<D, CAPPED>(a, smem, bar, b, 0);
    for (int it = 0;; ++it) {
        // buffers alternate, so buffer it & 1 completes its (it >> 1)-th phase now
        const int cur = dbl ? (it & 1) : 0;
        const int bn = next_instance(a, 0, &item);
        if (dbl) {
            if (bn >= 0 && threadIdx.x == 0) round_fetch<D, CAPPED>(a, smem, bar, bn, cur ^ 1);
            const bool ok = __syncthreads_and(mbar_wait(&bar[cur], (uint32_t)(it >> 1) & 1u));
            if (!ok) {
                // the copies did not arrive in time: report this instance and the
                // next one already taken from the list, give every copy issued
                // into this CTA's shared memory another bounded wait to land,
                // and stop taking work (the other CTAs drain the list)
                round_fail<D>(a, b, kTimeout);
                if (bn >= 0) round_fail<D>(a, bn, kTimeout);
                mbar_wait(&bar[cur], (uint32_t)(it >> 1) & 1u);
                if (bn >= 0) mbar_wait(&bar[cur ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
                return;
            }
        }
        round_instance<D, MAXT, CAPPED, BOX>(a, b, smem, cur);
        if (bn < 0) break;
        b = bn;
    }
}

}  // namespace pinmpc
