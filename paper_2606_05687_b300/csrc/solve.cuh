// Device code of the batched parallel-in-horizon ADMM solve (Sec. III).
//
// One CTA solves one instance; warp j owns stage j.  Per iteration (Sec. III,
// the three-block update written in closed form):
//   phase H : extrapolated (Nesterov, with restart) copies of the block-2
//             variables and duals of the warp's stage
//   phase 1 : block 1 -- du_j = J_j (v_j - beta_j) and the lifted state
//             xibar_j = H_{j-1} htilde_{j-1}, then Abar_j xibar_j
//   phase 2 : block 2 -- z_{j+1} = Proj((2 gtilde + g)/3), v_j, and the three
//             dual ascents; per-stage restart-residual partials
//   phase S : every thread folds the partials and takes the same restart
//             decision (Goldstein et al. 2014, fast ADMM with restart)
// Warp j computes xibar_j (the block-1 update of stage j-1) because it owns
// A_j, B_j: J and H are applied in factored (Woodbury) form,
//   J_k w        = g - B^T S_k B g,          g = B^T w_x + w_u,  S_k = (I + B B^T)^{-1}
//   H_{k} h      = D'^{-1}(h - T^T W_k T D'^{-1} h),  T = [A_{k+1} B_{k+1}],
//   W_k = (I/rho + T D'^{-1} T^T)^{-1},  D' = diag(Q_k + rho, R_k + 2 rho)
// (Abar^T Abar = T^T T + blkdiag(0, I)), so only two nx-by-nx caches per
// stage are built.  Every few iterations the active faces of z are read off
// and, when they changed, the equality-constrained LQR on those faces is
// solved by a backward Riccati scan ("polish"), and the KKT certificate is
// evaluated on the polished trajectory.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dims.cuh"

namespace pinmpc {

enum : int { kConverged = 0, kMaxIter = 1, kNonFinite = 2, kBadSet = 3, kTimeout = 4, kBadHorizon = 5, kBadDim = 6,
             kStalled = 7 };

// mode word of one contact after the projection (bit layout):
//   bit 2j   : tangential j clamped at +c_j n     bit 2j+1 : clamped at -c_j n
//   bit 2M   : n clamped at 0 (apex)              bit 2M+1 : n clamped at n_max
//   bit 31   : swing contact
constexpr uint32_t kSwingBit = 0x80000000u;

struct SolveArgs {
    const float* rec;       // packed records [B][irec]
    int irec;               // floats per instance record
    int N;                  // stage stride of this batch (<= N_max): CTA has 32*N threads
    float rho, sigma, kkt_tol, eta, dx, dy;
    int max_iter, check_start, check_every, polish, accel;
    int refine_steps;       // active-set updates after a failed polish
    float refine_alpha;     // projected-gradient step of those updates (scaled units)
    float* out_xi;          // [B][N][NX]
    float* out_u;           // [B][N][NU]
    int* out_status;        // [B]
    int* out_iters;         // [B]
    float* out_kkt;         // [B]
    unsigned long long* out_bits;  // [B][N]
    int* out_npol;          // [B] polish attempts
};

// Shared-memory carve-out (floats), identical on host and device.
template <class D>
struct Smem {
    int sd, Sm, Wm, var, hat, xb, ax, bdu, tmp, Kst, wk, xr, ur, y, wv, red, part, res, modes, lastm, total;
    static constexpr int kTmpVecs = 6;
    // polish work area
    static constexpr int wS = 0, wP = wS + D::NX * D::NX, wp = wP + D::NX * D::NX, ws = wp + D::NX,
                         wSA = ws + D::NX, wSB = wSA + D::NX * D::NX, wBt = wSB + D::NX * D::NU,
                         wM = wBt + D::NX * D::NU, wRHS = wM + D::NU * D::NU,
                         wSe = wRHS + D::NU * (D::NX + 1), wet = wSe + D::NX, wRt = wet + D::NX,
                         wgt = wRt + D::NU, wot = wgt + D::NU, wG = wot + D::NU,
                         wg2 = wG + D::NX * D::NX, wut = wg2 + D::NX, wEnd = wut + D::NU;
    __host__ __device__ explicit Smem(int N) {
        int o = 0;
        auto take = [&o](int n) { int r = o; o += (n + 3) & ~3; return r; };
        sd = take(N * D::SREC);
        Sm = take(N * D::NX * D::NX);
        Wm = take(N * D::NX * D::NX);
        var = take(2 * 5 * N * D::NBP);
        hat = take(5 * N * D::NBP);
        xb = take((N + 1) * D::NBP);
        ax = take(N * D::NBP);
        bdu = take(N * D::NBP);
        tmp = take(N * kTmpVecs * D::NBP);
        Kst = take(N * D::NU * (D::NX + 1));
        wk = take(wEnd);
        xr = take((N + 1) * D::NX);
        ur = take(N * D::NU);
        y = take(N * D::NX);
        wv = take(N * D::NU);
        red = take(64);
        part = take(N);
        res = take(N);
        modes = take(N * D::NC);
        lastm = take(N * D::NC);
        total = o;
    }
    __host__ __device__ int bytes() const { return total * 4; }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Max over the CTA; every thread gets the result.  `red` holds >= 33 floats.
__device__ inline float block_max(float v, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        float t = lane < nw ? red[lane] : -INFINITY;
        t = warp_max(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    float r = red[32];
    __syncthreads();
    return r;
}

// In-place inverse of an n x n SPD matrix (row-major) by Gauss-Jordan
// elimination without pivoting, one warp, n <= 32.
__device__ inline void warp_inverse_spd(float* M, int n, int lane) {
    for (int p = 0; p < n; ++p) {
        __syncwarp();
        const float piv = 1.0f / M[p * n + p];
        const float f = (lane < n && lane != p) ? M[lane * n + p] : 0.0f;
        __syncwarp();
        if (lane < n) M[p * n + lane] = (lane == p ? 1.0f : M[p * n + lane]) * piv;
        __syncwarp();
        if (lane < n && lane != p) {
            for (int c = 0; c < n; ++c) {
                const float cur = (c == p) ? 0.0f : M[lane * n + c];
                M[lane * n + c] = cur - f * M[p * n + c];
            }
        }
    }
    __syncwarp();
}

// Cone coefficient c_j of tangential component j.
template <int CD>
__device__ __forceinline__ float cone_coef(int j, float mu, float dx, float dy) {
    if (CD == 3) return mu;
    // (f_x, f_y, tau_x, tau_y, tau_z): (mu, mu, d_y, d_x, mu*min(d_x, d_y))
    return j < 2 ? mu : (j == 2 ? dy : (j == 3 ? dx : mu * fminf(dx, dy)));
}

// Exact Euclidean projection of a (CD components) onto the generalized
// pyramid {|t_j| <= c_j n, 0 <= n <= nmax}; returns the mode word.
// For fixed n the nearest t_j is clip(a_j, -c_j n, c_j n), leaving the convex
// piecewise-quadratic phi(n) = (n - a_n)^2 + sum_j max(|a_j| - c_j n, 0)^2.
// Its minimiser over the reals lies on the piece S = {j : |a_j|/c_j > n}
// where n = (a_n + sum_S c_j |a_j|) / (1 + sum_S c_j^2); the pieces are the
// super-level sets of the breakpoints, so the candidates are those sets plus
// the empty set, and the minimiser over [0, nmax] is the clamped candidate of
// least phi (phi is strictly convex, so it is unique).
template <int CD>
__device__ uint32_t project_contact(const float* a, float* out, float mu, float nmax, float dx, float dy) {
    constexpr int M = Cone<CD>::M;
    float at[M], c[M], bp[M];
    const float an = a[2];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        at[j] = fabsf(a[Cone<CD>::tang(j)]);
        c[j] = cone_coef<CD>(j, mu, dx, dy);
        bp[j] = c[j] > 0.0f ? at[j] / c[j] : INFINITY;
    }
    float best_n;
    if constexpr (CD == 6) {
        // the pieces in breakpoint order: sorted descending, the candidate
        // sets are nested (the m largest), and phi' is increasing, so the
        // minimiser over the reals is the first candidate m whose n_m is not
        // below the next breakpoint (n_m < b_(m) holds once candidate m - 1
        // failed: n_m is a weighted mean of n_(m-1) and b_(m)); the test is
        // num_m >= b_(m+1) den_m, and one division gives n
        float sb[M], sca[M], scc[M];
#pragma unroll
        for (int j = 0; j < M; ++j) {
            sb[j] = bp[j];
            sca[j] = c[j] * at[j];
            scc[j] = c[j] * c[j];
        }
#pragma unroll
        for (int i = 1; i < M; ++i) {
#pragma unroll
            for (int j = i; j > 0; --j) {
                const bool sw = sb[j] > sb[j - 1];
                const float b0 = sb[j - 1], a0 = sca[j - 1], c0 = scc[j - 1];
                sb[j - 1] = sw ? sb[j] : b0;
                sca[j - 1] = sw ? sca[j] : a0;
                scc[j - 1] = sw ? scc[j] : c0;
                sb[j] = sw ? b0 : sb[j];
                sca[j] = sw ? a0 : sca[j];
                scc[j] = sw ? c0 : scc[j];
            }
        }
        float num = an, den = 1.0f, fnum = an, fden = 1.0f;
        bool found = an >= sb[0];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            num += sca[m];
            den += scc[m];
            const bool ok = !found && (m + 1 == M || num >= sb[m + 1] * den);
            fnum = ok ? num : fnum;
            fden = ok ? den : fden;
            found = found || ok;
        }
        best_n = fminf(fmaxf(fnum / fden, 0.0f), nmax);
    } else {
        best_n = fminf(fmaxf(an, 0.0f), nmax);
        float best_phi = INFINITY;
#pragma unroll
        for (int s = -1; s < M; ++s) {
            float num = an, den = 1.0f;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const bool in = (s >= 0) && (bp[j] >= bp[s < 0 ? 0 : s]);
                num += in ? c[j] * at[j] : 0.0f;
                den += in ? c[j] * c[j] : 0.0f;
            }
            const float n = fminf(fmaxf(num / den, 0.0f), nmax);
            float phi = (n - an) * (n - an);
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float d = fmaxf(at[j] - c[j] * n, 0.0f);
                phi += d * d;
            }
            if (phi < best_phi) { best_phi = phi; best_n = n; }
        }
    }
    uint32_t mode = 0;
    const float n = best_n;
    if (n <= 0.0f) mode |= 1u << (2 * M);
    if (n >= nmax) mode |= 1u << (2 * M + 1);
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const float lim = c[j] * n;
        const float v = a[Cone<CD>::tang(j)];
        float t = v;
        if (v >= lim) { t = lim; mode |= 1u << (2 * j); }
        if (v <= -lim) { t = -lim; mode |= 1u << (2 * j + 1); }
        out[Cone<CD>::tang(j)] = t;
    }
    out[2] = n;
    return mode;
}

enum : int { VZ = 0, VV = 1, VTH = 2, VBE = 3, VLA = 4 };

template <class D>
struct Ctx {
    float *sd, *Sm, *Wm, *var, *hat, *xb, *ax, *bdu, *tmp, *Kst, *wk, *xr, *ur, *y, *wv, *red, *part, *res;
    uint32_t *modes, *lastm;
    int N, Nh;
    float rho, sigma, dx, dy;
    __device__ float* stage(int k) const { return sd + k * D::SREC; }
    __device__ float* V(int buf, int which, int j) const { return var + ((buf * 5 + which) * N + j) * D::NBP; }
    __device__ float* Hh(int which, int j) const { return hat + (which * N + j) * D::NBP; }
    __device__ float* T(int j, int t) const { return tmp + (j * Smem<D>::kTmpVecs + t) * D::NBP; }
    __device__ uint32_t mask(int k) const { return __float_as_uint(stage(k)[D::oMASK]); }
};

__device__ __forceinline__ int face_sign(uint32_t mw, int j) {
    return ((mw >> (2 * j)) & 1u) ? 1 : (((mw >> (2 * j + 1)) & 1u) ? -1 : 0);
}

// ---------------------------------------------------------------------------
// Reduced input map of the polish for one stage: the active faces in the mode
// words fix some components (u = T ut + o).  Writes Bt = Bs T, Rt = T'RsT
// (diagonal because the columns of T have disjoint supports, eliminated
// columns get 1), gt = T'Rs(o - rus), ot = o.
template <class D>
__device__ void polish_reduced_map(const Ctx<D>& c, int k, float* wk, int tid, int nthr) {
    const float* s = c.stage(k);
    float* Bt = wk + Smem<D>::wBt;
    float* Rt = wk + Smem<D>::wRt;
    float* gt = wk + Smem<D>::wgt;
    float* ot = wk + Smem<D>::wot;
    // one thread per (row r, contact q); row r == NX handles Rt, gt, ot
    for (int e = tid; e < (D::NX + 1) * D::NC; e += nthr) {
        const int r = e / D::NC, q = e % D::NC;
        const int base = q * D::CD;
        const uint32_t mw = c.modes[k * D::NC + q];
        const bool swing = (mw & kSwingBit) != 0;
        const bool apex = (mw >> (2 * D::M)) & 1u;
        const bool top = (mw >> (2 * D::M + 1)) & 1u;
        const float mu = s[D::oMU + q];
        const float fms = s[D::oFM + q];
        if (r < D::NX) {
            const float* Brow = s + D::oB + r * D::NU;
            float* Btrow = Bt + r * D::NU;
            if (swing || apex) {
                for (int i = 0; i < D::CD; ++i) Btrow[base + i] = 0.0f;
                continue;
            }
            float ncol = top ? 0.0f : Brow[base + D::NRM];
            for (int j = 0; j < D::M; ++j) {
                const int tj = base + Cone<D::CD>::tang(j);
                const int sg = face_sign(mw, j);
                if (sg == 0) {
                    Btrow[tj] = Brow[tj];
                } else {
                    Btrow[tj] = 0.0f;
                    if (!top) ncol += sg * cone_coef<D::CD>(j, mu, c.dx, c.dy) * Brow[tj];
                }
            }
            Btrow[base + D::NRM] = ncol;
        } else {
            const float* Rs = s + D::oR;
            const float* rus = s + D::oRU;
            if (swing || apex) {
                for (int i = 0; i < D::CD; ++i) { Rt[base + i] = 1.0f; gt[base + i] = 0.0f; ot[base + i] = 0.0f; }
                continue;
            }
            const int nn = base + D::NRM;
            float rn = top ? 1.0f : Rs[nn];
            float gn = top ? 0.0f : -Rs[nn] * rus[nn];
            ot[nn] = top ? fms : 0.0f;
            for (int j = 0; j < D::M; ++j) {
                const int tj = base + Cone<D::CD>::tang(j);
                const int sg = face_sign(mw, j);
                if (sg == 0) {
                    Rt[tj] = Rs[tj];
                    gt[tj] = -Rs[tj] * rus[tj];
                    ot[tj] = 0.0f;
                } else {
                    const float cj = sg * cone_coef<D::CD>(j, mu, c.dx, c.dy);
                    Rt[tj] = 1.0f;
                    gt[tj] = 0.0f;
                    ot[tj] = top ? cj * fms : 0.0f;
                    if (!top) {
                        rn += cj * cj * Rs[tj];
                        gn -= cj * Rs[tj] * rus[tj];
                    }
                }
            }
            Rt[nn] = rn;
            gt[nn] = gn;
        }
    }
}

// Map reduced inputs ut back to full (scaled) inputs for stage k, contact q:
// free components are read from ut, a face-fixed tangential is s_j c_j n,
// n is n_max when the top face is active, swing/apex contacts are 0.
template <class D>
__device__ void expand_contact(const Ctx<D>& c, int k, int q, const float* ut, float* u) {
    const float* s = c.stage(k);
    const int base = q * D::CD;
    const uint32_t mw = c.modes[k * D::NC + q];
    const bool swing = (mw & kSwingBit) != 0;
    const bool apex = (mw >> (2 * D::M)) & 1u;
    const bool top = (mw >> (2 * D::M + 1)) & 1u;
    if (swing || apex) {
        for (int i = 0; i < D::CD; ++i) u[base + i] = 0.0f;
        return;
    }
    const float mu = s[D::oMU + q];
    const int nn = base + D::NRM;
    const float n = top ? s[D::oFM + q] : ut[nn];
    u[nn] = n;
    for (int j = 0; j < D::M; ++j) {
        const int tj = base + Cone<D::CD>::tang(j);
        const int sg = face_sign(mw, j);
        u[tj] = (sg == 0) ? ut[tj] : sg * cone_coef<D::CD>(j, mu, c.dx, c.dy) * n;
    }
}

// Polish: backward Riccati scan of the equality-constrained LQR on the
// current active faces (Riccati recursion of the finite-horizon LQR with the
// reduced inputs ut, u = T ut + o), then the forward rollout into xr (states
// xi_1..xi_Nh at xr + (k+1)*NX) and ur (scaled inputs).  Whole CTA.
//   S = Q_k + P_{k+1}, s = Q_k r_k + p_{k+1}
//   M = Rt + Bt' S Bt,  K = -M^{-1} Bt' S A,  kappa = M^{-1}(Bt'(s - S et) - gt)
//   P_k = A' S (A + Bt K),  p_k = A'(s - S(Bt kappa + et))
template <class D>
__device__ void polish(const Ctx<D>& c) {
    constexpr int NX = D::NX, NU = D::NU, NK = NX + 1;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    float* wk = c.wk;
    float* S = wk + Smem<D>::wS;
    float* P = wk + Smem<D>::wP;
    float* p = wk + Smem<D>::wp;
    float* sv = wk + Smem<D>::ws;
    float* SA = wk + Smem<D>::wSA;
    float* SB = wk + Smem<D>::wSB;
    float* Bt = wk + Smem<D>::wBt;
    float* Mm = wk + Smem<D>::wM;
    float* Se = wk + Smem<D>::wSe;
    float* et = wk + Smem<D>::wet;
    float* Rt = wk + Smem<D>::wRt;
    float* gt = wk + Smem<D>::wgt;
    float* ot = wk + Smem<D>::wot;
    float* G = wk + Smem<D>::wG;
    float* g2 = wk + Smem<D>::wg2;
    float* ut = wk + Smem<D>::wut;
    for (int e = tid; e < NX * NX + NX; e += nthr) {
        if (e < NX * NX) P[e] = 0.0f; else p[e - NX * NX] = 0.0f;
    }
    __syncthreads();
    for (int k = c.Nh - 1; k >= 0; --k) {
        const float* s = c.stage(k);
        const float* A = s + D::oA;
        const float* Bs = s + D::oB;
        float* X = c.Kst + k * NU * NK;  // [NU][NK]: K | kappa
        polish_reduced_map<D>(c, k, wk, tid, nthr);
        __syncthreads();
        for (int e = tid; e < NX + NX * NX + NX; e += nthr) {
            if (e < NX) {
                float acc = s[D::oE + e];
                for (int i = 0; i < NU; ++i) acc = fmaf(Bs[e * NU + i], ot[i], acc);
                et[e] = acc;
            } else if (e < NX + NX * NX) {
                const int q = e - NX, r = q / NX, cc = q % NX;
                S[q] = P[q] + (r == cc ? s[D::oQ + r] : 0.0f);
            } else {
                const int r = e - NX - NX * NX;
                sv[r] = fmaf(s[D::oQ + r], s[D::oRY + r], p[r]);
            }
        }
        __syncthreads();
        for (int e = tid; e < NX * (NX + NU + 1); e += nthr) {
            const int r = e / (NX + NU + 1), cc = e % (NX + NU + 1);
            float acc = 0.0f;
            if (cc < NX) {
                for (int i = 0; i < NX; ++i) acc = fmaf(S[r * NX + i], A[i * NX + cc], acc);
                SA[r * NX + cc] = acc;
            } else if (cc < NX + NU) {
                const int col = cc - NX;
                for (int i = 0; i < NX; ++i) acc = fmaf(S[r * NX + i], Bt[i * NU + col], acc);
                SB[r * NU + col] = acc;
            } else {
                for (int i = 0; i < NX; ++i) acc = fmaf(S[r * NX + i], et[i], acc);
                Se[r] = acc;
            }
        }
        __syncthreads();
        for (int e = tid; e < NU * NU + NU * NK; e += nthr) {
            if (e < NU * NU) {
                const int i = e / NU, j = e % NU;
                float acc = (i == j) ? Rt[i] : 0.0f;
                for (int r = 0; r < NX; ++r) acc = fmaf(Bt[r * NU + i], SB[r * NU + j], acc);
                Mm[e] = acc;
            } else {
                const int q = e - NU * NU, i = q / NK, j = q % NK;
                float acc = 0.0f;
                if (j < NX) {
                    for (int r = 0; r < NX; ++r) acc = fmaf(Bt[r * NU + i], SA[r * NX + j], acc);
                    acc = -acc;
                } else {
                    for (int r = 0; r < NX; ++r) acc = fmaf(Bt[r * NU + i], sv[r] - Se[r], acc);
                    acc -= gt[i];
                }
                X[q] = acc;
            }
        }
        __syncthreads();
        if (warp == 0) {
            // Cholesky M = L L' in place (lower triangle), lane = row
            for (int pp = 0; pp < NU; ++pp) {
                __syncwarp();
                if (lane == pp) Mm[pp * NU + pp] = sqrtf(fmaxf(Mm[pp * NU + pp], 1e-30f));
                __syncwarp();
                const float d = Mm[pp * NU + pp];
                if (lane > pp && lane < NU) Mm[lane * NU + pp] /= d;
                __syncwarp();
                if (lane > pp && lane < NU) {
                    const float l = Mm[lane * NU + pp];
                    for (int cc = pp + 1; cc <= lane; ++cc) Mm[lane * NU + cc] -= l * Mm[cc * NU + pp];
                }
            }
            __syncwarp();
            // forward and backward substitution, lane = right-hand-side column
            if (lane < NK) {
                for (int i = 0; i < NU; ++i) {
                    float acc = X[i * NK + lane];
                    for (int kk = 0; kk < i; ++kk) acc -= Mm[i * NU + kk] * X[kk * NK + lane];
                    X[i * NK + lane] = acc / Mm[i * NU + i];
                }
                for (int i = NU - 1; i >= 0; --i) {
                    float acc = X[i * NK + lane];
                    for (int kk = i + 1; kk < NU; ++kk) acc -= Mm[kk * NU + i] * X[kk * NK + lane];
                    X[i * NK + lane] = acc / Mm[i * NU + i];
                }
            }
        }
        __syncthreads();
        // G = SA + SB K,  g2 = s - Se - SB kappa
        for (int e = tid; e < NX * NX + NX; e += nthr) {
            if (e < NX * NX) {
                const int r = e / NX, cc = e % NX;
                float acc = SA[e];
                for (int i = 0; i < NU; ++i) acc = fmaf(SB[r * NU + i], X[i * NK + cc], acc);
                G[e] = acc;
            } else {
                const int r = e - NX * NX;
                float acc = sv[r] - Se[r];
                for (int i = 0; i < NU; ++i) acc = fmaf(-SB[r * NU + i], X[i * NK + NX], acc);
                g2[r] = acc;
            }
        }
        __syncthreads();
        // P = sym(A' G), p = A' g2
        for (int e = tid; e < NX * NX + NX; e += nthr) {
            if (e < NX * NX) {
                const int r = e / NX, cc = e % NX;
                float a1 = 0.0f, a2 = 0.0f;
                for (int i = 0; i < NX; ++i) {
                    a1 = fmaf(A[i * NX + r], G[i * NX + cc], a1);
                    a2 = fmaf(A[i * NX + cc], G[i * NX + r], a2);
                }
                P[e] = 0.5f * (a1 + a2);
            } else {
                const int r = e - NX * NX;
                float acc = 0.0f;
                for (int i = 0; i < NX; ++i) acc = fmaf(A[i * NX + r], g2[i], acc);
                p[r] = acc;
            }
        }
        __syncthreads();
    }
    // forward rollout with ut = K x + kappa (warp 0); xr[0] = xi_0 is set at setup
    if (warp == 0) {
        for (int k = 0; k < c.Nh; ++k) {
            const float* s = c.stage(k);
            const float* X = c.Kst + k * NU * NK;
            const float* x = c.xr + k * NX;
            if (lane < NU) {
                float acc = X[lane * NK + NX];
                for (int r = 0; r < NX; ++r) acc = fmaf(X[lane * NK + r], x[r], acc);
                ut[lane] = acc;
            }
            __syncwarp();
            if (lane < D::NC) expand_contact<D>(c, k, lane, ut, c.ur + k * NU);
            __syncwarp();
            if (lane < NX) {
                const float* u = c.ur + k * NU;
                float acc = s[D::oE + lane];
                for (int cc = 0; cc < NX; ++cc) acc = fmaf(s[D::oA + lane * NX + cc], x[cc], acc);
                for (int i = 0; i < NU; ++i) acc = fmaf(s[D::oB + lane * NU + i], u[i], acc);
                c.xr[(k + 1) * NX + lane] = acc;
            }
            __syncwarp();
        }
    }
    __syncthreads();
}

// Use the ADMM iterate itself as the output: u from z (feasible by
// construction), xi by forward rollout of u (dynamics-feasible).
template <class D>
__device__ void iterate_as_output(const Ctx<D>& c, int cb) {
    constexpr int NX = D::NX, NU = D::NU;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < c.Nh * NU; e += blockDim.x) {
        const int k = e / NU, i = e % NU;
        c.ur[e] = c.V(cb, VZ, k)[NX + i];
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < c.Nh; ++k) {
            const float* s = c.stage(k);
            const float* x = c.xr + k * NX;
            const float* u = c.ur + k * NU;
            if (lane < NX) {
                float acc = s[D::oE + lane];
                for (int cc = 0; cc < NX; ++cc) acc = fmaf(s[D::oA + lane * NX + cc], x[cc], acc);
                for (int i = 0; i < NU; ++i) acc = fmaf(s[D::oB + lane * NU + i], u[i], acc);
                c.xr[(k + 1) * NX + lane] = acc;
            }
            __syncwarp();
        }
    }
    __syncthreads();
}

// KKT certificate of (xr, ur) in the original units (the reading of the
// KKT residual used throughout): costates y_k = Q_k(xi_{k+1} - r_k) + A_{k+1}'y_{k+1},
// w_k = R_k(u_k - r^u_k) + B_k'y_k, per-contact multipliers mu >= 0 minimising
// ||w + G'mu||^2 + ||diag(g(u)) mu||^2 (cyclic coordinate descent), and
// KKT = max(r_feas, r_stat, r_comp); r_dyn is zero by construction because
// xi is the rollout of u.
template <class D>
__device__ float certificate(const Ctx<D>& c) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const float sig = c.sigma, isig = 1.0f / c.sigma;
    if (warp == 0) {
        for (int k = c.Nh - 1; k >= 0; --k) {
            const float* s = c.stage(k);
            if (lane < NX) {
                float acc = s[D::oQ + lane] * (c.xr[(k + 1) * NX + lane] - s[D::oRY + lane]);
                if (k + 1 < c.Nh) {
                    const float* An = c.stage(k + 1) + D::oA;
                    for (int i = 0; i < NX; ++i) acc = fmaf(An[i * NX + lane], c.y[(k + 1) * NX + i], acc);
                }
                c.y[k * NX + lane] = acc;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    float den = 0.0f, uinf = 0.0f;
    for (int e = tid; e < c.Nh * NU; e += nthr) {
        const int k = e / NU, i = e % NU;
        const float* s = c.stage(k);
        const float rdu = s[D::oR + i] * (c.ur[e] - s[D::oRU + i]) * isig;
        float bty = 0.0f;
        for (int r = 0; r < NX; ++r) bty = fmaf(s[D::oB + r * NU + i], c.y[k * NX + r], bty);
        bty *= isig;
        c.wv[e] = rdu + bty;
        den = fmaxf(den, fmaxf(fabsf(rdu), fabsf(bty)));
        uinf = fmaxf(uinf, fabsf(c.ur[e]) * sig);
    }
    __syncthreads();
    den = block_max(den, c.red);
    uinf = block_max(uinf, c.red);
    float feas = 0.0f, stat = 0.0f, comp = 0.0f;
    for (int e = tid; e < c.Nh * D::NC; e += nthr) {
        const int k = e / D::NC, q = e % D::NC;
        const float* s = c.stage(k);
        const float fmax = s[D::oFM + q] * sig;
        const float* us = c.ur + k * NU + q * CD;
        float u[CD], w[CD];
        for (int i = 0; i < CD; ++i) { u[i] = us[i] * sig; w[i] = c.wv[k * NU + q * CD + i]; }
        if (!((c.mask(k) >> q) & 1u)) {
            float m = 0.0f;
            for (int i = 0; i < CD; ++i) m = fmaxf(m, fabsf(u[i]));
            feas = fmaxf(feas, m / (1.0f + fmax));
            continue;
        }
        const float mu = s[D::oMU + q];
        float cf[M], g[F], lam[F], nrm2[F];
        const float n = u[D::NRM];
        for (int j = 0; j < M; ++j) {
            cf[j] = cone_coef<CD>(j, mu, c.dx, c.dy);
            const float t = u[Cone<CD>::tang(j)];
            g[2 * j] = t - cf[j] * n;
            g[2 * j + 1] = -t - cf[j] * n;
            nrm2[2 * j] = nrm2[2 * j + 1] = 1.0f + cf[j] * cf[j];
        }
        g[2 * M] = -n;
        g[2 * M + 1] = n - fmax;
        nrm2[2 * M] = nrm2[2 * M + 1] = 1.0f;
        float gmax = -INFINITY;
        for (int f = 0; f < F; ++f) { lam[f] = 0.0f; gmax = fmaxf(gmax, g[f]); }
        feas = fmaxf(feas, fmaxf(gmax, 0.0f) / (1.0f + fmax));
        float r[CD];
        float wmax = 0.0f;
        for (int i = 0; i < CD; ++i) { r[i] = w[i]; wmax = fmaxf(wmax, fabsf(w[i])); }
        for (int sweep = 0; sweep < 100; ++sweep) {
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
            // stop once a sweep moves no multiplier by more than 1e-9 (absolute,
            // far below the 1e-6-level residuals certified) or 1e-7 relative
            if (change <= 1e-9f + 1e-7f * wmax) break;
        }
        float rs = 0.0f, rc = 0.0f;
        for (int i = 0; i < CD; ++i) rs = fmaxf(rs, fabsf(r[i]));
        for (int f = 0; f < F; ++f) rc = fmaxf(rc, fabsf(lam[f] * g[f]));
        stat = fmaxf(stat, rs);
        comp = fmaxf(comp, rc);
    }
    feas = block_max(feas, c.red);
    stat = block_max(stat, c.red);
    comp = block_max(comp, c.red);
    return fmaxf(feas, fmaxf(stat / (1.0f + den), comp / (1.0f + uinf)));
}

// Active-set update after a failed polish: the faces of each stance contact
// are read off Proj(u - alpha * grad_u), u the polished (scaled) inputs and
// grad_u = sigma * w the reduced-cost gradient left by the certificate.  A
// violated face is clamped by the projection (added); a face whose multiplier
// came out negative is pushed inside (dropped): one step of a primal
// active-set method done by the projection.  Returns whether any mode word
// changed (CTA-uniform).
template <class D>
__device__ bool refine_modes(const Ctx<D>& c, float alpha) {
    constexpr int NU = D::NU, CD = D::CD;
    bool changed = false;
    for (int e = threadIdx.x; e < c.Nh * D::NC; e += blockDim.x) {
        const int k = e / D::NC, q = e % D::NC;
        if (!((c.mask(k) >> q) & 1u)) continue;
        const float* s = c.stage(k);
        float a[CD], out[CD];
        for (int i = 0; i < CD; ++i)
            a[i] = c.ur[k * NU + q * CD + i] - alpha * c.sigma * c.wv[k * NU + q * CD + i];
        const uint32_t mw = project_contact<CD>(a, out, s[D::oMU + q], s[D::oFM + q], c.dx, c.dy);
        if (mw != c.modes[e]) {
            changed = true;
            c.modes[e] = mw;
        }
    }
    return __syncthreads_or(changed);
}

// Write (xr, ur) and the per-instance results; stages beyond the horizon are 0.
template <class D>
__device__ void write_output(const Ctx<D>& c, const SolveArgs& a, int b, int status, int iters, float kkt,
                             int npol) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int Nv = a.N;
    float* oxi = a.out_xi + (size_t)b * Nv * NX;
    float* ou = a.out_u + (size_t)b * Nv * NU;
    const bool ok = status == kConverged || status == kMaxIter;
    for (int e = tid; e < Nv * NX; e += nthr) {
        const int k = e / NX;
        oxi[e] = (ok && k < c.Nh) ? c.xr[(k + 1) * NX + (e % NX)] : 0.0f;
    }
    for (int e = tid; e < Nv * NU; e += nthr) {
        const int k = e / NU;
        ou[e] = (ok && k < c.Nh) ? c.ur[e] * c.sigma : 0.0f;
    }
    for (int k = tid; k < Nv; k += nthr) {
        unsigned long long bits = 0ull;
        if (ok && k < c.Nh) {
            const float* s = c.stage(k);
            for (int q = 0; q < D::NC; ++q) {
                if (!((c.mask(k) >> q) & 1u)) continue;
                const float fmax = s[D::oFM + q] * c.sigma;
                const float mu = s[D::oMU + q];
                const float* us = c.ur + k * NU + q * CD;
                const float n = us[D::NRM] * c.sigma;
                const float thr = -1e-5f * (1.0f + fmax);
                float g[F];
                for (int j = 0; j < M; ++j) {
                    const float cj = cone_coef<CD>(j, mu, c.dx, c.dy);
                    const float t = us[Cone<CD>::tang(j)] * c.sigma;
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
    if (tid == 0) {
        a.out_status[b] = status;
        a.out_iters[b] = iters;
        a.out_kkt[b] = ok ? kkt : INFINITY;
        a.out_npol[b] = npol;
    }
}

// ---------------------------------------------------------------------------
// Block 1 of one stage (warp j): du_j and xibar_j (+ xibar_N for the last
// stage), then Abar_j xibar_j.
template <class D>
__device__ void block1(const Ctx<D>& c, int j, int lane) {
    constexpr int NX = D::NX, NU = D::NU, NB = D::NB;
    const float rho = c.rho;
    const float* sj = c.stage(j);
    const float* Aj = sj + D::oA;
    const float* Bj = sj + D::oB;
    float* om = c.T(j, 0);
    float* g = c.T(j, 1);
    float* pv = c.T(j, 2);
    float* bdu = c.bdu + j * D::NBP;
    const float* Sj = c.Sm + j * NX * NX;
    {
        const float* vh = c.Hh(VV, j);
        const float* bh = c.Hh(VBE, j);
        for (int i = lane; i < NB; i += 32) om[i] = vh[i] - bh[i];
        __syncwarp();
        if (lane < NU) {
            float acc = om[NX + lane];
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(Bj[r * NU + lane], om[r], acc);
            g[lane] = acc;
        }
        __syncwarp();
        if (lane < NX) {
            float acc = 0.0f;
#pragma unroll
            for (int cc = 0; cc < NU; ++cc) acc = fmaf(Bj[lane * NU + cc], g[cc], acc);
            pv[lane] = acc;
        }
        __syncwarp();
        if (lane < NX) {
            float acc = 0.0f;
#pragma unroll
            for (int cc = 0; cc < NX; ++cc) acc = fmaf(Sj[lane * NX + cc], pv[cc], acc);
            bdu[lane] = acc;  // B du = S B g
        }
        __syncwarp();
        if (lane < NU) {
            float acc = g[lane];
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(-Bj[r * NU + lane], bdu[r], acc);
            bdu[NX + lane] = acc;  // du = g - B' S B g
        }
        __syncwarp();
    }
    if (j >= 1) {
        const float* sp = c.stage(j - 1);
        const float* Wj = c.Wm + j * NX * NX;
        float* w = c.T(j, 3);
        float* cp = c.T(j, 4);
        float* tv = c.T(j, 5);
        const float* zh = c.Hh(VZ, j);
        const float* vh = c.Hh(VV, j);
        const float* lh = c.Hh(VLA, j);
        for (int i = lane; i < NB; i += 32) w[i] = zh[i] - vh[i] - (i < NX ? sj[D::oE + i] : 0.0f) + lh[i];
        __syncwarp();
        const float* zp = c.Hh(VZ, j - 1);
        const float* tp = c.Hh(VTH, j - 1);
        for (int i = lane; i < NB; i += 32) {
            const float qb = i < NX ? sp[D::oQ + i] * sp[D::oRY + i] : sp[D::oR + i - NX] * sp[D::oRU + i - NX];
            const float dp = i < NX ? sp[D::oQ + i] + rho : sp[D::oR + i - NX] + 2.0f * rho;
            float cc = qb + rho * (zp[i] - tp[i]);
            if (i >= NX) cc += rho * w[i];
            cp[i] = cc / dp;
        }
        __syncwarp();
        if (lane < NX) {
            float acc = -w[lane];
#pragma unroll
            for (int cc = 0; cc < NX; ++cc) acc = fmaf(Aj[lane * NX + cc], cp[cc], acc);
#pragma unroll
            for (int cc = 0; cc < NU; ++cc) acc = fmaf(Bj[lane * NU + cc], cp[NX + cc], acc);
            tv[lane] = acc;
        }
        __syncwarp();
        if (lane < NX) {
            float acc = 0.0f;
#pragma unroll
            for (int cc = 0; cc < NX; ++cc) acc = fmaf(Wj[lane * NX + cc], tv[cc], acc);
            pv[lane] = acc;
        }
        __syncwarp();
        float* xbj = c.xb + j * D::NBP;
        for (int i = lane; i < NB; i += 32) {
            float acc = 0.0f;
            if (i < NX) {
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(Aj[r * NX + i], pv[r], acc);
            } else {
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(Bj[r * NU + i - NX], pv[r], acc);
            }
            const float dp = i < NX ? sp[D::oQ + i] + rho : sp[D::oR + i - NX] + 2.0f * rho;
            xbj[i] = cp[i] - acc / dp;
        }
        __syncwarp();
        float* axj = c.ax + j * D::NBP;
        if (lane < NX) {
            float acc = 0.0f;
#pragma unroll
            for (int cc = 0; cc < NX; ++cc) acc = fmaf(Aj[lane * NX + cc], xbj[cc], acc);
#pragma unroll
            for (int cc = 0; cc < NU; ++cc) acc = fmaf(Bj[lane * NU + cc], xbj[NX + cc], acc);
            axj[lane] = acc;
        }
        for (int i = NX + lane; i < NB; i += 32) axj[i] = xbj[i];
        __syncwarp();
    }
    if (j == c.Nh - 1) {
        float* xbN = c.xb + c.Nh * D::NBP;
        const float* zh = c.Hh(VZ, j);
        const float* th = c.Hh(VTH, j);
        for (int i = lane; i < NB; i += 32) {
            const float qb = i < NX ? sj[D::oQ + i] * sj[D::oRY + i] : sj[D::oR + i - NX] * sj[D::oRU + i - NX];
            const float dd = i < NX ? sj[D::oQ + i] + rho : sj[D::oR + i - NX] + rho;
            xbN[i] = (qb + rho * (zh[i] - th[i])) / dd;
        }
        __syncwarp();
    }
}

// Block 2 and the dual ascents of stage j (warp j); new values go to buffer nb.
template <class D>
__device__ void block2(const Ctx<D>& c, int j, int lane, int nb) {
    constexpr int NX = D::NX, NB = D::NB, CD = D::CD;
    const float* sj = c.stage(j);
    const float* xbn = c.xb + (j + 1) * D::NBP;
    const float* axj = c.ax + j * D::NBP;
    const float* bdu = c.bdu + j * D::NBP;
    const float* zh = c.Hh(VZ, j);
    const float* vh = c.Hh(VV, j);
    const float* th = c.Hh(VTH, j);
    const float* bh = c.Hh(VBE, j);
    const float* lh = c.Hh(VLA, j);
    float* arg = c.T(j, 0);
    float gam[2];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
        const int i = lane + 32 * s2;
        gam[s2] = 0.0f;
        if (i < NB) {
            const float eb = i < NX ? sj[D::oE + i] : 0.0f;
            const float g_ = bdu[i] + bh[i] - axj[i] - eb + lh[i];
            const float gt_ = xbn[i] + th[i] + axj[i] + eb - lh[i];
            arg[i] = (2.0f * gt_ + g_) * (1.0f / 3.0f);
            gam[s2] = g_;
        }
    }
    __syncwarp();
    float* zn = c.V(nb, VZ, j);
    if (lane < NX) zn[lane] = arg[lane];
    if (lane < D::NC) {
        const int q = lane;
        uint32_t mw;
        if ((c.mask(j) >> q) & 1u) {
            mw = project_contact<CD>(arg + NX + q * CD, zn + NX + q * CD, sj[D::oMU + q], sj[D::oFM + q], c.dx, c.dy);
        } else {
            for (int i = 0; i < CD; ++i) zn[NX + q * CD + i] = 0.0f;
            mw = kSwingBit;
        }
        c.modes[j * D::NC + q] = mw;
    }
    __syncwarp();
    float* vn = c.V(nb, VV, j);
    float* tn = c.V(nb, VTH, j);
    float* bn = c.V(nb, VBE, j);
    float* ln = c.V(nb, VLA, j);
    float cm = 0.0f, rp = 0.0f;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
        const int i = lane + 32 * s2;
        if (i < NB) {
            const float eb = i < NX ? sj[D::oE + i] : 0.0f;
            const float z = zn[i];
            const float v = 0.5f * (z + gam[s2]);
            const float th_ = th[i] + xbn[i] - z;
            const float be_ = bh[i] + bdu[i] - v;
            const float la_ = lh[i] + z - axj[i] - v - eb;
            vn[i] = v;
            tn[i] = th_;
            bn[i] = be_;
            ln[i] = la_;
            const float d1 = th_ - th[i], d2 = be_ - bh[i], d3 = la_ - lh[i];
            const float d4 = z - zh[i], d5 = v - vh[i], d6 = d4 - d5;
            cm += d1 * d1 + d2 * d2 + d3 * d3 + d4 * d4 + d5 * d5 + d6 * d6;
            rp = fmaxf(rp, fmaxf(fabsf(xbn[i] - z), fmaxf(fabsf(bdu[i] - v), fabsf(z - axj[i] - v - eb))));
        }
    }
    cm = warp_sum(cm);
    rp = warp_max(rp);
    if (lane == 0) {
        c.part[j] = cm;
        c.res[j] = rp;
    }
}

// ---------------------------------------------------------------------------
template <class D>
__global__ void __launch_bounds__(1024, 1) solve_kernel(SolveArgs a, int n_rec) {
    extern __shared__ __align__(16) float smem[];
    constexpr int NX = D::NX, NU = D::NU, NB = D::NB;
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
    const int b = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const float* rec = a.rec + (size_t)b * a.irec;
    const float* tail = rec + (size_t)n_rec * D::SREC;
    const int Nh = __float_as_int(tail[D::tH]);
    c.Nh = (Nh >= 1 && Nh <= a.N) ? Nh : 0;
    if (c.Nh == 0) {
        // invalid horizon: report and write zeros (uniform branch)
        write_output<D>(c, a, b, kBadHorizon, 0, 0.0f, 0);
        return;
    }
    // load the stage records (float4) and the tail
    {
        const float4* src = reinterpret_cast<const float4*>(rec);
        float4* dst = reinterpret_cast<float4*>(c.sd);
        const int n4 = c.Nh * D::SREC / 4;
        for (int e = tid; e < n4; e += nthr) dst[e] = src[e];
    }
    float* x0 = c.xb;  // xibar_0 = [xi_0; u_{-1}]
    for (int i = tid; i < NB; i += nthr) x0[i] = i < NX ? tail[D::tXI0 + i] : tail[D::tUP + i - NX];
    __syncthreads();
    // input checks: finite values, non-empty contact sets
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
        write_output<D>(c, a, b, any_bad ? kNonFinite : kBadSet, 0, 0.0f, 0);
        return;
    }
    // per-stage caches S_j = (I + B B')^{-1}, W_j = (I/rho + T_j D'^{-1}_{j-1} T_j')^{-1}
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
        } else {
            // Abar_0 xibar_0 is constant
            float* ax0 = c.ax;
            if (lane < NX) {
                float acc = 0.0f;
                for (int cc = 0; cc < NX; ++cc) acc = fmaf(sj[D::oA + lane * NX + cc], x0[cc], acc);
                for (int i = 0; i < NU; ++i) acc = fmaf(sj[D::oB + lane * NU + i], x0[NX + i], acc);
                ax0[lane] = acc;
            }
            for (int i = NX + lane; i < NB; i += 32) ax0[i] = x0[i];
        }
    }
    for (int e = tid; e < 2 * 5 * a.N * D::NBP; e += nthr) c.var[e] = 0.0f;
    for (int e = tid; e < 5 * a.N * D::NBP; e += nthr) c.hat[e] = 0.0f;
    for (int e = tid; e < a.N * D::NC; e += nthr) { c.lastm[e] = 0xffffffffu; c.modes[e] = 0u; }
    for (int i = tid; i < NX; i += nthr) c.xr[i] = x0[i];
    __syncthreads();

    int cb = 0, npol = 0;
    float alpha = 1.0f, cprev = INFINITY, wgt = 0.0f;
    bool restart = false;
    for (int m = 1; m <= a.max_iter; ++m) {
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
        if (m >= a.check_start && ((m - a.check_start) % a.check_every) == 0) {
            const bool changed = __syncthreads_or(tid < c.Nh * D::NC && c.modes[tid] != c.lastm[tid]);
            if (!a.polish || changed) {
                if (tid < c.Nh * D::NC) c.lastm[tid] = c.modes[tid];
                __syncthreads();
                if (a.polish) { polish<D>(c); ++npol; } else iterate_as_output<D>(c, cb);
                float kkt = certificate<D>(c);
                for (int r = 0; a.polish && kkt > a.kkt_tol && r < a.refine_steps; ++r) {
                    if (!refine_modes<D>(c, a.refine_alpha)) break;
                    polish<D>(c);
                    ++npol;
                    kkt = certificate<D>(c);
                }
                if (kkt <= a.kkt_tol) {
                    write_output<D>(c, a, b, kConverged, m, kkt, npol);
                    return;
                }
            }
        }
    }
    iterate_as_output<D>(c, cb);
    const float kkt = certificate<D>(c);
    write_output<D>(c, a, b, kkt <= a.kkt_tol ? kConverged : kMaxIter, a.max_iter, kkt, npol);
}

// ---------------------------------------------------------------------------
// Pack/scale (A0): copy the caller's instance-major arrays into one record per
// instance, scaling inputs by sigma: B -> sigma B, R -> sigma^2 R,
// r^u -> r^u/sigma, n_max -> n_max/sigma, u_{-1} -> u_{-1}/sigma.
struct PackArgs {
    const float *A, *Bm, *e, *Q, *R, *ry, *ru, *mu, *fmax, *xi0, *u_prev;
    const uint32_t* mask;
    const int32_t* horizon;
    const float* C;          // [B][S][NX] diagonal output map, or null (C = I)
    const int32_t* nu;       // [B] inputs present per instance, or null (all)
    const float *xlo, *xhi;  // [B][S][NX] state boxes of xi_{k+1} (either may be null: unbounded)
    float* xbox;             // [B][n_rec][2][NX] packed boxes, or null (no boxes this batch)
    int N;          // stages read per instance
    int S;          // stages between consecutive instances in the caller's arrays (>= N)
    int n_rec;      // stage capacity of a record
    int irec;       // floats per record
    float sigma;
    float* rec;
};

template <class D>
__global__ void pack_kernel(PackArgs a) {
    constexpr int NX = D::NX, NU = D::NU, NC = D::NC;
    const int b = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const int N = a.N;
    float* rec = a.rec + (size_t)b * a.irec;
    const float sg = a.sigma, isg = 1.0f / a.sigma;
    const size_t sb = (size_t)b * a.S;
    // inputs present: the first nu[b] / CD contacts; a count that is not a
    // multiple of CD in [0, NU] leaves every contact out and flags the instance
    const int nub = a.nu ? a.nu[b] : NU;
    const bool nu_ok = nub >= 0 && nub <= NU && nub % D::CD == 0;
    const uint32_t present = nu_ok ? (nub / D::CD >= 32 ? 0xffffffffu : ((1u << (nub / D::CD)) - 1u)) : 0u;
    // inputs through the read-only path (they never alias the records), so
    // the unrolled copy loops keep several loads in flight per thread
#pragma unroll 4
    for (int e = tid; e < N * NX * NX; e += nthr) {
        const int k = e / (NX * NX), r = e % (NX * NX);
        rec[k * D::SREC + D::oA + r] = __ldg(a.A + sb * NX * NX + e);
    }
#pragma unroll 4
    for (int e = tid; e < N * NX * NU; e += nthr) {
        const int k = e / (NX * NU), r = e % (NX * NU);
        rec[k * D::SREC + D::oB + r] = sg * __ldg(a.Bm + sb * NX * NU + e);
    }
    for (int e = tid; e < N * NX; e += nthr) {
        const int k = e / NX, r = e % NX;
        float* s = rec + k * D::SREC;
        s[D::oE + r] = a.e ? __ldg(a.e + sb * NX + e) : 0.0f;
        const float q = __ldg(a.Q + sb * NX + e), ry = __ldg(a.ry + sb * NX + e);
        if (a.C) {
            // ||c x - r||^2_q = ||x - r / c||^2_{c^2 q} (a zero c drops the component's cost)
            const float cc = __ldg(a.C + sb * NX + e);
            s[D::oQ + r] = cc * cc * q;
            s[D::oRY + r] = cc != 0.0f ? ry / cc : 0.0f;
        } else {
            s[D::oQ + r] = q;
            s[D::oRY + r] = ry;
        }
    }
    for (int e = tid; e < N * NU; e += nthr) {
        const int k = e / NU, r = e % NU;
        float* s = rec + k * D::SREC;
        s[D::oR + r] = sg * sg * __ldg(a.R + sb * NU + e);
        s[D::oRU + r] = a.ru ? __ldg(a.ru + sb * NU + e) * isg : 0.0f;
    }
    for (int e = tid; e < N * NC; e += nthr) {
        const int k = e / NC, r = e % NC;
        float* s = rec + k * D::SREC;
        s[D::oMU + r] = __ldg(a.mu + sb * NC + e);
        s[D::oFM + r] = __ldg(a.fmax + sb * NC + e) * isg;
    }
    for (int k = tid; k < N; k += nthr) {
        float* s = rec + k * D::SREC;
        s[D::oMASK] = __uint_as_float(a.mask[sb + k] & present);
        for (int r = D::oMASK + 1; r < D::SREC; ++r) s[r] = 0.0f;
    }
    if (a.xbox) {
        float* bx = a.xbox + (size_t)b * a.n_rec * 2 * NX;
        for (int e = tid; e < N * NX; e += nthr) {
            const int k = e / NX, r = e % NX;
            bx[(k * 2 + 0) * NX + r] = a.xlo ? __ldg(a.xlo + sb * NX + e) : -INFINITY;
            bx[(k * 2 + 1) * NX + r] = a.xhi ? __ldg(a.xhi + sb * NX + e) : INFINITY;
        }
    }
    float* tail = rec + (size_t)a.n_rec * D::SREC;
    for (int i = tid; i < D::TAIL; i += nthr) {
        float v = 0.0f;
        if (i < NX) v = a.xi0[(size_t)b * NX + i];
        else if (i < NX + NU) v = a.u_prev ? a.u_prev[(size_t)b * NU + i - NX] * isg : 0.0f;
        else if (i == D::tH) v = __int_as_float(a.horizon ? a.horizon[b] : N);
        else if (i == D::tFLAG) v = __int_as_float(nu_ok ? 0 : 4);
        tail[i] = v;
    }
}

}  // namespace pinmpc
