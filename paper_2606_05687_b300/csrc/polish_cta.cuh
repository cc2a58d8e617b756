// Polish, certificate and active-set refinement with one 128-thread CTA per
// instance (4 warps), after each ADMM round.
//   polish:      the active faces of the latest projection fix some input
//                components (u = T ut + o); the equality-constrained LQR on
//                the remaining free components is solved by a backward
//                Riccati scan (full-size per-stage systems whose eliminated
//                columns are unit vectors, Gauss-Jordan over the free pivots
//                only, operands in registers and 80-byte shared rows; with
//                state boxes, active bounds as equality rows where inputs
//                reach them, else an augmented Lagrangian), then a forward
//                rollout;
//   certificate: costate scan, stationarity, per-contact nonnegative
//                multipliers (cyclic coordinate descent) and the KKT
//                residual this implementation stops on (the paper gives only an
//                iteration budget);
//   refinement:  faces re-read from the projection of u - alpha sigma w, then
//                polish again (at most refine_steps times).
// Stage records are staged through shared memory with a register prefetch
// of the next stage.
#pragma once
#include "polish.cuh"

namespace pinmpc {

constexpr int kPT = 128;  // threads per polish CTA
constexpr int kPivotBlock = 4;  // pivots eliminated per Gauss-Jordan step (divides nu)

// Approximate reciprocal (PTX rcp.approx, relative error below 2^-22); used
// for elimination pivots, whose rounding is far below the certificate's tolerance.
__device__ __forceinline__ float rcp_approx(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

template <class D>
struct CtaSmem {
    static constexpr int NX = D::NX, NU = D::NU, NK = NX + 1;
    // padded row length: 16-byte aligned rows (float4), and consecutive rows
    // start in different bank quads, so lanes reading different rows as
    // float4 do not conflict
    static constexpr int XP = 20;
    static_assert(NK <= 16 && NU <= 32, "polish layout assumes nx < 16 and nu <= 32");
    static constexpr int al(int x) { return (x + 15) & ~15; }
    // backward scan (rows of XP floats):
    //   Xp = [P | p] of the stage after, S = Q + sym(P), AT = A', BtT = Bt' (reduced map),
    //   SBT = (S Bt)', SAT = (S A)', K16 = [K | kappa], GR = [G | g2]
    static constexpr int oXp = 0, oS = al(oXp + NX * XP), oAT = al(oS + XP * XP), oBtT = al(oAT + NX * XP),
                         oRt = al(oBtT + NU * XP), ogt = al(oRt + 32), oot = al(ogt + 32), oet = al(oot + 32),
                         osv = al(oet + XP), odv = al(osv + XP), oSBT = al(odv + XP), oSAT = al(oSBT + NU * XP),
                         oK16 = al(oSAT + NX * XP), oGR = al(oK16 + NU * XP), opcol = al(oGR + NX * XP),
                         oprow = al(opcol + 128), ofree = al(oprow + 4 * 48), oMC = al(ofree + 4),
                         opcb = al(oMC + (NU + kNCB + NK) * 32),
                         // exactly held state bounds (state-box variant): per slot of the stage the
                         // multiplier gains [K_lambda | kappa_lambda], the row F on x_{k+1}, its
                         // input row F Bt, feedback row -F A and affine term d - F et; the rows
                         // carried back to earlier stages (two lists, read and written in turn),
                         // with their bound and origin (stage * NX + component)
                         oKl = al(opcb + 2 * kPivotBlock * 32), osF = al(oKl + kNCB * XP),
                         osc = al(osF + kNCB * XP), osfb = al(osc + kNCB * 32), osaff = al(osfb + kNCB * XP),
                         opF = al(osaff + 2 * kNCB), opd = al(opF + 2 * kNPend * XP),
                         opo = al(opd + 2 * kNPend), opn = al(opo + 2 * kNPend),
                         oScanEnd = al(opn + 4),
                         // forward rollout and certificate
                         oK = oScanEnd, out = al(oK + (NU + kNCB) * NK), obuf0 = al(out + NU), obuf1 = al(obuf0 + D::SREC),
                         ored = al(obuf1 + D::SREC), ostep = al(ored + 32), oFixed = al(ostep + 16);  // ostep: the refinement's state
    static_assert(NU + NK <= 48, "pivot-row buffer");
    // column stride of the column-major [M | RHS]: a multiple of 4 at least NU
    // with an odd number of float4s, so consecutive columns read as float4
    // fall in different bank quads
    // (with room for the kNCB rows of exactly held state bounds)
    static constexpr int NRB = NU + kNCB;
    static constexpr int CP = (((NRB + 3) / 4) % 2 == 1) ? 4 * ((NRB + 3) / 4) : 4 * ((NRB + 3) / 4) + 4;
    static_assert(CP <= 32, "column buffer");
    int xr, ur, y, wv, modes, cmu, cfm, cmask, nub, rhob, dprev, dlast, sbits, dbits, albits, sorig, total;
    __host__ __device__ explicit CtaSmem(int N) {
        int o = oFixed;
        auto take = [&o](int n) { int r = o; o += (n + 3) & ~3; return r; };
        xr = take((N + 1) * NX);
        ur = take(N * NU);
        // the certificate runs after the scan: costates and the gradient
        // reuse scan buffers when they fit
        y = (N * NX <= (oK16 - oSBT)) ? oSBT : take(N * NX);
        wv = (N * NU <= (oprow - oK16)) ? oK16 : take(N * NU);
        modes = take(N * D::NC);
        cmu = take(N * D::NC);
        cfm = take(N * D::NC);
        cmask = take(N);
        nub = take(N * NX);   // signed multipliers of the active state bounds
        rhob = take(N * NX);  // their augmented-Lagrangian penalties
        dprev = take(N * NX); // their violations after the previous scan
        dlast = take(N * NX); // and signed, when the penalty stayed (0: not comparable)
        sbits = take(N);      // active state bounds per stage (bit i lower, 16 + i upper)
        dbits = take(N);      // of those, the components held exactly by the last scan (bit i)
        albits = take(N);     // and those left to the augmented Lagrangian by this polish
        sorig = take(N * kNCB);  // origin (stage * NX + component) of each stage's exact rows, -1 if none
        total = o;
    }
};

// Block-strided register prefetch of FLOATS floats (float4 granules).
template <int FLOATS, bool READONLY>
struct CPrefetch {
    static constexpr int V4 = FLOATS / 4;
    static constexpr int PER = (V4 + kPT - 1) / kPT;
    float4 r[PER];
    __device__ __forceinline__ void load(const float* src, int tid) {
        const float4* s = reinterpret_cast<const float4*>(src);
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int idx = tid + kPT * t;
            if (idx < V4) r[t] = READONLY ? __ldg(s + idx) : s[idx];
        }
    }
    __device__ __forceinline__ void store(float* dst, int tid) const {
        float4* d = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int idx = tid + kPT * t;
            if (idx < V4) d[idx] = r[t];
        }
    }
};

template <class D>
struct CCtx {
    const float* rec;
    float* sm;
    CtaSmem<D> L;
    uint32_t* modes;
    float* K;  // global gains [N][NU][NK]
    int Nh, tid, lane, warp;
    float sigma, dx, dy;
    float kc;  // certificate normalisation constant kkt_tol_abs / kkt_tol (1 by default)
    const float* box;  // this instance's state boxes [N][2][NX], or null
    __device__ CCtx(int N) : L(N) {}
    __device__ const float* grec(int k) const { return rec + (size_t)k * D::SREC; }
    __device__ float* buf(int k) const { return sm + ((k & 1) ? CtaSmem<D>::obuf1 : CtaSmem<D>::obuf0); }
    __device__ float* xr() const { return sm + L.xr; }
    __device__ float* ur() const { return sm + L.ur; }
    __device__ float* y() const { return sm + L.y; }
    __device__ float* wv() const { return sm + L.wv; }
    __device__ float mu(int k, int q) const { return sm[L.cmu + k * D::NC + q]; }
    __device__ float fms(int k, int q) const { return sm[L.cfm + k * D::NC + q]; }
    __device__ uint32_t mask(int k) const { return __float_as_uint(sm[L.cmask + k]); }
    __device__ float* nub() const { return sm + L.nub; }
    __device__ float* rhob() const { return sm + L.rhob; }
    __device__ float* dprev() const { return sm + L.dprev; }
    __device__ float* dlast() const { return sm + L.dlast; }
    __device__ uint32_t* sbits() const { return reinterpret_cast<uint32_t*>(sm + L.sbits); }
    __device__ uint32_t* dbits() const { return reinterpret_cast<uint32_t*>(sm + L.dbits); }
    __device__ uint32_t* albits() const { return reinterpret_cast<uint32_t*>(sm + L.albits); }
    __device__ int* sorig() const { return reinterpret_cast<int*>(sm + L.sorig); }
    // the bound of component i of xi_{k+1} that is active (upper if both), and whether any is
    __device__ bool box_active(int k, int i, float* bound, bool* upper) const {
        const uint32_t sb = sbits()[k];
        const bool hi = (sb >> (16 + i)) & 1u, lo = (sb >> i) & 1u;
        if (!(hi || lo)) return false;
        *upper = hi;
        *bound = box[(k * 2 + (hi ? 1 : 0)) * D::NX + i];
        return true;
    }
};

// CTA-wide maxima of several values at once (one pair of barriers); the
// reduction buffer holds 32 floats, 4 warps x NV values
template <class D, int NV>
__device__ void cta_max_n(const CCtx<D>& c, float (&v)[NV]) {
    static_assert(NV * (kPT / 32) <= 32, "reduction buffer");
    float* red = c.sm + CtaSmem<D>::ored;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_max(v[i]);
    __syncthreads();
    if (c.lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) red[i * (kPT / 32) + c.warp] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float r = red[i * (kPT / 32)];
#pragma unroll
        for (int w = 1; w < kPT / 32; ++w) r = fmaxf(r, red[i * (kPT / 32) + w]);
        v[i] = r;
    }
}

template <class D>
__device__ float cta_max(const CCtx<D>& c, float v) {
    float* red = c.sm + CtaSmem<D>::ored;
    v = warp_max(v);
    __syncthreads();
    if (c.lane == 0) red[c.warp] = v;
    __syncthreads();
    float r = red[0];
#pragma unroll
    for (int w = 1; w < kPT / 32; ++w) r = fmaxf(r, red[w]);
    return r;
}

// x_{k+1} = A x_k + Bs u_k + e_k for threads < NX (stage record s in shared memory)
template <class D>
__device__ __forceinline__ void cta_rollout_step(const CCtx<D>& c, const float* s, int k) {
    constexpr int NX = D::NX, NU = D::NU;
    if (c.tid < NX) {
        const float* xk = c.xr() + k * NX;
        const float* u = c.ur() + k * NU;
        float acc = s[D::oE + c.tid];
#pragma unroll
        for (int cc = 0; cc < NX; ++cc) acc = fmaf(s[D::oA + c.tid * NX + cc], xk[cc], acc);
#pragma unroll
        for (int i = 0; i < NU; ++i) acc = fmaf(s[D::oB + c.tid * NU + i], u[i], acc);
        c.xr()[(k + 1) * NX + c.tid] = acc;
    }
}

// first 4 ceil(NX/4) entries of a 16-byte aligned row into registers
template <int NX>
__device__ __forceinline__ void load_row(const float* src, float (&v)[4 * ((NX + 3) / 4)]) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int q = 0; q < (NX + 3) / 4; ++q) {
        const float4 t = s4[q];
        v[4 * q + 0] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

// dot of the first NX entries of a 16-byte aligned row with a register vector
template <int NX>
__device__ __forceinline__ float dot_reg(const float* a, const float (&v)[4 * ((NX + 3) / 4)]) {
    const float4* a4 = reinterpret_cast<const float4*>(a);
    float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int q = 0; q < (NX + 3) / 4; ++q) {
        const float4 u = a4[q];
        if (4 * q + 0 < NX) s0 = fmaf(u.x, v[4 * q + 0], s0);
        if (4 * q + 1 < NX) s1 = fmaf(u.y, v[4 * q + 1], s1);
        if (4 * q + 2 < NX) s0 = fmaf(u.z, v[4 * q + 2], s0);
        if (4 * q + 3 < NX) s1 = fmaf(u.w, v[4 * q + 3], s1);
    }
    return s0 + s1;
}

// Backward Riccati scan + forward rollout of one instance by one CTA;
// returns the number of free pivots eliminated (in every thread).
//
// Stage k of the scan, with (P, p) of stage k+1 (zero after the last stage)
// and the reduced input map u = T ut + o of the stage's faces (Bt = Bs T,
// Rt = T'RsT diagonal, gt = T'Rs(o - rus); an eliminated column has Bt = 0,
// Rt = 1, gt = 0):
//   S = Q + P, s = Q ry + p, et = e + Bs o,
//   M = Rt + Bt'S Bt, [K | kappa] = M^{-1} [-Bt'S A | Bt'(s - S et) - gt],
//   G = S A + S Bt K, g2 = s - S et - S Bt kappa, P = A'G, p = A'g2.
// M is kept at full size: an eliminated column makes row and column of M a
// unit vector and its row of the right-hand side zero, so its elimination
// step is skipped and its gains come out zero.
// With state bounds (BOX), the rows F of active bounds on x_{k+1} that the
// stage's free inputs reach (F = e_i for a bound of this stage, or a row
// carried back from a later stage) are equality rows of the stage's system,
//   [M    (F Bt)'] [ut    ]   [-Bt'S A | Bt'(s - S et) - gt]
//   [F Bt   0    ] [lambda] = [ -F A   | d - F et          ]  [x; 1],
// lambda = K_lambda x + kappa_lambda their multipliers (L = f + lambda'(F x_{k+1} - d)),
// and then G += F'K_lambda, g2 -= F'kappa_lambda.
template <class D, bool BOX = false>
__device__ int cta_polish(const CCtx<D>& c) {
    constexpr int NX = D::NX, NU = D::NU, NK = NX + 1;
    using CS = CtaSmem<D>;
    constexpr int XP = CS::XP;
    const int tid = c.tid;
    float* sm = c.sm;
    float* Xp = sm + CS::oXp;
    float* S = sm + CS::oS;
    float* AT = sm + CS::oAT;
    float* BtT = sm + CS::oBtT;
    float* Rt = sm + CS::oRt;
    float* gts = sm + CS::ogt;
    float* ots = sm + CS::oot;
    float* et = sm + CS::oet;
    float* sv = sm + CS::osv;
    float* dv = sm + CS::odv;
    float* SBT = sm + CS::oSBT;
    float* SAT = sm + CS::oSAT;
    float* K16 = sm + CS::oK16;
    float* GR = sm + CS::oGR;
    uint32_t* freep = reinterpret_cast<uint32_t*>(sm + CS::ofree);
    float* Ks = sm + CS::oK;
    int npiv = 0;
    // all scan buffers start at zero: their padding stays zero
    for (int e = tid; e < CS::oScanEnd; e += kPT) sm[e] = 0.0f;
    CPrefetch<D::SREC, true> pf;
    pf.load(c.grec(c.Nh - 1), tid);
    for (int k = c.Nh - 1; k >= 0; --k) {
        float* s = c.buf(k);
        __syncthreads();
        pf.store(s, tid);
        __syncthreads();
        if (k > 0) pf.load(c.grec(k - 1), tid);
        // (1) warp 0: reduced input map (one column per lane), free columns, et.
        //     warps 1..3: S = Q + sym(P), s = Q ry + p, AT = A' (with state
        //     bounds: AT only, S and s once the bounds' cost terms are set)
        if (tid < 32) {
            bool fr = false;
            if (tid < NU) {
                float bt[NX], rt, gt, ot;
                reduced_column<D>(c, s, c.modes[k * D::NC + tid / D::CD], tid, bt, rt, gt, ot);
                float4* row = reinterpret_cast<float4*>(BtT + tid * XP);
#pragma unroll
                for (int q = 0; q < XP / 4; ++q) {
                    const int r = 4 * q;
                    row[q] = make_float4(r < NX ? bt[r] : 0.0f, r + 1 < NX ? bt[r + 1] : 0.0f,
                                         r + 2 < NX ? bt[r + 2] : 0.0f, r + 3 < NX ? bt[r + 3] : 0.0f);
                }
#pragma unroll
                for (int r = 0; r < NX; ++r) fr |= (bt[r] != 0.0f);
                fr |= (rt != 1.0f) || (gt != 0.0f);
                Rt[tid] = rt;
                gts[tid] = gt;
                ots[tid] = ot;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, fr);
            if (tid == 0) freep[0] = ball;
            __syncwarp();
            if (tid < NX) {
                float acc = s[D::oE + tid];
#pragma unroll
                for (int i = 0; i < NU; ++i) acc = fmaf(s[D::oB + tid * NU + i], ots[i], acc);
                et[tid] = acc;
            }
        } else {
            for (int e = tid - 32; e < NX * XP + NX + NX * NX; e += kPT - 32) {
                if (e < NX * XP) {
                    if (!BOX) {
                        const int r = e / XP, cc = e % XP;
                        S[e] = cc < NX ? 0.5f * (Xp[r * XP + cc] + Xp[cc * XP + r]) + (r == cc ? s[D::oQ + r] : 0.0f)
                                       : 0.0f;
                    }
                } else if (e < NX * XP + NX) {
                    if (!BOX) {
                        const int r = e - NX * XP;
                        sv[r] = fmaf(s[D::oQ + r], s[D::oRY + r], Xp[r * XP + NX]);
                    }
                } else {
                    const int f = e - NX * XP - NX, i = f / NX, cc = f % NX;
                    AT[cc * XP + i] = s[D::oA + f];
                }
            }
        }
        __syncthreads();
        uint32_t cmask = 0u;  // constraint slots in use
        if constexpr (BOX) {
            // Active state bounds.  A bound b_i on component i of xi_{k+1} is
            // the row F = e_i on x_{k+1} = F (A x + Bt ut + et), held exactly
            // by this stage when F Bt is nonzero: an equality row F Bt ut =
            // d - F A x - F et of the stage's KKT system.  When F Bt = 0 (no
            // free input of the stage moves it) the row is carried back as
            // F A on x_k, d - F et, to the next stage, and so on until a
            // stage's inputs reach it.  Rows are taken in turn (carried rows,
            // then the stage's own bounds in component order) while they add
            // rank (Gram-Schmidt residual above 1e-6 of the norm), up to kNCB;
            // a bound not held exactly gets the augmented Lagrangian's terms
            // in its stage cost, p_i/2 (x_i - b_i + nu_i / p_i)^2, i.e.
            // Q_i + p_i and Q_i r_i + p_i b_i - nu_i (now, or from the next
            // scan when it was carried).
            float* sF = sm + CS::osF;
            float* sc = sm + CS::osc;
            float* sfb = sm + CS::osfb;
            float* saff = sm + CS::osaff;
            int* pn = reinterpret_cast<int*>(sm + CS::opn);
            const int rd = k & 1;  // the list read at this stage; the other is written
            float* pFr = sm + CS::opF + rd * kNPend * XP;
            float* pFw = sm + CS::opF + (1 - rd) * kNPend * XP;
            float* pdr = sm + CS::opd + rd * kNPend;
            float* pdw = sm + CS::opd + (1 - rd) * kNPend;
            int* por = reinterpret_cast<int*>(sm + CS::opo) + rd * kNPend;
            int* pow_ = reinterpret_cast<int*>(sm + CS::opo) + (1 - rd) * kNPend;
            if (tid < 32) {
                const int lane = tid;
                if (lane == 0) c.dbits()[k] = 0u;
                if (lane < kNCB) c.sorig()[k * kNCB + lane] = -1;
                __syncwarp();
                float q[kNCB];
                int nd = 0, nw = 0;
                uint32_t alm = 0u;  // the stage's own bounds held by the augmented Lagrangian
                const int nr = (k + 1 < c.Nh) ? pn[rd] : 0;
                const uint32_t al_k = c.albits()[k];
                // state rows the stage's inputs act on (nonzero rows of B)
                bool brow = false;
                if (lane < NX)
                    for (int a = 0; a < NU; ++a) brow |= s[D::oB + lane * NU + a] != 0.0f;
                const uint32_t bmask = __ballot_sync(0xffffffffu, brow);
                for (int e = 0; e < nr + NX; ++e) {
                    // candidate row F (lane r < NX holds F_r), bound d, origin
                    float Fr, d;
                    int org;
                    if (e < nr) {
                        Fr = lane < NX ? pFr[e * XP + lane] : 0.0f;
                        d = pdr[e];
                        org = por[e];
                    } else {
                        const int i = e - nr;
                        float bnd;
                        bool up;
                        if (!c.box_active(k, i, &bnd, &up)) continue;  // uniform
                        if ((al_k >> i) & 1u) {
                            alm |= 1u << i;
                            continue;
                        }
                        Fr = lane == i ? 1.0f : 0.0f;
                        d = bnd;
                        org = k * NX + i;
                    }
                    // its input row F Bt (lane a: F against Bt's column a)
                    float v = 0.0f;
#pragma unroll
                    for (int r = 0; r < NX; ++r) {
                        const float fr = __shfl_sync(0xffffffffu, Fr, r);
                        if (lane < NU) v = fmaf(fr, BtT[lane * XP + r], v);
                    }
                    const float n2 = warp_sum(v * v);
                    bool keep = false;
                    if (n2 > 0.0f && nd < kNCB) {
                        float w = v;
#pragma unroll
                        for (int t = 0; t < kNCB; ++t) {
                            if (t < nd) {
                                const float pr = warp_sum(w * q[t]);
                                w = fmaf(-pr, q[t], w);
                            }
                        }
                        const float r2 = warp_sum(w * w);
                        keep = r2 > 1e-6f * n2;
                        if (keep) {
                            const float inv = rsqrtf(r2);
#pragma unroll
                            for (int t = 0; t < kNCB; ++t)
                                if (t == nd) q[t] = w * inv;
                        }
                    }
                    // F A and F et (lane cc < NX: column cc of F A)
                    float fa = 0.0f, fe = 0.0f;
#pragma unroll
                    for (int r = 0; r < NX; ++r) {
                        const float fr = __shfl_sync(0xffffffffu, Fr, r);
                        if (lane < NX) fa = fmaf(fr, s[D::oA + r * NX + lane], fa);
                        fe = fmaf(fr, et[r], fe);
                    }
                    if (keep) {
                        if (lane < NX) {
                            sF[nd * XP + lane] = Fr;
                            sfb[nd * XP + lane] = -fa;
                        }
                        if (lane < NU) sc[nd * 32 + lane] = v;
                        if (lane == 0) {
                            saff[nd] = d - fe;
                            c.sorig()[k * kNCB + nd] = org;
                            c.dbits()[org / NX] |= 1u << (org % NX);
                        }
                        ++nd;
                    } else if (n2 == 0.0f && k > 0 && nw < kNPend &&
                               warp_sum(lane < NX && ((bmask >> lane) & 1u) ? fa * fa : 0.0f) >=
                                   1e-2f * warp_sum(lane < NX ? fa * fa : 0.0f)) {
                        // carried to stage k - 1 as the row F A on x_k, when the
                        // inputs act on it there at scale (a position behind its
                        // velocity sees them only through dt: its multiplier form
                        // would cancel in FP32, so it stays with the augmented
                        // Lagrangian)
                        if (lane < NX) pFw[nw * XP + lane] = fa;
                        if (lane == 0) {
                            pdw[nw] = d - fe;
                            pow_[nw] = org;
                        }
                        ++nw;
                    } else if (org / NX == k) {
                        alm |= 1u << (org % NX);
                    } else if (lane == 0) {
                        atomicOr(c.albits() + org / NX, 1u << (org % NX));
                    }
                    __syncwarp();
                }
                if (lane == 0) pn[1 - rd] = nw;
                if (lane < NX && ((alm >> lane) & 1u)) {
                    float bnd;
                    bool up;
                    c.box_active(k, lane, &bnd, &up);
                    const float qq = s[D::oQ + lane], pen = c.rhob()[k * NX + lane];
                    const float qn = qq + pen;
                    s[D::oRY + lane] = (fmaf(qq, s[D::oRY + lane], pen * bnd) - c.nub()[k * NX + lane]) / qn;
                    s[D::oQ + lane] = qn;
                }
                if (lane == 0) pn[2] = nd;
            }
            __syncthreads();
            for (int e = tid; e < NX * XP + NX; e += kPT) {
                if (e < NX * XP) {
                    const int r = e / XP, cc = e % XP;
                    S[e] = cc < NX ? 0.5f * (Xp[r * XP + cc] + Xp[cc * XP + r]) + (r == cc ? s[D::oQ + r] : 0.0f) : 0.0f;
                } else {
                    const int r = e - NX * XP;
                    sv[r] = fmaf(s[D::oQ + r], s[D::oRY + r], Xp[r * XP + NX]);
                }
            }
            cmask = (1u << pn[2]) - 1u;
            __syncthreads();
        }
        const uint32_t fmask = freep[0];
        npiv += __popc(fmask);
        // (2) SBT = (S Bt)', SAT = (S A)', Se: thread (column, row group) with
        //     its 16-float column in registers
        {
            constexpr int W2 = NU + NX + 1, G2 = kPT / W2, R2 = (NX + G2 - 1) / G2;
            const int col = tid % W2, g = tid / W2;
            if (g < G2) {
                const float* src = col < NU ? BtT + col * XP : (col < NU + NX ? AT + (col - NU) * XP : et);
                float v[4 * ((NX + 3) / 4)];
                load_row<NX>(src, v);
#pragma unroll
                for (int t = 0; t < R2; ++t) {
                    const int r = g * R2 + t;
                    if (r < NX) {
                        const float acc = dot_reg<NX>(S + r * XP, v);
                        if (col < NU) SBT[col * XP + r] = acc;
                        else if (col < NU + NX) SAT[(col - NU) * XP + r] = acc;
                        else dv[r] = sv[r] - acc;
                    }
                }
            }
        }
        __syncthreads();
        // (3) [M | RHS] column-major into MC: thread (column j, row group g)
        //     forms rows g RG .. g RG + RG - 1 of column j
        constexpr int W = NU + NK, CP = CS::CP;
        float* MC = sm + CS::oMC;
        {
            constexpr int G = kPT / W, RG = (NU + G - 1) / G;
            const int j = tid % W, g = tid / W;
            if (g < G) {
                const float* src = j < NU ? SBT + j * XP : (j < NU + NX ? SAT + (j - NU) * XP : dv);
                float v[4 * ((NX + 3) / 4)];
                load_row<NX>(src, v);
                float m[RG];
#pragma unroll
                for (int t = 0; t < RG; ++t) {
                    const int a = g * RG + t;
                    float acc = 0.0f;
                    if (a < NU) {
                        acc = dot_reg<NX>(BtT + a * XP, v);
                        if (j < NU) acc += (a == j) ? Rt[a] : 0.0f;
                        else if (j < NU + NX) acc = -acc;
                        else acc -= gts[a];
                    }
                    m[t] = acc;
                }
                // with state bounds the right-hand sides follow the kNCB bound columns
                const int jm = (BOX && j >= NU) ? j + kNCB : j;
                if constexpr (RG % 4 == 0 && (NU % RG) == 0) {
#pragma unroll
                    for (int q = 0; q < RG / 4; ++q)
                        reinterpret_cast<float4*>(MC + jm * CP + g * RG)[q] =
                            make_float4(m[4 * q], m[4 * q + 1], m[4 * q + 2], m[4 * q + 3]);
                } else {
#pragma unroll
                    for (int t = 0; t < RG; ++t)
                        if (g * RG + t < NU) MC[jm * CP + g * RG + t] = m[t];
                }
            }
        }
        if constexpr (BOX) {
            // the bound rows NU + t of [M | RHS]: [F Bt | 0 | -F A | d - F et],
            // and the bound columns NU + t: (F Bt)' (a unit pivot for a free slot)
            const float* sc = sm + CS::osc;
            const float* sfb = sm + CS::osfb;
            const float* saff = sm + CS::osaff;
            const int nd = reinterpret_cast<const int*>(sm + CS::opn)[2];
            constexpr int NR = NU + kNCB, WB = NR + NK;
            for (int e = tid; e < kNCB * WB; e += kPT) {
                const int t = e / WB, col = e % WB;
                float v = 0.0f;
                if (t >= nd) {
                    v = (col == NU + t) ? 1.0f : 0.0f;
                } else if (col < NU) {
                    v = sc[t * 32 + col];
                } else if (col >= NR) {
                    const int cc = col - NR;
                    v = cc < NX ? sfb[t * XP + cc] : saff[t];
                }
                MC[col * CP + NU + t] = v;
            }
            for (int e = tid; e < kNCB * NU; e += kPT) {
                const int t = e / NU, a = e % NU;
                MC[(NU + t) * CP + a] = t < nd ? sc[t * 32 + a] : 0.0f;
            }
        }
        __syncthreads();
        // (4) Gauss-Jordan elimination without pivoting (M is SPD), a block of
        //     PB pivots (columns p0 .. p0 + PB - 1) per step, by two warps
        //     (warps 0-1 or 2-3 by CTA parity, so co-resident CTAs spread this
        //     phase over the SM's schedulers), thread j holding all NU entries
        //     of column j in registers.  Step (a rolled loop: the rows are
        //     held in rotated order, so the block's pivot rows are always the
        //     first four registers and every register index is fixed, which
        //     keeps the scan's code small enough for the instruction caches;
        //     skipped uniformly when the whole block is eliminated, apart
        //     from the rotation): the block's owners publish their columns into a
        //     double-buffered set, then every column solves the PB x PB pivot
        //     block for its block rows, M_bb y = x_b (Gaussian elimination,
        //     no pivoting: the block is SPD), and takes x -= M_.b y, x_b = y
        //     (the pivot columns become unit vectors).  An eliminated column
        //     is already the unit vector and its row zero in every other
        //     column, so the block solve reduces exactly to the free pivots.
        //     Afterwards column NU + c holds column c of [K | kappa];
        //     eliminated rows stay zero.
        const int gj = tid - ((blockIdx.x & 1) ? 64 : 0);  // column index in the eliminating warps
        if (gj >= 0 && gj < 64) {
            constexpr int PB = kPivotBlock;
            // rows: the inputs, then (with state bounds) the kNCB bound rows
            constexpr int NR = BOX ? NU + kNCB : NU, WR = NR + NK;
            static_assert(WR <= 64, "elimination runs on two warps");
            static_assert(NU % PB == 0 && kNCB % PB == 0, "pivot blocks tile the rows");
            static_assert(NR <= CP, "column buffer");
            float* pcb = sm + CS::opcb;
            const bool act = gj < WR;
            const uint32_t pmask = fmask | (cmask << NU);
            // rows held in rotated order: before block pq, register 4 t + i
            // holds row 4 (pq + t) + i (mod NR), so the block's pivot rows are
            // always registers 0..3 and the block loop need not be unrolled
            constexpr int NQ = NR / PB;
            float xc[NR];
            {
                const float4* c4 = reinterpret_cast<const float4*>(MC + (act ? gj : 0) * CP);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 t4 = c4[q];
                    xc[4 * q + 0] = t4.x;
                    xc[4 * q + 1] = t4.y;
                    xc[4 * q + 2] = t4.z;
                    xc[4 * q + 3] = t4.w;
                }
            }
            int bsel = 0;
#pragma unroll 1
            for (int pq = 0; pq < NQ; ++pq) {
                const int p0 = PB * pq;
                if ((pmask >> p0) & ((1u << PB) - 1u)) {
                    float* buf = pcb + bsel * (PB * 32);
                    if (gj >= p0 && gj < p0 + PB) {
                        float4* dst = reinterpret_cast<float4*>(buf + (gj - p0) * 32);
#pragma unroll
                        for (int q = 0; q < NQ; ++q) dst[q] = make_float4(xc[4 * q], xc[4 * q + 1], xc[4 * q + 2], xc[4 * q + 3]);
                    }
                    asm volatile("bar.sync 1, 64;" ::: "memory");
                    // m[i][j] = M[p0 + i][p0 + j] (column j of the block), y = x_b
                    float m[PB][PB], y[PB];
#pragma unroll
                    for (int j = 0; j < PB; ++j) {
                        const float4 t4 = reinterpret_cast<const float4*>(buf + j * 32)[0];
                        m[0][j] = t4.x;
                        m[1][j] = t4.y;
                        m[2][j] = t4.z;
                        m[3][j] = t4.w;
                    }
#pragma unroll
                    for (int i = 0; i < PB; ++i) y[i] = xc[i];
#pragma unroll
                    for (int i = 0; i < PB; ++i) {
                        const float ip = rcp_approx(m[i][i]);
#pragma unroll
                        for (int r = i + 1; r < PB; ++r) {
                            const float f = m[r][i] * ip;
#pragma unroll
                            for (int j = i + 1; j < PB; ++j) m[r][j] = fmaf(-f, m[i][j], m[r][j]);
                            y[r] = fmaf(-f, y[i], y[r]);
                        }
                    }
#pragma unroll
                    for (int i = PB - 1; i >= 0; --i) {
                        float v = y[i];
#pragma unroll
                        for (int j = i + 1; j < PB; ++j) v = fmaf(-m[i][j], y[j], v);
                        y[i] = v * rcp_approx(m[i][i]);
                    }
#pragma unroll
                    for (int q = 1; q < NQ; ++q) {
#pragma unroll
                        for (int j = 0; j < PB; ++j) {
                            const float4 cj = reinterpret_cast<const float4*>(buf + j * 32)[q];
                            xc[4 * q + 0] = fmaf(-cj.x, y[j], xc[4 * q + 0]);
                            xc[4 * q + 1] = fmaf(-cj.y, y[j], xc[4 * q + 1]);
                            xc[4 * q + 2] = fmaf(-cj.z, y[j], xc[4 * q + 2]);
                            xc[4 * q + 3] = fmaf(-cj.w, y[j], xc[4 * q + 3]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < PB; ++i) xc[i] = y[i];
                    bsel ^= 1;
                }
                // rotate by one block: registers 0..3 move to the end
                float t0 = xc[0], t1 = xc[1], t2 = xc[2], t3 = xc[3];
#pragma unroll
                for (int i = 0; i < NR - PB; ++i) xc[i] = xc[i + PB];
                xc[NR - 4] = t0;
                xc[NR - 3] = t1;
                xc[NR - 2] = t2;
                xc[NR - 1] = t3;
            }
            // (5) gains to K16 (scan) and to global memory (rollout); with state
            // bounds also the bounds' multiplier gains (rows NU + t)
            if (act && gj >= NR) {
                float* Kg = c.K + (size_t)k * NR * NK;
                const int cc = gj - NR;
#pragma unroll
                for (int a = 0; a < NU; ++a) {
                    K16[a * XP + cc] = xc[a];
                    Kg[a * NK + cc] = xc[a];
                }
                if constexpr (BOX) {
                    float* Kl = sm + CS::oKl;
#pragma unroll
                    for (int t = 0; t < kNCB; ++t) {
                        Kl[t * XP + cc] = xc[NU + t];
                        Kg[(NU + t) * NK + cc] = xc[NU + t];
                    }
                }
            }
        }
        __syncthreads();
        // (6) GR = [G | g2]: G = SA + SB K (+ F'K_lambda for exactly held rows),
        //     g2 = dv - SB kappa (- F'kappa_lambda); thread (row r, column quad
        //     cq, half h of the inputs), halves combined by a shuffle
        {
            const int h = tid & 1, cq = (tid >> 1) & 3, r = tid >> 3;
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (r < NX) {
#pragma unroll
                for (int a = 0; a < NU; a += 2) {
                    const int aa = a + h;
                    if (aa < NU && ((fmask >> aa) & 1u)) {
                        const float sb = SBT[aa * XP + r];
                        const float4 kv = reinterpret_cast<const float4*>(K16 + aa * XP)[cq];
                        acc.x = fmaf(sb, kv.x, acc.x);
                        acc.y = fmaf(sb, kv.y, acc.y);
                        acc.z = fmaf(sb, kv.z, acc.z);
                        acc.w = fmaf(sb, kv.w, acc.w);
                    }
                }
            }
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, 1);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, 1);
            if (r < NX && h == 0) {
                float o[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int cc = 4 * cq + q;
                    o[q] = cc < NX ? SAT[cc * XP + r] + o[q] : (cc == NX ? dv[r] - o[q] : 0.0f);
                }
                if constexpr (BOX) {
                    // exactly held rows F: G += F'K_lambda, g2 -= F'kappa_lambda
                    const float* sF = sm + CS::osF;
                    const float* Kl = sm + CS::oKl;
                    const int nd = reinterpret_cast<const int*>(sm + CS::opn)[2];
                    for (int t = 0; t < nd; ++t) {
                        const float f = sF[t * XP + r];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int cc = 4 * cq + q;
                            if (cc < NX) o[q] = fmaf(f, Kl[t * XP + cc], o[q]);
                            else if (cc == NX) o[q] = fmaf(-f, Kl[t * XP + NX], o[q]);
                        }
                    }
                }
                reinterpret_cast<float4*>(GR + r * XP)[cq] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
        __syncthreads();
        // (7) Xp = A' [G | g2] = [P | p] (symmetrised when the next stage reads it)
        {
            const int h = tid & 1, cq = (tid >> 1) & 3, r = tid >> 3;
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (r < NX) {
#pragma unroll
                for (int i = 0; i < NX; i += 2) {
                    const int ii = i + h;
                    if (ii < NX) {
                        const float at = AT[r * XP + ii];
                        const float4 gv = reinterpret_cast<const float4*>(GR + ii * XP)[cq];
                        acc.x = fmaf(at, gv.x, acc.x);
                        acc.y = fmaf(at, gv.y, acc.y);
                        acc.z = fmaf(at, gv.z, acc.z);
                        acc.w = fmaf(at, gv.w, acc.w);
                    }
                }
            }
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, 1);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, 1);
            if (r < NX && h == 0) reinterpret_cast<float4*>(Xp + r * XP)[cq] = acc;
        }
    }
    // forward rollout: ut = K x + kappa, u = T ut + o, x' = A x + Bs u + e
    float* ut = sm + CS::out;
    constexpr int NRK = (BOX ? NU + kNCB : NU) * NK;  // gains per stage
    CPrefetch<NRK, false> pk;
    __syncthreads();
    pf.load(c.grec(0), tid);
    pk.load(c.K, tid);
    for (int k = 0; k < c.Nh; ++k) {
        float* s = c.buf(k);
        __syncthreads();
        pf.store(s, tid);
        pk.store(Ks, tid);
        __syncthreads();
        if (k + 1 < c.Nh) {
            pf.load(c.grec(k + 1), tid);
            pk.load(c.K + (size_t)(k + 1) * NRK, tid);
        }
        const float* xk = c.xr() + k * NX;
        if (tid < NU) {
            float acc = Ks[tid * NK + NX];
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(Ks[tid * NK + r], xk[r], acc);
            ut[tid] = acc;
        } else if (BOX && tid < NU + kNCB) {
            // the multiplier of the exactly held row in slot t, lambda =
            // K_lambda x + kappa_lambda, is the multiplier of its bound
            const int t = tid - NU, org = c.sorig()[k * kNCB + t];
            if (org >= 0) {
                float acc = Ks[(NU + t) * NK + NX];
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(Ks[(NU + t) * NK + r], xk[r], acc);
                c.nub()[org] = acc;
            }
        }
        __syncthreads();
        if (tid < D::NC) {
            const int q = tid, base = q * D::CD;
            const uint32_t mw = c.modes[k * D::NC + q];
            float* u = c.ur() + k * NU;
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
                    u[tj] = (sg == 0) ? ut[tj] : sg * cone_coef<D::CD>(jj, mu, c.dx, c.dy) * n;
                }
            }
        }
        __syncthreads();
        cta_rollout_step<D>(c, s, k);
    }
    __syncthreads();
    return npiv;
}

// Forward rollout of given (scaled) inputs ur.
template <class D>
__device__ void cta_rollout(const CCtx<D>& c) {
    CPrefetch<D::SREC, true> pf;
    __syncthreads();
    pf.load(c.grec(0), c.tid);
    for (int k = 0; k < c.Nh; ++k) {
        float* s = c.buf(k);
        __syncthreads();
        pf.store(s, c.tid);
        __syncthreads();
        if (k + 1 < c.Nh) pf.load(c.grec(k + 1), c.tid);
        cta_rollout_step<D>(c, s, k);
    }
    __syncthreads();
}

// Multipliers of the active state bounds read off the ADMM iterate: at a
// fixed point of Sec. III's iteration, rho (theta_k - lambda_k) restricted to
// the state components is the normal-cone element of z_{k+1}'s state part,
// i.e. the signed multiplier of its box (the state part is not scaled).  An
// estimate of the wrong sign starts at 0.
template <class D>
__device__ void cta_box_init(const CCtx<D>& c, const RoundArgs& a, int b) {
    const float* st = a.state + (size_t)b * RoundState<D>::floats(a.N);
    const int cb = __float_as_int(st[RoundState<D>::var_floats(a.N) + RoundState<D>::sCb]);
    for (int e = c.tid; e < c.Nh * D::NX; e += kPT) {
        const int k = e / D::NX, i = e % D::NX;
        float bnd, v = 0.0f;
        bool up;
        if (c.box_active(k, i, &bnd, &up)) {
            v = a.rho * (st[RoundState<D>::at(a.N, cb, k, VTH) + i] - st[RoundState<D>::at(a.N, cb, k, VLA) + i]);
            if (up ? v < 0.0f : v > 0.0f) v = 0.0f;
        }
        c.nub()[e] = v;
        c.rhob()[e] = kBoxPenalty;
        c.dprev()[e] = INFINITY;
        c.dlast()[e] = 0.0f;
    }
    // no bound held exactly until a scan holds it (a certificate of the
    // iterate weights every active bound as held by the augmented Lagrangian)
    for (int k = c.tid; k < c.Nh; k += kPT) c.dbits()[k] = 0u;
    __syncthreads();
}

// Polish with active state bounds: scans (see cta_polish, which holds a
// bound exactly when the stage's free inputs move its component), each
// followed by the multiplier step nu += p (x - b) on the bounds held by the
// augmented Lagrangian instead, until every active bound holds to kBoxViol
// (relative) or kBoxIters scans.  Without active bounds this is one plain
// scan.  Returns the pivots eliminated and adds the scans to *nscan.
template <class D, bool BOX>
__device__ int cta_polish_box(const CCtx<D>& c, int* nscan) {
    constexpr int NX = D::NX;
    bool any = false;
    if constexpr (BOX) {
        for (int k = c.tid; k < c.Nh; k += kPT) {
            any |= c.sbits()[k] != 0u;
            c.albits()[k] = 0u;  // every bound first tries to be held exactly
        }
        any = __syncthreads_or(any);
    }
    int npiv = 0;
    for (int t = 0; t < (any ? kBoxIters : 1); ++t) {
        npiv += cta_polish<D, BOX>(c);
        ++*nscan;
        if (!any) break;
        float viol = 0.0f;
        for (int e = c.tid; e < c.Nh * NX; e += kPT) {
            const int k = e / NX, i = e % NX;
            float bnd;
            bool up;
            if (c.box_active(k, i, &bnd, &up) && !((c.dbits()[k] >> i) & 1u)) {
                // held by the augmented Lagrangian (an exactly held bound has
                // its multiplier from the scan, and more scans cannot improve it)
                const float d = c.xr()[(k + 1) * NX + i] - bnd;
                const float vi = fabsf(d) / (1.0f + fabsf(bnd));
                const float pen = c.rhob()[e];
                // while the penalty stays, the multiplier's error contracts by
                // r = h / (h + p) per scan, and r = d / d_last: the step that
                // lands on the limit is p d / (1 - r) (Aitken's extrapolation
                // of the geometric sequence); a jump is not followed by another
                const float dl = c.dlast()[e];
                const float r = dl != 0.0f ? d / dl : 0.0f;
                const bool jump = r > 0.0f && r < kBoxAitkenMax;
                c.nub()[e] = fmaf(jump ? pen / (1.0f - r) : pen, d, c.nub()[e]);
                // a stiff bound (its violation falls too slowly) gets a larger penalty
                const bool grow = vi > kBoxViol && fabsf(d) > kBoxRate * c.dprev()[e] && pen < kBoxPenaltyMax;
                if (grow) c.rhob()[e] = fminf(pen * kBoxGrow, kBoxPenaltyMax);
                c.dlast()[e] = (grow || jump) ? 0.0f : d;
                c.dprev()[e] = fabsf(d);
                viol = fmaxf(viol, vi);
            }
        }
        viol = cta_max(c, viol);
        if (viol <= kBoxViol) break;
    }
    __syncthreads();
    return npiv;
}

// KKT certificate (the terms of `certificate` in solve.cuh).
template <class D, bool BOX = false>
__device__ float cta_certificate(const CCtx<D>& c) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int tid = c.tid;
    const float sig = c.sigma, isig = 1.0f / c.sigma;
    float den = 0.0f, uinf = 0.0f;
    CPrefetch<D::SREC, true> pf;
    pf.load(c.grec(c.Nh - 1), tid);
    for (int k = c.Nh - 1; k >= 0; --k) {
        float* s = c.buf(k);
        __syncthreads();
        pf.store(s, tid);
        __syncthreads();
        if (k > 0) pf.load(c.grec(k - 1), tid);
        if (tid < NX) {
            float acc = s[D::oQ + tid] * (c.xr()[(k + 1) * NX + tid] - s[D::oRY + tid]);
            if (k + 1 < c.Nh) {
                const float* An = c.buf(k + 1) + D::oA;  // stage k+1, kept from the previous step
#pragma unroll
                for (int i = 0; i < NX; ++i) acc = fmaf(An[i * NX + tid], c.y()[(k + 1) * NX + i], acc);
            }
            if constexpr (BOX) {
                // an active state bound's multiplier (of the right sign) enters y_k
                float bnd;
                bool up;
                if (c.box_active(k, tid, &bnd, &up)) {
                    const float v = c.nub()[k * NX + tid];
                    if (up ? v >= 0.0f : v <= 0.0f) acc += v;
                }
            }
            c.y()[k * NX + tid] = acc;
        }
        __syncthreads();
        if (tid < NU) {
            const int e = k * NU + tid;
            const float rdu = s[D::oR + tid] * (c.ur()[e] - s[D::oRU + tid]) * isig;
            float bty = 0.0f;
#pragma unroll
            for (int r = 0; r < NX; ++r) bty = fmaf(s[D::oB + r * NU + tid], c.y()[k * NX + r], bty);
            bty *= isig;
            c.wv()[e] = rdu + bty;
            den = fmaxf(den, fmaxf(fabsf(rdu), fabsf(bty)));
            uinf = fmaxf(uinf, fabsf(c.ur()[e]) * sig);
        }
    }
    {
        float m2[2] = {den, uinf};
        cta_max_n<D, 2>(c, m2);
        den = m2[0];
        uinf = m2[1];
    }
    float feas = 0.0f, stat = 0.0f, comp = 0.0f;
    for (int e = tid; e < c.Nh * D::NC; e += kPT) {
        const int k = e / D::NC, q = e % D::NC;
        const float fmax = c.fms(k, q) * sig;
        const float* us = c.ur() + k * NU + q * CD;
        float u[CD], r[CD];
#pragma unroll
        for (int i = 0; i < CD; ++i) { u[i] = us[i] * sig; r[i] = c.wv()[k * NU + q * CD + i]; }
        if (!((c.mask(k) >> q) & 1u)) {
            float mm = 0.0f;
#pragma unroll
            for (int i = 0; i < CD; ++i) mm = fmaxf(mm, fabsf(u[i]));
            feas = fmaxf(feas, mm / (c.kc + fmax));
            continue;
        }
        const float mu = c.mu(k, q);
        float cf[M], g[F], lam[F], nrm2[F];
        const float n = u[D::NRM];
#pragma unroll
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
        float gmax = -INFINITY, wmax = 0.0f;
#pragma unroll
        for (int f = 0; f < F; ++f) { lam[f] = 0.0f; gmax = fmaxf(gmax, g[f]); }
#pragma unroll
        for (int i = 0; i < CD; ++i) wmax = fmaxf(wmax, fabsf(r[i]));
        feas = fmaxf(feas, fmaxf(gmax, 0.0f) / (c.kc + fmax));
        // at most kNnlsSweeps sweeps: each sweep lowers the fit's squared
        // residual, so a cut-off fit leaves it larger than the converged one
        for (int sweep = 0; sweep < kNnlsSweeps; ++sweep) {
            float change = 0.0f;
#pragma unroll
            for (int f = 0; f < F; ++f) {
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
    if constexpr (BOX) {
        // state boxes: violation max(x - hi, lo - x, 0) / (kc + |bound|), and
        // |nu (x - b)| of the active bounds whose multiplier counts; both
        // weighted by kBoxFeasWeight unless the scan held the bound exactly
        // (it then sits on its bound to rounding)
        for (int e = tid; e < c.Nh * NX; e += kPT) {
            const int k = e / NX, i = e % NX;
            const float lo = c.box[(k * 2) * NX + i], hi = c.box[(k * 2 + 1) * NX + i];
            const float x = c.xr()[(k + 1) * NX + i];
            float bnd;
            bool up;
            const bool act = c.box_active(k, i, &bnd, &up);
            const float wgt = ((c.dbits()[k] >> i) & 1u) ? 1.0f : kBoxFeasWeight;
            if (x > hi) feas = fmaxf(feas, wgt * (x - hi) / (c.kc + fabsf(hi)));
            if (x < lo) feas = fmaxf(feas, wgt * (lo - x) / (c.kc + fabsf(lo)));
            if (act) {
                const float v = c.nub()[e];
                if (up ? v >= 0.0f : v <= 0.0f) comp = fmaxf(comp, wgt * fabsf(v * (x - bnd)));
            }
        }
    }
    {
        float m3[3] = {feas, stat, comp};
        cta_max_n<D, 3>(c, m3);
        feas = m3[0];
        stat = m3[1];
        comp = m3[2];
    }
    // each term |res| / (kc + scale) <= kkt_tol  <=>  |res| <= kkt_tol_abs + kkt_tol scale
    return fmaxf(feas, fmaxf(stat / (c.kc + den), comp / (c.kc + uinf)));
}

// Faces re-read off Proj(u - alpha sigma w); returns whether any changed.
template <class D, bool BOX = false>
__device__ bool cta_refine_modes(const CCtx<D>& c, float alpha) {
    constexpr int NU = D::NU, CD = D::CD;
    bool changed = false;
    for (int e = c.tid; e < c.Nh * D::NC; e += kPT) {
        const int k = e / D::NC, q = e % D::NC;
        if (!((c.mask(k) >> q) & 1u)) continue;
        float a[CD], out[CD];
#pragma unroll
        for (int i = 0; i < CD; ++i)
            a[i] = c.ur()[k * NU + q * CD + i] - alpha * c.sigma * c.wv()[k * NU + q * CD + i];
        const uint32_t mw = project_contact<CD>(a, out, c.mu(k, q), c.fms(k, q), c.dx, c.dy);
        if (mw != c.modes[e]) {
            changed = true;
            c.modes[e] = mw;
        }
    }
    if constexpr (BOX) {
        // state bounds: a violated one joins (multiplier 0), an active one whose
        // multiplier has the wrong sign leaves
        constexpr int NX = D::NX;
        for (int e = c.tid; e < c.Nh * NX; e += kPT) {
            const int k = e / NX, i = e % NX;
            const float lo = c.box[(k * 2) * NX + i], hi = c.box[(k * 2 + 1) * NX + i];
            const float x = c.xr()[(k + 1) * NX + i], v = c.nub()[e];
            const uint32_t sb = c.sbits()[k];
            const bool alo = (sb >> i) & 1u, ahi = (sb >> (16 + i)) & 1u;
            uint32_t set = 0u, clr = 0u;
            if (ahi && v < 0.0f) clr |= 1u << (16 + i);
            if (alo && v > 0.0f) clr |= 1u << i;
            if (!ahi && x > hi) set |= 1u << (16 + i);
            if (!alo && x < lo) set |= 1u << i;
            if (set | clr) {
                changed = true;
                if (set) {
                    atomicOr(c.sbits() + k, set);
                    c.nub()[e] = 0.0f;
                    c.rhob()[e] = kBoxPenalty;
                    c.dprev()[e] = INFINITY;
                    c.dlast()[e] = 0.0f;
                }
                if (clr) atomicAnd(c.sbits() + k, ~clr);
            }
        }
    }
    return __syncthreads_or(changed);
}

// A 32-bit hash of the faces being polished (and, with state bounds, of the
// active bounds): each entry mixed with its index by the murmur3 finaliser,
// the results XORed over the CTA (valid in every thread).
template <class D, bool BOX>
__device__ uint32_t cta_faces_hash(const CCtx<D>& c) {
    auto mix = [](uint32_t x) {
        x ^= x >> 16;
        x *= 0x85EBCA6Bu;
        x ^= x >> 13;
        x *= 0xC2B2AE35u;
        return x ^ (x >> 16);
    };
    uint32_t h = 0u;
    for (int e = c.tid; e < c.Nh * D::NC; e += kPT) h ^= mix(c.modes[e] ^ ((uint32_t)(e + 1) * 0x9E3779B9u));
    if constexpr (BOX)
        for (int k = c.tid; k < c.Nh; k += kPT) h ^= mix(c.sbits()[k] ^ ((uint32_t)(k + 1) * 0x7F4A7C15u));
    h = __reduce_xor_sync(0xffffffffu, h);
    uint32_t* red = reinterpret_cast<uint32_t*>(c.sm + CtaSmem<D>::ored);
    __syncthreads();
    if (c.lane == 0) red[c.warp] = h;
    __syncthreads();
    uint32_t r = 0u;
#pragma unroll
    for (int w = 0; w < kPT / 32; ++w) r ^= red[w];
    return r;
}

// The point (xi, u, active faces, certificate) of instance b into the
// outputs; zeros and an infinite certificate when !ok.
template <class D>
__device__ void cta_write_point(const CCtx<D>& c, const RoundArgs& a, int b, bool ok, float kkt) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int Nv = a.N;
    float* oxi = a.out_xi + (size_t)b * Nv * NX;
    float* ou = a.out_u + (size_t)b * Nv * NU;
    for (int e = c.tid; e < Nv * NX; e += kPT) {
        const int k = e / NX;
        oxi[e] = (ok && k < c.Nh) ? c.xr()[(k + 1) * NX + (e % NX)] : 0.0f;
    }
    for (int e = c.tid; e < Nv * NU; e += kPT) {
        const int k = e / NU;
        ou[e] = (ok && k < c.Nh) ? c.ur()[e] * c.sigma : 0.0f;
    }
    for (int k = c.tid; k < Nv; k += kPT) {
        unsigned long long bits = 0ull;
        if (ok && k < c.Nh) {
            for (int q = 0; q < D::NC; ++q) {
                if (!((c.mask(k) >> q) & 1u)) continue;
                const float fmax = c.fms(k, q) * c.sigma;
                const float mu = c.mu(k, q);
                const float* us = c.ur() + k * NU + q * CD;
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
    if (c.tid == 0) a.out_kkt[b] = ok ? kkt : INFINITY;
}

// Final status of instance b (its point already in the outputs).
__device__ __forceinline__ void finish_instance(const RoundArgs& a, int b, int status, int iters, int npol) {
    if (threadIdx.x == 0) {
        a.out_status[b] = status;
        a.out_iters[b] = iters;
        a.out_npol[b] = npol;
        a.done[b] = 1;
    }
}

template <class D>
__device__ void cta_write_output(const CCtx<D>& c, const RoundArgs& a, int b, int status, int iters, float kkt,
                                 int npol) {
    cta_write_point<D>(c, a, b, status == kConverged || status == kMaxIter, kkt);
    finish_instance(a, b, status, iters, npol);
}

// Polish / certify / refine after a round: one CTA per instance.
template <class D, bool BOX>
__device__ __forceinline__ void polish_instance(const RoundArgs& a, int b, float* psm) {
    constexpr int NX = D::NX, NU = D::NU;
    if (a.done[b]) return;
    CCtx<D> c(a.N);
    c.sm = psm;
    c.rec = a.rec + (size_t)b * a.irec;
    c.modes = reinterpret_cast<uint32_t*>(c.sm + c.L.modes);
    c.K = a.Kst + (size_t)b * a.N * (NU + kNCB) * (NX + 1);  // [N][NU (+ kNCB)][NX + 1]
    c.tid = threadIdx.x;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    c.sigma = a.sigma;
    c.kc = a.kkt_c;
    c.box = BOX ? a.xbox + (size_t)b * a.n_rec * 2 * NX : nullptr;
    c.dx = a.dx;
    c.dy = a.dy;
    const float* tail = c.rec + (size_t)a.n_rec * D::SREC;
    c.Nh = __float_as_int(__ldg(tail + D::tH));
    const bool final_round = a.m1 >= a.max_iter;
    uint32_t* gmodes = a.modes + (size_t)b * a.N * D::NC;
    uint32_t* glast = a.lastm + (size_t)b * a.N * D::NC;
    bool changed = false;
    for (int e = c.tid; e < c.Nh * D::NC; e += kPT) {
        const uint32_t mw = gmodes[e];
        c.modes[e] = mw;
        changed |= (mw != glast[e]);
        const int k = e / D::NC, q = e % D::NC;
        c.sm[c.L.cmu + e] = __ldg(c.grec(k) + D::oMU + q);
        c.sm[c.L.cfm + e] = __ldg(c.grec(k) + D::oFM + q);
    }
    for (int k = c.tid; k < c.Nh; k += kPT) c.sm[c.L.cmask + k] = __ldg(c.grec(k) + D::oMASK);
    // the state bounds the round's z sits at; a change also calls for a polish
    uint32_t* gsm = BOX ? a.smodes + (size_t)b * a.N : nullptr;
    uint32_t* gsl = BOX ? a.slast + (size_t)b * a.N : nullptr;
    if constexpr (BOX) {
        for (int k = c.tid; k < c.Nh; k += kPT) {
            const uint32_t sb = gsm[k];
            c.sbits()[k] = sb;
            changed |= (sb != gsl[k]);
        }
    }
    for (int i = c.tid; i < NX; i += kPT) c.xr()[i] = __ldg(tail + D::tXI0 + i);
    changed = __syncthreads_or(changed);
    int npol = a.out_npol[b];
    int npiv = a.out_piv[b];
    float kkt = INFINITY;
    // the outputs hold the best polished point within kStallBand of the
    // tolerance so far (its certificate in kkt; the solve starts with a huge
    // value) and, in iters, a stall count (the solve starts with 0): checks
    // since there is such a point at which the faces did not change or the
    // polish did not halve the best certificate; thread 0 reads and writes
    // both and shares its decisions through a barrier
    if (a.polish && !changed &&
        __syncthreads_or(c.tid == 0 && a.out_kkt[b] <= kStallBand * a.kkt_tol && a.out_iters[b] + 1 >= kStallChecks)) {
        finish_instance(a, b, kStalled, a.m1, npol);
        return;
    }
    if (a.polish && changed) {
        for (int e = c.tid; e < c.Nh * D::NC; e += kPT) glast[e] = c.modes[e];
        if constexpr (BOX) {
            for (int k = c.tid; k < c.Nh; k += kPT) gsl[k] = c.sbits()[k];
            cta_box_init<D>(c, a, b);
        }
        npiv += cta_polish_box<D, BOX>(c, &npol);
        kkt = cta_certificate<D, BOX>(c);
        // The refinement's state, in shared memory and written by thread 0:
        // the step, the best certificate of this call, the refinements since
        // it improved, and the hashes of the face sets polished in this call
        // (a ring of 8 and its count).  Against active-set cycles (faces
        // flipped in and out again): from the second refinement in a row that
        // does not improve the best certificate each next step is 3x longer
        // (up to 27x), an improvement restores the configured step, and a
        // refinement that lands on a face set already polished is retried
        // with a 3x longer step (twice at most) instead of polishing it again.
        float* step = c.sm + CtaSmem<D>::ostep;
        uint32_t* ring = reinterpret_cast<uint32_t*>(step + 4);
        {
            const uint32_t h0 = cta_faces_hash<D, BOX>(c);
            if (c.tid == 0) {
                step[0] = a.refine_alpha;
                step[1] = kkt;
                step[2] = 0.0f;
                ring[0] = h0;
                ring[8] = 1u;
            }
        }
        for (int r = 0; kkt > a.kkt_tol && r < a.refine_steps; ++r) {
            __syncthreads();
            bool fresh = false;
            float alpha = step[0];
            for (int t = 0; t < 3; ++t) {
                if (!cta_refine_modes<D, BOX>(c, alpha)) break;
                const uint32_t h = cta_faces_hash<D, BOX>(c);
                const uint32_t n = min(ring[8], 8u);
                bool seen = false;
                for (uint32_t i = 0; i < n; ++i) seen |= ring[i] == h;
                if (!seen) {
                    fresh = true;
                    __syncthreads();
                    if (c.tid == 0) {
                        ring[ring[8] & 7u] = h;
                        ring[8] += 1u;
                    }
                    break;
                }
                alpha *= 3.0f;
            }
            if (!fresh) break;
            npiv += cta_polish_box<D, BOX>(c, &npol);
            kkt = cta_certificate<D, BOX>(c);
            if (c.tid == 0) {
                const bool better = kkt < step[1];
                step[2] = better ? 0.0f : step[2] + 1.0f;
                step[0] = better ? a.refine_alpha
                                 : (step[2] >= 2.0f ? fminf(3.0f * step[0], 27.0f * a.refine_alpha) : step[0]);
                step[1] = fminf(step[1], kkt);
            }
        }
        if (c.tid == 0) a.out_piv[b] = npiv;
        if (kkt <= a.kkt_tol) {
            cta_write_output<D>(c, a, b, kConverged, a.m1, kkt, npol);
            return;
        }
        // thread 0: keep the point if it is the closest miss within the band
        // so far; a point that halves the best restarts the stall count,
        // another one within the band advances it like a check without a
        // polish.  With state bounds every polish within the band restarts
        // it and one outside the band holds it off (their augmented
        // Lagrangian restarts from the iterate's multipliers, so later
        // polishes on the same faces still move)
        float* flag = c.sm + CtaSmem<D>::ored;
        if (c.tid == 0) {
            const float best = a.out_kkt[b];
            const bool inb = kkt <= kStallBand * a.kkt_tol;
            const int stall = BOX ? (inb ? 0 : -(1 << 20))
                                  : ((inb && kkt < 0.5f * best) ? 0 : a.out_iters[b] + (inb ? 1 : 0));
            a.out_iters[b] = stall;
            flag[0] = (inb && kkt < best) ? 1.0f : 0.0f;
            flag[1] = stall >= kStallChecks ? 1.0f : 0.0f;
        }
        __syncthreads();
        const bool stop = flag[1] != 0.0f;
        if (flag[0] != 0.0f) cta_write_point<D>(c, a, b, true, kkt);
        if (stop) {
            finish_instance(a, b, kStalled, a.m1, npol);
            return;
        }
    }
    if (!a.polish || final_round) {
        // certify the ADMM iterate itself: u from z of the current buffer
        const float* st = a.state + (size_t)b * RoundState<D>::floats(a.N);
        const int cb = __float_as_int(st[RoundState<D>::var_floats(a.N) + RoundState<D>::sCb]);
        __syncthreads();
        for (int e = c.tid; e < c.Nh * NU; e += kPT) {
            const int k = e / NU, i = e % NU;
            c.ur()[e] = st[RoundState<D>::at(a.N, cb, k, VZ) + NX + i];
        }
        if constexpr (BOX) {
            // the round's bounds and multipliers (a polish may have moved them)
            for (int k = c.tid; k < c.Nh; k += kPT) c.sbits()[k] = gsm[k];
            __syncthreads();
            cta_box_init<D>(c, a, b);
        }
        cta_rollout<D>(c);
        kkt = cta_certificate<D, BOX>(c);
        if (kkt <= a.kkt_tol) {
            cta_write_output<D>(c, a, b, kConverged, a.m1, kkt, npol);
            return;
        }
        if (final_round) {
            // the iterate, unless a polished point came closer
            if (__syncthreads_or(c.tid == 0 && kkt <= a.out_kkt[b])) cta_write_point<D>(c, a, b, true, kkt);
            finish_instance(a, b, kMaxIter, a.m1, npol);
            return;
        }
    }
    if (c.tid == 0) {
        // a check without a polish advances the stall count once there is a
        // point within the band
        if (a.polish && !changed && a.out_kkt[b] <= kStallBand * a.kkt_tol) a.out_iters[b] += 1;
        a.out_npol[b] = npol;
        // still running: next round, in its horizon class's list
        const int cl = horizon_class(c.Nh, a.N, a.ncls, a.cls_cap);
        a.list_out[(size_t)cl * a.cls_stride + atomicAdd(a.cnt_out + cl, 1)] = b;
    }
}

// Polish / certify / refine after a round: CTA i takes slot i of the round's
// lists, the classes' lists taken one after another (grid = batch size;
// slots past their total length return at once).
template <class D, bool BOX = false>
__global__ void __launch_bounds__(kPT, D::CD == 3 ? 5 : 3) polish_cta_kernel(RoundArgs a) {
    extern __shared__ __align__(16) float psm[];
    int b = -1;
    if (!a.list_in) {
        b = blockIdx.x < a.B ? (int)blockIdx.x : -1;
    } else {
        int i = blockIdx.x;
        for (int cl = 0; cl < a.ncls; ++cl) {
            const int n = a.cnt_in[cl];
            if (i < n) {
                b = a.list_in[(size_t)cl * a.cls_stride + i];
                break;
            }
            i -= n;
        }
    }
    if (b < 0) return;
    polish_instance<D, BOX>(a, b, psm);
}

}  // namespace pinmpc
