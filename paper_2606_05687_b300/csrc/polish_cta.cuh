// Polish, certificate and active-set refinement with one 128-thread CTA per
// instance (4 warps).  The algebra is that of warp_polish / warp_certificate
// in polish.cuh (backward Riccati scan on the reduced inputs, forward
// rollout, KKT terms, projected-gradient face update); here the per-stage
// products are spread over 128 threads with CTA barriers, the 24x24
// Cholesky factorisation stays in one warp's registers, and the 14
// right-hand sides of the two triangular solves are split over the 4 warps.
#pragma once
#include "polish.cuh"

namespace pinmpc {

constexpr int kPT = 128;  // threads per polish CTA

template <class D>
struct CtaSmem {
    static constexpr int NX = D::NX, NU = D::NU, NK = NX + 1, W = NU + NK;  // W: columns of [M | RHS]
    static constexpr int al(int x) { return (x + 3) & ~3; }
    static constexpr int oP = 0, op = al(oP + NX * NX), oS = al(op + NX), osv = al(oS + NX * NX),
                         oSA = al(osv + NX), oSB = al(oSA + NX * NX), oSe = al(oSB + NX * NU), oet = al(oSe + NX),
                         oBt = al(oet + NX), oRt = al(oBt + NX * NU), ogt = al(oRt + NU), oot = al(ogt + NU),
                         oA0 = al(oot + NU), oA1 = al(oA0 + NU * W), oK = al(oA1 + NU * W),
                         og2 = al(oK + NU * NK), oidx = al(og2 + NX), opos = al(oidx + NU), onf = al(opos + NU),
                         out = al(onf + 4),
                         obuf0 = al(out + NU), obuf1 = al(obuf0 + D::SREC), ored = al(obuf1 + D::SREC),
                         oFixed = al(ored + 32);
    static_assert(oK % 4 == 0 && obuf0 % 4 == 0 && obuf1 % 4 == 0, "16-byte regions for float4 traffic");
    int xr, ur, y, wv, modes, cmu, cfm, cmask, total;
    __host__ __device__ explicit CtaSmem(int N) {
        int o = oFixed;
        auto take = [&o](int n) { int r = o; o += (n + 3) & ~3; return r; };
        xr = take((N + 1) * NX);
        ur = take(N * NU);
        // the certificate runs after the scan: costates reuse an elimination
        // buffer, the gradient the S/SA/SB/Se area, when they fit
        y = (N * NX <= NU * W) ? oA0 : take(N * NX);
        wv = (N * NU <= oet - oS) ? oS : take(N * NU);
        modes = take(N * D::NC);
        cmu = take(N * D::NC);
        cfm = take(N * D::NC);
        cmask = take(N);
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
};

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

// Backward Riccati scan + forward rollout of one instance by one CTA.
template <class D>
__device__ void cta_polish(const CCtx<D>& c) {
    constexpr int NX = D::NX, NU = D::NU, NK = NX + 1;
    using CS = CtaSmem<D>;
    const int tid = c.tid;
    float* sm = c.sm;
    float* P = sm + CS::oP;
    float* p = sm + CS::op;
    float* S = sm + CS::oS;
    float* sv = sm + CS::osv;
    float* SA = sm + CS::oSA;
    float* SB = sm + CS::oSB;
    float* Se = sm + CS::oSe;
    float* et = sm + CS::oet;
    float* Bt = sm + CS::oBt;
    float* Rt = sm + CS::oRt;
    float* gts = sm + CS::ogt;
    float* ots = sm + CS::oot;
    float* Aug0 = sm + CS::oA0;
    float* Aug1 = sm + CS::oA1;
    float* Ks = sm + CS::oK;
    float* g2 = sm + CS::og2;
    for (int e = tid; e < NX * NX + NX; e += kPT) {
        if (e < NX * NX) P[e] = 0.0f; else p[e - NX * NX] = 0.0f;
    }
    CPrefetch<D::SREC, true> pf;
    pf.load(c.grec(c.Nh - 1), tid);
    for (int k = c.Nh - 1; k >= 0; --k) {
        float* s = c.buf(k);
        __syncthreads();
        pf.store(s, tid);
        __syncthreads();
        if (k > 0) pf.load(c.grec(k - 1), tid);
        // reduced input map, one column per thread; eliminated columns (swing
        // or apex contacts, face-fixed components) have bt = 0 and rt = 1
        int* idx = reinterpret_cast<int*>(sm + CS::oidx);  // free columns, compacted
        int* pos = reinterpret_cast<int*>(sm + CS::opos);  // column -> position in idx, or -1
        int* nfs = reinterpret_cast<int*>(sm + CS::onf);
        if (tid < 32) {
            bool fr = false;
            if (tid < NU) {
                float bt[NX], rt, gt, ot;
                reduced_column<D>(c, s, c.modes[k * D::NC + tid / D::CD], tid, bt, rt, gt, ot);
#pragma unroll
                for (int r = 0; r < NX; ++r) {
                    Bt[r * NU + tid] = bt[r];
                    fr |= (bt[r] != 0.0f);
                }
                fr |= (rt != 1.0f) || (gt != 0.0f);
                Rt[tid] = rt;
                gts[tid] = gt;
                ots[tid] = ot;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, fr);
            const int a = __popc(ball & ((1u << tid) - 1u));
            if (tid < NU) {
                pos[tid] = fr ? a : -1;
                if (fr) idx[a] = tid;
            }
            if (tid == 0) nfs[0] = __popc(ball);
        }
        __syncthreads();
        const int nf = nfs[0];
        // et = e + Bs ot ; S = diag(Q) + P ; s = Q ry + p
        for (int e = tid; e < NX * NX + 2 * NX; e += kPT) {
            if (e < NX * NX) {
                const int r = e / NX, cc = e % NX;
                S[e] = P[e] + (r == cc ? s[D::oQ + r] : 0.0f);
            } else if (e < NX * NX + NX) {
                const int r = e - NX * NX;
                float acc = s[D::oE + r];
#pragma unroll
                for (int i = 0; i < NU; ++i) acc = fmaf(s[D::oB + r * NU + i], ots[i], acc);
                et[r] = acc;
            } else {
                const int r = e - NX * NX - NX;
                sv[r] = fmaf(s[D::oQ + r], s[D::oRY + r], p[r]);
            }
        }
        __syncthreads();
        // SB = S Bt on the free columns (SB[r][a], a < nf), SA = S A, Se = S et
        for (int e = tid; e < NX * (nf + NX + 1); e += kPT) {
            const int r = e / (nf + NX + 1), col = e % (nf + NX + 1);
            float acc = 0.0f;
            if (col < nf) {
                const int ic = idx[col];
#pragma unroll
                for (int i = 0; i < NX; ++i) acc = fmaf(S[r * NX + i], Bt[i * NU + ic], acc);
                SB[r * NU + col] = acc;
            } else if (col < nf + NX) {
#pragma unroll
                for (int i = 0; i < NX; ++i) acc = fmaf(S[r * NX + i], s[D::oA + i * NX + col - nf], acc);
                SA[r * NX + col - nf] = acc;
            } else {
#pragma unroll
                for (int i = 0; i < NX; ++i) acc = fmaf(S[r * NX + i], et[i], acc);
                Se[r] = acc;
            }
        }
        __syncthreads();
        // [M_ff | RHS_f] on the free rows/columns: M = Rt + Bt' S Bt,
        // RHS = [-Bt' S A | Bt'(s - S et) - gt]
        const int W = nf + NK;
        for (int e = tid; e < nf * W; e += kPT) {
            const int a = e / W, j = e % W, ia = idx[a];
            float acc;
            if (j < nf) {
                acc = (a == j) ? Rt[ia] : 0.0f;
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(Bt[r * NU + ia], SB[r * NU + j], acc);
            } else if (j < nf + NX) {
                acc = 0.0f;
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(Bt[r * NU + ia], SA[r * NX + j - nf], acc);
                acc = -acc;
            } else {
                acc = -gts[ia];
#pragma unroll
                for (int r = 0; r < NX; ++r) acc = fmaf(Bt[r * NU + ia], sv[r] - Se[r], acc);
            }
            Aug0[e] = acc;
        }
        __syncthreads();
        // Gauss-Jordan elimination without pivoting (M_ff is SPD): after nf
        // steps the right block holds X = M_ff^{-1} RHS_f.  Each thread owns one
        // column and a group of rows; the two buffers alternate so a step
        // needs one barrier.
        {
            const int G = kPT / W;                 // row groups (>= 3)
            const int RPG = (nf + G - 1) / G;      // rows per group (<= 8)
            const int j = tid % W, g = tid / W;
            const float* X = Aug0;
            float* Y = Aug1;
#pragma unroll 1
            for (int pp = 0; pp < nf; ++pp) {
                if (g < G && j > pp) {
                    const float prj = X[pp * W + j] * __frcp_rn(X[pp * W + pp]);
#pragma unroll
                    for (int t = 0; t < (NU + 2) / 3; ++t) {
                        const int i = g * RPG + t;
                        if (t < RPG && i < nf)
                            Y[i * W + j] = (i == pp) ? prj : fmaf(-X[i * W + pp], prj, X[i * W + j]);
                    }
                }
                __syncthreads();
                const float* T = X;
                X = Y;
                Y = const_cast<float*>(T);
            }
            // gains: free rows from the solve, eliminated rows 0
            float* Kg = c.K + (size_t)k * NU * NK;
            for (int e = tid; e < NU * NK; e += kPT) {
                const int a = pos[e / NK];
                const float v = (a >= 0) ? X[a * W + nf + (e % NK)] : 0.0f;
                Ks[e] = v;
                Kg[e] = v;
            }
        }
        __syncthreads();
        // G = SA + SB K (in place over SA), g2 = s - Se - SB kappa
        for (int e = tid; e < NX * NX + NX; e += kPT) {
            if (e < NX * NX) {
                const int r = e / NX, cc = e % NX;
                float acc = SA[e];
                for (int a = 0; a < nf; ++a) acc = fmaf(SB[r * NU + a], Ks[idx[a] * NK + cc], acc);
                SA[e] = acc;
            } else {
                const int r = e - NX * NX;
                float acc = sv[r] - Se[r];
                for (int a = 0; a < nf; ++a) acc = fmaf(-SB[r * NU + a], Ks[idx[a] * NK + NX], acc);
                g2[r] = acc;
            }
        }
        __syncthreads();
        // P = sym(A' G), p = A' g2
        for (int e = tid; e < NX * NX + NX; e += kPT) {
            if (e < NX * NX) {
                const int r = e / NX, cc = e % NX;
                float a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int i = 0; i < NX; ++i) {
                    a1 = fmaf(s[D::oA + i * NX + r], SA[i * NX + cc], a1);
                    a2 = fmaf(s[D::oA + i * NX + cc], SA[i * NX + r], a2);
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
    }
    // forward rollout: ut = K x + kappa, u = T ut + o, x' = A x + Bs u + e
    float* ut = sm + CS::out;
    CPrefetch<NU * NK, false> pk;
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
            pk.load(c.K + (size_t)(k + 1) * NU * NK, tid);
        }
        const float* xk = c.xr() + k * NX;
        if (tid < NU) {
            float acc = Ks[tid * NK + NX];
#pragma unroll
            for (int r = 0; r < NX; ++r) acc = fmaf(Ks[tid * NK + r], xk[r], acc);
            ut[tid] = acc;
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

// KKT certificate (the terms of `certificate` in solve.cuh).
template <class D>
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
    den = cta_max(c, den);
    uinf = cta_max(c, uinf);
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
            feas = fmaxf(feas, mm / (1.0f + fmax));
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
        feas = fmaxf(feas, fmaxf(gmax, 0.0f) / (1.0f + fmax));
        for (int sweep = 0; sweep < 100; ++sweep) {
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
    feas = cta_max(c, feas);
    stat = cta_max(c, stat);
    comp = cta_max(c, comp);
    return fmaxf(feas, fmaxf(stat / (1.0f + den), comp / (1.0f + uinf)));
}

// Faces re-read off Proj(u - alpha sigma w); returns whether any changed.
template <class D>
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
    return __syncthreads_or(changed);
}

template <class D>
__device__ void cta_write_output(const CCtx<D>& c, const RoundArgs& a, int b, int status, int iters, float kkt,
                                 int npol) {
    constexpr int NX = D::NX, NU = D::NU, CD = D::CD, M = D::M, F = D::F;
    const int Nv = a.N;
    const bool ok = status == kConverged || status == kMaxIter;
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
    if (c.tid == 0) {
        a.out_status[b] = status;
        a.out_iters[b] = iters;
        a.out_kkt[b] = ok ? kkt : INFINITY;
        a.out_npol[b] = npol;
        a.done[b] = 1;
    }
}

// Polish / certify / refine after a round: one CTA per instance.
template <class D>
__global__ void __launch_bounds__(kPT) polish_cta_kernel(RoundArgs a) {
    extern __shared__ __align__(16) float psm[];
    constexpr int NX = D::NX, NU = D::NU;
    const int b = blockIdx.x;
    if (a.done[b]) return;
    CCtx<D> c(a.N);
    c.sm = psm;
    c.rec = a.rec + (size_t)b * a.irec;
    c.modes = reinterpret_cast<uint32_t*>(c.sm + c.L.modes);
    c.K = a.Kst + (size_t)b * a.N * NU * (NX + 1);
    c.tid = threadIdx.x;
    c.lane = threadIdx.x & 31;
    c.warp = threadIdx.x >> 5;
    c.sigma = a.sigma;
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
    for (int i = c.tid; i < NX; i += kPT) c.xr()[i] = __ldg(tail + D::tXI0 + i);
    changed = __syncthreads_or(changed);
    int npol = a.out_npol[b];
    float kkt = INFINITY;
    if (a.polish && changed) {
        for (int e = c.tid; e < c.Nh * D::NC; e += kPT) glast[e] = c.modes[e];
        cta_polish<D>(c);
        ++npol;
        kkt = cta_certificate<D>(c);
        for (int r = 0; kkt > a.kkt_tol && r < a.refine_steps; ++r) {
            if (!cta_refine_modes<D>(c, a.refine_alpha)) break;
            cta_polish<D>(c);
            ++npol;
            kkt = cta_certificate<D>(c);
        }
        if (kkt <= a.kkt_tol) {
            cta_write_output<D>(c, a, b, kConverged, a.m1, kkt, npol);
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
            c.ur()[e] = st[((cb * 5 + VZ) * a.N + k) * D::NBP + NX + i];
        }
        cta_rollout<D>(c);
        kkt = cta_certificate<D>(c);
        if (kkt <= a.kkt_tol || final_round) {
            cta_write_output<D>(c, a, b, kkt <= a.kkt_tol ? kConverged : kMaxIter, a.m1, kkt, npol);
            return;
        }
    }
    if (c.tid == 0) {
        a.out_npol[b] = npol;
        atomicAdd(a.active, 1);
    }
}

}  // namespace pinmpc
