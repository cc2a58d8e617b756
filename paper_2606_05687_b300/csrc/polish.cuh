// State shared by the round kernel (ADMM iterations) and the polish kernel
// (polish, certificate, refinement) of one instance between rounds, and the
// reduced input map both polish forms use.
#pragma once
#include "solve.cuh"

namespace pinmpc {

// Global-memory state of an instance between rounds.
template <class D>
struct RoundState {
    // [2 buffers][N stages][5 vars][NBP] ADMM variables (stage-major), then scalars
    __host__ __device__ static int var_floats(int N) { return 2 * 5 * N * D::NBP; }
    __host__ __device__ static int floats(int N) { return var_floats(N) + 8; }
    // offset of variable `which` of stage j in buffer buf
    __host__ __device__ static int at(int N, int buf, int j, int which) { return ((buf * N + j) * 5 + which) * D::NBP; }
    // scalar slots after the variables
    static constexpr int sAlpha = 0, sCprev = 1, sWgt = 2, sRestart = 3, sCb = 4;
};

// Horizon classes of one solve (mpc_set_horizon_classes): at most this many.
constexpr int kMaxClasses = 4;

struct RoundArgs {
    const float* rec;
    int irec, n_rec, N;
    float rho, sigma, kkt_tol, eta, dx, dy;
    float kkt_c;             // kkt_tol_abs / kkt_tol: the constant of the certificate's normalisations
    int max_iter, polish, accel, refine_steps;
    float refine_alpha;
    int m0, m1;              // this round runs iterations m0+1 .. m1
    float* cache;            // [B][N][2][NX][16]  S_j, W_j (padded rows)
    const int* flags;        // [B] input-check bits of factor_kernel
    float* state;            // [B][RoundState::floats(N)]
    uint32_t* modes;         // [B][N][NC] faces of the latest z
    uint32_t* lastm;         // [B][N][NC] faces of the last polished z
    int* done;               // [B] 1 once the instance has its final output
    // work of this round (persistent CTAs take instances from a cursor):
    // list_in[i], i < *cnt_in, or every i < B when list_in is null (round 0);
    // the polish appends the instances still running to list_out / *cnt_out
    const int* list_in;
    const int* cnt_in;
    int B;
    int* list_out;
    int* cnt_out;
    int* cursor;             // [2] work cursors of the round and polish kernels, zeroed per round
    int warm_B;              // instances b < warm_B start round 0 from the stored (shifted) iterate
    int dbl;                 // round kernel: records and factors arrive by TMA into two alternating buffers
    float* Kst;              // [B][N][NU + kNCB][NX+1] polish gains (and bound multiplier gains)
    float* out_xi;
    float* out_u;
    int* out_status;
    int* out_iters;
    float* out_kkt;
    unsigned long long* out_bits;
    int* out_npol;
    int* out_piv;            // [B] free pivots eliminated by the polish
    // horizon classes: the work lists hold one list per class (class c at
    // offset c * cls_stride of list_in / list_out, its count at cnt_in[c] /
    // cnt_out[c]); the polish kernel reads all ncls lists of list_in and
    // appends each running instance to its class's list of list_out.  A round
    // kernel launch serves one class: its list and count, and CTAs sized for
    // cap stages (every horizon of the class fits; N for a single class)
    int ncls, cls_stride, cap;
    int cls_cap[kMaxClasses];
    // state boxes X_k on xi_{k+1} (null: none set): [B][N][2][NX] lower, upper
    const float* xbox;
    uint32_t* smodes;        // [B][N] bounds the latest z sits at (bit i: lower, bit 16 + i: upper)
    uint32_t* slast;         // [B][N] the bounds of the last polish
};

// Augmented Lagrangian that holds active state bounds in the polish: the
// starting penalty of a bound, the factor it grows by whenever a step cuts
// that bound's violation by less than kBoxRate, its cap, the iteration limit
// and the stopping violation (relative).  A bound the inputs reach only
// through several stages (a position behind a velocity) is stiff: its
// multiplier converges at rate h / (h + penalty), h the cost of moving it,
// so its penalty has to grow past h.
constexpr float kBoxPenalty = 1e4f;
constexpr float kBoxGrow = 10.0f;
constexpr float kBoxRate = 0.1f;
constexpr float kBoxPenaltyMax = 1e7f;
constexpr int kBoxIters = 12;
// A polished point whose certificate misses the tolerance by at most a
// factor kStallBand is kept in the outputs; when kStallChecks later checks
// bring no improvement (the faces of the ADMM iterate unchanged, or a polish
// that does not halve the best certificate) the instance stops with that
// point (the FP32 floor of the certificate rises with the horizon: past ~40
// stages a few instances on the right faces sit above it)
// Coordinate-descent sweeps of the certificate's per-contact multiplier fit
// (measured: statuses, iterations and polishes unchanged from 100 sweeps on
// the walking, uneven and foot-wrench workloads; the foot-wrench batches,
// whose faces are more correlated, 3-9 % faster)
constexpr int kNnlsSweeps = 25;
constexpr float kStallBand = 4.0f;
constexpr int kStallChecks = 2;
constexpr float kBoxViol = 1e-7f;
// largest contraction rate from which the multiplier step extrapolates
constexpr float kBoxAitkenMax = 0.95f;
// weight of the certificate's terms of a state bound that the scan does not
// hold exactly (its violation and |nu (x - b)|): a bound the inputs reach only
// through a velocity (the CoM
// height) is stiff, with a large multiplier, so a small violation moves u
// (a relative 1.7e-6 was measured to move it by 3e-4) and a small slack on
// the feasible side moves the objective (by nu times the slack: relative
// gaps to 2.9e-6 at certificates near 1e-6); weighted 10x, a certified point
// holds its bounds, and their complementarity, to a tenth of the tolerance
constexpr float kBoxFeasWeight = 10.0f;
// At most this many active state bounds per stage are held exactly in the
// polish (an equality row added to the KKT system of a stage whose free
// inputs move the bounded quantity); the others go through the augmented
// Lagrangian above.
constexpr int kNCB = 4;
// A bound on a component no free input of its stage moves (a position behind
// a velocity) is carried back, as a row F on an earlier stage's state, to the
// first stage whose inputs reach it; at most this many are carried at once.
constexpr int kNPend = 8;

// Class of an instance with horizon Nh: the first class whose cap holds it;
// a horizon outside [1, N] goes to the last class (cap N), whose round kernel
// reports it.
__host__ __device__ inline int horizon_class(int Nh, int N, int ncls, const int* caps) {
    if (Nh >= 1 && Nh <= N)
        for (int c = 0; c + 1 < ncls; ++c)
            if (Nh <= caps[c]) return c;
    return ncls - 1;
}

// Round 0 with several classes: instance b of the batch goes to its class's
// list (list_out / cnt_out of `a`, counts zeroed before).  Order within a
// list is arbitrary: every instance is solved on its own.
template <class D>
__global__ void bin_classes_kernel(RoundArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.B) return;
    const float* tail = a.rec + (size_t)b * a.irec + (size_t)a.n_rec * D::SREC;
    const int cl = horizon_class(__float_as_int(tail[D::tH]), a.N, a.ncls, a.cls_cap);
    a.list_out[(size_t)cl * a.cls_stride + atomicAdd(a.cnt_out + cl, 1)] = b;
}

// Next instance for a persistent CTA (all threads get the same value), or -1
// when the round's list is exhausted; `which` selects the kernel's cursor.
// Starts with a barrier, so the CTA's shared memory is free for the next item.
__device__ __forceinline__ int next_instance(const RoundArgs& a, int which, int* slot) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int i = atomicAdd(a.cursor + which, 1);
        const int n = a.list_in ? *a.cnt_in : a.B;
        *slot = (i < n) ? (a.list_in ? a.list_in[i] : i) : -1;
    }
    __syncthreads();
    return *slot;
}

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

}  // namespace pinmpc
