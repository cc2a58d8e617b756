// Compile-time problem shape and the packed per-instance record layout.
#pragma once
#include <cstdint>

namespace pinmpc {

// Contact-set kinds: 3 = point force (f_x, f_y, f_z), 6 = foot wrench (f, tau).
// The generalized pyramid of a stance contact is {|t_j| <= c_j n, 0 <= n <= n_max};
// the normal component n is component 2 in both kinds.
template <int CD>
struct Cone;
template <>
struct Cone<3> {
    static constexpr int M = 2;  // tangential components
    __host__ __device__ static constexpr int tang(int j) { return j; }  // f_x, f_y
};
template <>
struct Cone<6> {
    static constexpr int M = 5;
    __host__ __device__ static constexpr int tang(int j) { return j < 2 ? j : j + 1; }  // fx fy tx ty tz
};

template <int NX_, int NU_, int CD_>
struct Dims {
    static constexpr int NX = NX_;
    static constexpr int NU = NU_;
    static constexpr int CD = CD_;
    static constexpr int NC = NU_ / CD_;          // contacts per stage
    static constexpr int NB = NX + NU;            // lifted dimension nbar = nx + nu
    // row split of the register-resident ADMM products: a row of T = [A B] is
    // held by two lanes, columns [0, CS) and [CS, 2 CS) (zero beyond NB)
    static constexpr int CS = (((NB + 1) / 2) + 3) & ~3;
    static constexpr int NBP = ((NB + 3) & ~3) > 2 * CS ? ((NB + 3) & ~3) : 2 * CS;  // padded vector stride
    static constexpr int M = Cone<CD>::M;         // tangential components per contact
    static constexpr int F = 2 * M + 2;           // faces per contact
    static constexpr int NRM = 2;                 // normal component index
    // per-stage record (floats): A | sigma*B | e | Q | sigma^2*R | r^y | r^u/sigma | mu | fmax/sigma | mask
    static constexpr int oA = 0;
    static constexpr int oB = oA + NX * NX;
    static constexpr int oE = oB + NX * NU;
    static constexpr int oQ = oE + NX;
    static constexpr int oR = oQ + NX;
    static constexpr int oRY = oR + NU;
    static constexpr int oRU = oRY + NX;
    static constexpr int oMU = oRU + NU;
    static constexpr int oFM = oMU + NC;
    static constexpr int oMASK = oFM + NC;
    static constexpr int SREC = (oMASK + 1 + 3) & ~3;
    // instance tail: xi_0 | u_{-1}/sigma | horizon (int bits) | input-check bits of the pack
    static constexpr int tXI0 = 0;
    static constexpr int tUP = NX;
    static constexpr int tH = NX + NU;
    static constexpr int tFLAG = NX + NU + 1;
    static constexpr int TAIL = (NX + NU + 2 + 3) & ~3;
    static_assert(NU % CD == 0, "nu must be a multiple of the contact dimension");
    static_assert(NB <= 64, "lifted dimension must fit two lanes per element");
    static_assert(NU <= 32 && NX <= 32, "one lane per row of the Riccati solve");
    static_assert(NC * F <= 64, "active-face bits must fit 64 bits per stage");
};

__host__ __device__ inline int instance_record_floats(int srec, int tail, int n_max) {
    return n_max * srec + tail;
}

}  // namespace pinmpc
