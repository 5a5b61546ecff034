// The two-site generator L_op of one gate (16x16, real, normalised Pauli
// basis, index s1*4+s2), shared by the gate builder and the adjoint.
//
// L_op = bond commutator -i[K_ab, .] of Eq. (K_def) (each unordered bond once:
// K = J/2 (XX+YY) + Jz/2 ZZ) + w_a L_a (x) 1 + w_b 1 (x) L_b, with L_q the
// one-qubit Liouvillian of Eq. (H0) and Eqs. (D0)-(D2) and w_q = 1/deg(q).
//
// One-qubit generator, written from the Bloch equations it encodes
// (r = (x, y, z), rho = (I + r.sigma)/2):  dr/dt = h x r  for H = h.sigma/2,
// D0: x,y decay at g0/2, z -> +1 at rate g0;  D1: x,y decay at g1/2,
// z -> -1 at rate g1;  D2: x,y decay at 2 g2.
//
// Bond generator from the Pauli product rule P_j P_a = w(j,a) P_{j xor a}
// (I=0, X=1, Y=2, Z=3; w = 1 if the two commute, else i*eps_{j a k}):
// -i[s_j s_j, P_a P_b] = 2 eps(j,a) P_{j^a} P_{j^b} if only the first factor
// anticommutes, 2 eps(j,b) ... if only the second does, 0 otherwise.
//
// L_op is linear in (h_x, h_y, h_z, g0, g1, g2) of both qubits and in (J, Jz),
// so its derivative with respect to one parameter is the generator with that
// parameter set to 1 and every other one to 0.
#pragma once

#include "internal.h"

namespace mpdo {

__device__ __forceinline__ int gen_eps_sign(int j, int a) {
    // +1 for cyclic (X,Y), (Y,Z), (Z,X); -1 otherwise (j, a distinct, non-zero)
    return ((j % 3) + 1 == a) ? 1 : -1;
}

__device__ __forceinline__ bool gen_anticommutes(int j, int a) { return a != 0 && a != j; }

// one-qubit generator entry (r, c), r, c in Pauli indices, from the six parameters
__device__ __forceinline__ double site_gen6(double hx, double hy, double hz, double g0, double g1, double g2, int r,
                                            int c) {
    const double gt = 0.5 * (g0 + g1) + 2.0 * g2;   // transverse decay
    switch (r * 4 + c) {
        case 1 * 4 + 1: return -gt;
        case 2 * 4 + 2: return -gt;
        case 3 * 4 + 3: return -(g0 + g1);
        case 3 * 4 + 0: return g0 - g1;
        case 1 * 4 + 2: return -hz;   // dx/dt = hy z - hz y
        case 1 * 4 + 3: return hy;
        case 2 * 4 + 1: return hz;    // dy/dt = hz x - hx z
        case 2 * 4 + 3: return -hx;
        case 3 * 4 + 1: return -hy;   // dz/dt = hx y - hy x
        case 3 * 4 + 2: return hx;
        default: return 0.0;
    }
}

// one-qubit generator entry with parameter u (0..5 = h_x, h_y, h_z, g0, g1, g2) at 1, the rest 0
__device__ __forceinline__ double site_gen_unit(int u, int r, int c) {
    return site_gen6(u == 0, u == 1, u == 2, u == 3, u == 4, u == 5, r, c);
}

// bond commutator entry ((a1 a2), (b1 b2)) for couplings J (XX+YY) and Jz (ZZ)
__device__ __forceinline__ double bond_gen(double J, double Jz, int a1, int a2, int b1, int b2) {
    double v = 0.0;
    for (int j = 1; j <= 3; ++j) {
        if ((j ^ b1) != a1 || (j ^ b2) != a2) continue;
        const double cj = (j == 3) ? 0.5 * Jz : 0.5 * J;
        const bool x1 = gen_anticommutes(j, b1), x2 = gen_anticommutes(j, b2);
        if (x1 && !x2) v += cj * 2.0 * gen_eps_sign(j, b1);
        if (x2 && !x1) v += cj * 2.0 * gen_eps_sign(j, b2);
    }
    return v;
}

// L_op entry (row, col) for instance parameter block P = [h_x, h_y, h_z, g0, g1, g2 (each [n]), J, Jz (each [nb])]
__device__ __forceinline__ double op_generator(const double* P, int n, int nb, const GateSpec& sp, int row,
                                               int col) {
    const int a1 = row >> 2, a2 = row & 3, b1 = col >> 2, b2 = col & 3;
    double v = 0.0;
    if (a2 == b2) {
        const int q = sp.qa;
        v += sp.wa * site_gen6(P[q], P[n + q], P[2 * n + q], P[3 * n + q], P[4 * n + q], P[5 * n + q], a1, b1);
    }
    if (a1 == b1) {
        const int q = sp.qb;
        v += sp.wb * site_gen6(P[q], P[n + q], P[2 * n + q], P[3 * n + q], P[4 * n + q], P[5 * n + q], a2, b2);
    }
    v += bond_gen(P[6 * n + sp.bond], P[6 * n + nb + sp.bond], a1, a2, b1, b2);
    return v;
}

}  // namespace mpdo
