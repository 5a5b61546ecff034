// Two-site propagator gates exp(L_op * tau) in the normalised Pauli basis.
//
// L_op (16x16, index s1*4+s2) = bond commutator -i[K_ab, .] of Eq. (K_def)
// (each unordered bond once: K = J/2 (XX+YY) + Jz/2 ZZ) + w_a L_a (x) 1 +
// w_b 1 (x) L_b, with L_q the one-qubit Liouvillian of Eq. (H0) and
// Eqs. (D0)-(D2) and w_q = 1/deg(q).  All entries are real.
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
// exp by scaling and squaring with a truncated Taylor series (Moler & Van
// Loan, "Nineteen dubious ways to compute the exponential of a matrix",
// method 3): scale so ||A||_1 <= 1/4, sum 14 Taylor terms (remainder
// < 1e-21 relative), square back.  FP64 throughout.
#include "internal.h"

namespace mpdo {

namespace {

__device__ __forceinline__ int eps_sign(int j, int a) {
    // +1 for cyclic (X,Y), (Y,Z), (Z,X); -1 otherwise (j, a distinct, non-zero)
    return ((j % 3) + 1 == a) ? 1 : -1;
}

__device__ __forceinline__ bool anticommutes(int j, int a) { return a != 0 && a != j; }

__device__ double site_gen(const double* P, int n, int q, int r, int c) {
    // P = instance parameter block: h_x, h_y, h_z, g0, g1, g2 (each [n])
    const double hx = P[0 * n + q], hy = P[1 * n + q], hz = P[2 * n + q];
    const double g0 = P[3 * n + q], g1 = P[4 * n + q], g2 = P[5 * n + q];
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

__global__ void __launch_bounds__(256) build_gates_kernel(const GateSpec* specs, int n, int nb,
                                                          const double* params, double* gates) {
    __shared__ double A[256], E[256], T[256];
    __shared__ double colsum[16];
    __shared__ int s_shift;
    const GateSpec sp = specs[blockIdx.x];
    const int t = threadIdx.x, row = t >> 4, col = t & 15;
    double* out = gates + (size_t)blockIdx.x * 256;
    if (sp.kind == 1) {   // swap: |a,b>> -> |b,a>>
        const int a1 = row >> 2, a2 = row & 3, b1 = col >> 2, b2 = col & 3;
        out[t] = (a1 == b2 && a2 == b1) ? 1.0 : 0.0;
        return;
    }
    const double* P = params + (size_t)sp.b * (6 * n + 2 * nb);
    const double J = P[6 * n + sp.bond], Jz = P[6 * n + nb + sp.bond];
    const int a1 = row >> 2, a2 = row & 3, b1 = col >> 2, b2 = col & 3;
    double v = 0.0;
    if (a2 == b2) v += sp.wa * site_gen(P, n, sp.qa, a1, b1);
    if (a1 == b1) v += sp.wb * site_gen(P, n, sp.qb, a2, b2);
    for (int j = 1; j <= 3; ++j) {
        if ((j ^ b1) != a1 || (j ^ b2) != a2) continue;
        const double cj = (j == 3) ? 0.5 * Jz : 0.5 * J;
        const bool x1 = anticommutes(j, b1), x2 = anticommutes(j, b2);
        if (x1 && !x2) v += cj * 2.0 * eps_sign(j, b1);
        if (x2 && !x1) v += cj * 2.0 * eps_sign(j, b2);
    }
    A[t] = v * sp.tau;
    __syncthreads();
    // ||A||_1 and the scaling exponent
    if (t < 16) {
        double s = 0.0;
        for (int r = 0; r < 16; ++r) s += fabs(A[r * 16 + t]);
        colsum[t] = s;
    }
    __syncthreads();
    if (t == 0) {
        double nrm = 0.0;
        for (int c = 0; c < 16; ++c) nrm = fmax(nrm, colsum[c]);
        int s = 0;
        while (nrm > 0.25 && s < 60) {
            nrm *= 0.5;
            ++s;
        }
        s_shift = s;
    }
    __syncthreads();
    const int s = s_shift;
    A[t] = ldexp(A[t], -s);
    const double id = (row == col) ? 1.0 : 0.0;
    constexpr int kTerms = 14;
    __syncthreads();
    E[t] = id + A[t] / kTerms;   // Horner: E = I + A/k (I + A/(k+1)(...))
    __syncthreads();
    for (int k = kTerms - 1; k >= 1; --k) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 16; ++q) acc += A[row * 16 + q] * E[q * 16 + col];
        __syncthreads();
        E[t] = id + acc / k;
        __syncthreads();
    }
    for (int r = 0; r < s; ++r) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 16; ++q) acc += E[row * 16 + q] * E[q * 16 + col];
        T[t] = acc;
        __syncthreads();
        E[t] = T[t];
        __syncthreads();
    }
    out[t] = E[t];
}

}  // namespace

cudaError_t launch_build_gates(const GateSpec* d_specs, int count, int n, int nb, const double* d_params,
                               double* d_gates, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    build_gates_kernel<<<count, 256, 0, st>>>(d_specs, n, nb, d_params, d_gates);
    return cudaGetLastError();
}

}  // namespace mpdo
