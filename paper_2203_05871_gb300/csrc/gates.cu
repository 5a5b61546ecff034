// Two-site propagator gates exp(L_op * tau) in the normalised Pauli basis,
// with L_op as defined in generator.cuh.
//
// exp by scaling and squaring with a truncated Taylor series (Moler & Van
// Loan, "Nineteen dubious ways to compute the exponential of a matrix",
// method 3): scale so ||A||_1 <= 1/4, sum 14 Taylor terms (remainder
// < 1e-21 relative), square back.  FP64 throughout.
#include "generator.cuh"
#include "internal.h"

namespace mpdo {

namespace {

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
    A[t] = op_generator(P, n, nb, sp, row, col) * sp.tau;
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
