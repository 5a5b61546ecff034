// Kernels of the adjoint (reverse-mode gradient) of the Trotter sweep.
//
// The paper has no gradient; this is the reverse mode of the update it
// describes (App. B two-site update, Sec. 2.3 observables), op by op:
//
//   forward op:  Theta = A B, Theta' = G Theta, theta~ = D Theta' with
//                D = diag(lambda_{p-1}) (x) 1_4, theta~ = U S V^T, k kept,
//                lambda_p = s_k, B_{p+1}' = V_k^T, B_p' = Theta' V_k.
//   backward:    V-bar_k = B-bar_{p+1}'^T + Theta'^T B-bar_p',
//                theta~-bar = theta~ H with (eigen-perturbation of C = theta~^T theta~,
//                eigenvalues s_i^2, the complement of the c computed vectors
//                carrying eigenvalue 0)
//                  H = V_c Om V_k^T + V_k [diag(s-bar/s) V_k^T + (Om^T - S_k^-2 K^T) V_c^T
//                      + S_k^-2 V-bar_k^T],
//                  K = V_c^T V-bar_k,  Om_ij = F_ij K_ij (i != j),
//                  F_ij = 1/(s_j^2 - s_i^2), Lorentzian-broadened to
//                  D/(D^2 + delta^2), D = s_j^2 - s_i^2, delta = eps s_0^2,
//                  and 0 inside a degenerate pair (|s_i - s_j| <= 1e-10 max),
//                so theta~-bar = D [(Theta' V_k) H_k + (Theta' V_c Om) V_k^T]
//                with H_k = Mk V_c^T + S_k^-2 V-bar_k^T, Mk = Om^T - S_k^-2 K^T + diag(s-bar/s);
//                Theta'-bar = D theta~-bar + B-bar_p' V_k^T,
//                lambda-bar_{p-1}[l] += sum over (l, s1) rows of theta~-bar o Theta',
//                G-bar += sum_{l,r} Theta'-bar Theta^T (per (l, r) pair, 16 x 16),
//                Theta-bar = G^T Theta'-bar, A-bar = Theta-bar B^T, B-bar = A^T Theta-bar.
//   parameters:  X = tau L_op, G = exp(X): X-bar = L_exp(X^T, G-bar), the top
//                right block of exp([[X^T, G-bar], [0, X^T]]) (Van Loan, "Computing
//                integrals involving the matrix exponential", 1978), L-bar = tau X-bar,
//                d/dtheta = <L-bar, dL_op/dtheta> (L_op is linear in the parameters).
//
// The dense products run in the batched GEMM (gemm.cu); this file holds the
// element-wise and reduction steps between them, the loss cotangent at the
// final state and the parameter gradient.  FP64 throughout.
#include <mpdo.h>

#include <algorithm>

#include "generator.cuh"
#include "internal.h"

namespace mpdo {

namespace {

constexpr int CT = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// batched strided copy (one warp per row)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CT) copy2d_kernel(const Copy2D* descs) {
    const Copy2D d = descs[blockIdx.y];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * (CT / 32) + warp; i < d.rows; i += gridDim.x * (CT / 32)) {
        double* dst = d.dst + (size_t)i * d.dst_ld;
        if (d.src) {
            const double* src = d.src + (size_t)i * d.src_ld;
            for (int j = lane; j < d.cols; j += 32) dst[j] = d.scale * src[j];
        } else {
            for (int j = lane; j < d.cols; j += 32) dst[j] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// truncated-SVD backward: Om, Mk, V-bar scaling, stacked operands
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CT) svd_bwd_coeffs_kernel(const BwdDesc* descs, double eps, double deg_tol) {
    const BwdDesc& d = descs[blockIdx.y];
    const int c = d.c, k = d.k, n = d.n;
    const double s0 = d.s[0];
    const double delta = eps * s0 * s0;
    // V spans all of R^n (c == n, no zeroed row): the projector I - V V^T
    // vanishes, so its two terms (-S^-2 K^T V and S^-2 V-bar) are dropped
    // exactly instead of cancelling in rounding
    const bool complete = (c == n) && (d.s[c - 1] > 0.0);
    const size_t e1 = (size_t)c * k, e2 = e1 + (size_t)k * n;
    for (size_t e = (size_t)blockIdx.x * CT + threadIdx.x; e < e2; e += (size_t)gridDim.x * CT) {
        if (e < e1) {
            const int i = (int)(e / k), j = (int)(e % k);
            const double kij = d.K[e];
            const double si = d.s[i], sj = d.s[j];
            const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
            // pairs equal to deg_tol (relative) span one degenerate subspace:
            // the loss does not change under rotations inside it, so the
            // exact coefficient is 0 (rounding splits such pairs by ~1 ulp,
            // and 1/(s_j^2 - s_i^2) would amplify rounding noise instead)
            double om = 0.0;
            if (i != j && !(fabs(sj - si) <= deg_tol * fmax(si, sj))) {
                const double D = sj * sj - si * si;
                const double den = D * D + delta * delta;
                om = den > 0.0 ? D / den * kij : 0.0;
            }
            d.Om[e] = om;
            d.Mk[(size_t)j * c + i] = om - (complete ? 0.0 : kij * inv * inv) + (i == j ? d.sbar[j] * inv : 0.0);
        } else {
            const size_t f = e - e1;
            const int j = (int)(f / n);
            const double sj = d.s[j];
            const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
            d.Vbar[f] = complete ? 0.0 : d.Vbar[f] * inv * inv;
            const double v = d.V[f];       // row j < k of V, same offset
            d.S2[f] = v;                   // rows 0..k-1
            d.S3[(size_t)k * n + f] = v;   // rows k..2k-1
        }
    }
}

// lambda-bar_{p-1}[l] += lambda_l * sum_{s1, col} X1 o Theta'  and  X1 rows *= lambda_l^2
__global__ void __launch_bounds__(CT) lambda_bwd_kernel(const BwdDesc* descs) {
    const BwdDesc& d = descs[blockIdx.y];
    if (!d.lam) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = d.n;
    for (int l = blockIdx.x * (CT / 32) + warp; l < d.cl; l += gridDim.x * (CT / 32)) {
        const double lam = d.lam[l];
        const double l2 = lam * lam;
        double dot = 0.0;
        for (int s1 = 0; s1 < 4; ++s1) {
            double* x = d.X1 + (size_t)(l * 4 + s1) * n;
            const double* t = d.thetap + (size_t)(l * 4 + s1) * n;
            for (int j = lane; j < n; j += 32) {
                const double v = x[j];
                dot = fma(v, t[j], dot);
                x[j] = v * l2;
            }
        }
        dot = warp_sum_d(dot);
        if (lane == 0) d.lbar_left[l] += lam * dot;
    }
}

// ---------------------------------------------------------------------------
// gate backward: G-bar partial sums and Theta-bar = G^T Theta'-bar (in place)
// ---------------------------------------------------------------------------
constexpr int GP = 64;   // (l, r) pairs per tile

__global__ void __launch_bounds__(CT) gate_bwd_kernel(const BwdDesc* descs) {
    const BwdDesc& d = descs[blockIdx.y];
    __shared__ double xs[16][GP + 1], ys[16][GP + 1], Gs[256];
    const int t = threadIdx.x;
    Gs[t] = d.G[t];
    const int cr = d.cr, n = d.n;
    const int np = d.cl * cr;
    const int ga = t >> 4, gb = t & 15;
    double acc = 0.0;
    for (int base = blockIdx.x * GP; base < np; base += gridDim.x * GP) {
        __syncthreads();
        for (int e = t; e < 16 * GP; e += CT) {
            const int a = e / GP, i = e % GP;
            const int pr = base + i;
            double xv = 0.0, yv = 0.0;
            if (pr < np) {
                const int l = pr / cr, r = pr % cr;
                const size_t addr = (size_t)(l * 4 + (a >> 2)) * n + (a & 3) * cr + r;
                xv = d.X2[addr];
                yv = d.X1[addr];
            }
            xs[a][i] = xv;
            ys[a][i] = yv;
        }
        __syncthreads();
#pragma unroll 8
        for (int i = 0; i < GP; ++i) acc = fma(xs[ga][i], ys[gb][i], acc);
        for (int e = t; e < 16 * GP; e += CT) {
            const int b = e / GP, i = e % GP;
            const int pr = base + i;
            if (pr >= np) continue;
            double v = 0.0;
#pragma unroll
            for (int a = 0; a < 16; ++a) v = fma(Gs[a * 16 + b], xs[a][i], v);
            const int l = pr / cr, r = pr % cr;
            d.X2[(size_t)(l * 4 + (b >> 2)) * n + (b & 3) * cr + r] = v;
        }
    }
    d.gpart[(size_t)blockIdx.x * 256 + t] = acc;
}

__global__ void __launch_bounds__(256) gbar_reduce_kernel(const BwdDesc* descs, int parts) {
    const BwdDesc& d = descs[blockIdx.x];
    if (!d.is_gate) return;
    double s = 0.0;
    for (int p = 0; p < parts; ++p) s += d.gpart[(size_t)p * 256 + threadIdx.x];
    d.gacc[threadIdx.x] += s;
}

// ---------------------------------------------------------------------------
// loss cotangent at the final state
//
// With E(string) the product of the selected Pauli slices (measure.cu),
// Z = E(I..I), e_i = E(z_i)/Z, e_ij = E(z_i z_j)/Z and
// L = sum_i a_i e_i + sum_{i<j} W_ij (e_ij - e_i e_j):
//   dL = (1/Z) [ sum_{i<j} W_ij dE_ij + sum_i b_i dE_i - c dZ ],
//   b_i = a_i - sum_{j != i} W_ij e_j,
//   c = sum_i a_i e_i + sum_{i<j} W_ij (e_ij - 2 e_i e_j).
// dE(string)/dB_k[l][s][r] = (prefix env)[l] (suffix env)[r] when the string
// has Pauli s at k.  Environments (row vectors on the left of site k, column
// vectors on the right):
//   L0[k]       = prod_{q<k} M_q^I,         R0[p]    = prod_{q>=p} M_q^I
//   L1[k][i]    = Z at i < k, I elsewhere,  R1[p][j] = Z at j >= p
//   L2[k]       = sum_{i<j<k} W_ij (Z at i, j),  R2[p] = sum_{p<=i<j} W_ij (Z at i, j)
// ---------------------------------------------------------------------------
constexpr int LT = 512;

__device__ __forceinline__ const double* site_c(const double* sites, int b, int p, int n, int cap) {
    return sites + ((size_t)b * n + p) * (size_t)cap * 4 * cap;
}

// out[r] = sum_l in[l] M[l][a][r]  (r < cr)
__device__ __forceinline__ void left_mul(const double* M, int a, int cl, int cr, int cap, const double* in,
                                         double* out) {
    for (int r = threadIdx.x; r < cr; r += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < cl; ++l) acc = fma(in[l], M[((size_t)l * 4 + a) * cap + r], acc);
        out[r] = acc;
    }
}

// out[l] = sum_r M[l][a][r] in[r]  (l < cl), one warp per l
__device__ __forceinline__ void right_mul(const double* M, int a, int cl, int cr, int cap, const double* in,
                                          double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int l = warp; l < cl; l += nw) {
        const double* row = M + ((size_t)l * 4 + a) * cap;
        double acc = 0.0;
        for (int r = lane; r < cr; r += 32) acc = fma(row[r], in[r], acc);
        acc = warp_sum_d(acc);
        if (lane == 0) out[l] = acc;
    }
}

struct EnvIdx {
    int n, cap;
    __device__ size_t v(int b, int k) const { return ((size_t)b * (n + 1) + k) * cap; }                 // L0, L2, R0, R2
    __device__ size_t w(int b, int k, int i) const { return (((size_t)b * (n + 1) + k) * n + i) * cap; }  // L1, R1
};

__global__ void __launch_bounds__(LT) env0_kernel(const double* sites, const int* dims, int n, int cap,
                                                  LossScratch s) {
    const int b = blockIdx.x;
    const int* dm = dims + (size_t)b * (n + 1);
    const EnvIdx ix{n, cap};
    if (blockIdx.y == 0) {
        if (threadIdx.x == 0) s.L0[ix.v(b, 0)] = 1.0;
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            left_mul(site_c(sites, b, k, n, cap), 0, dm[k], dm[k + 1], cap, s.L0 + ix.v(b, k), s.L0 + ix.v(b, k + 1));
            __syncthreads();
        }
    } else {
        if (threadIdx.x == 0) s.R0[ix.v(b, n)] = 1.0;
        __syncthreads();
        for (int p = n - 1; p >= 0; --p) {
            right_mul(site_c(sites, b, p, n, cap), 0, dm[p], dm[p + 1], cap, s.R0 + ix.v(b, p + 1),
                      s.R0 + ix.v(b, p));
            __syncthreads();
        }
    }
}

// blockIdx.x = the qubit carrying Z
__global__ void __launch_bounds__(LT) env1_kernel(const double* sites, const int* dims, int n, int cap,
                                                  LossScratch s) {
    const int i = blockIdx.x, b = blockIdx.y;
    const int* dm = dims + (size_t)b * (n + 1);
    const EnvIdx ix{n, cap};
    if (blockIdx.z == 0) {
        left_mul(site_c(sites, b, i, n, cap), 3, dm[i], dm[i + 1], cap, s.L0 + ix.v(b, i), s.L1 + ix.w(b, i + 1, i));
        __syncthreads();
        for (int k = i + 1; k < n; ++k) {
            left_mul(site_c(sites, b, k, n, cap), 0, dm[k], dm[k + 1], cap, s.L1 + ix.w(b, k, i),
                     s.L1 + ix.w(b, k + 1, i));
            __syncthreads();
        }
    } else {
        const int j = i;
        right_mul(site_c(sites, b, j, n, cap), 3, dm[j], dm[j + 1], cap, s.R0 + ix.v(b, j + 1), s.R1 + ix.w(b, j, j));
        __syncthreads();
        for (int p = j - 1; p >= 0; --p) {
            right_mul(site_c(sites, b, p, n, cap), 0, dm[p], dm[p + 1], cap, s.R1 + ix.w(b, p + 1, j),
                      s.R1 + ix.w(b, p, j));
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(LT) env2_kernel(const double* sites, const int* dims, int n, int cap,
                                                  const double* W, LossScratch s) {
    const int b = blockIdx.x;
    const int* dm = dims + (size_t)b * (n + 1);
    const double* Wb = W + (size_t)b * n * n;
    const EnvIdx ix{n, cap};
    __shared__ double tmp[kMaxChi], t2[kMaxChi], t3[kMaxChi];
    if (blockIdx.y == 0) {
        if (threadIdx.x == 0) s.L2[ix.v(b, 0)] = 0.0;
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            const int cl = dm[k], cr = dm[k + 1];
            for (int l = threadIdx.x; l < cl; l += blockDim.x) {
                double acc = 0.0;
                for (int i = 0; i < k; ++i) acc = fma(Wb[(size_t)i * n + k], s.L1[ix.w(b, k, i) + l], acc);
                tmp[l] = acc;
            }
            __syncthreads();
            const double* M = site_c(sites, b, k, n, cap);
            left_mul(M, 0, cl, cr, cap, s.L2 + ix.v(b, k), t2);
            left_mul(M, 3, cl, cr, cap, tmp, t3);
            __syncthreads();
            for (int r = threadIdx.x; r < cr; r += blockDim.x) s.L2[ix.v(b, k + 1) + r] = t2[r] + t3[r];
            __syncthreads();
        }
    } else {
        if (threadIdx.x == 0) s.R2[ix.v(b, n)] = 0.0;
        __syncthreads();
        for (int p = n - 1; p >= 0; --p) {
            const int cl = dm[p], cr = dm[p + 1];
            for (int r = threadIdx.x; r < cr; r += blockDim.x) {
                double acc = 0.0;
                for (int j = p + 1; j < n; ++j) acc = fma(Wb[(size_t)p * n + j], s.R1[ix.w(b, p + 1, j) + r], acc);
                tmp[r] = acc;
            }
            __syncthreads();
            const double* M = site_c(sites, b, p, n, cap);
            right_mul(M, 0, cl, cr, cap, s.R2 + ix.v(b, p + 1), t2);
            right_mul(M, 3, cl, cr, cap, tmp, t3);
            __syncthreads();
            for (int l = threadIdx.x; l < cl; l += blockDim.x) s.R2[ix.v(b, p) + l] = t2[l] + t3[l];
            __syncthreads();
        }
    }
}

// coef[b] = (b_0 .. b_{n-1}, c, Z, L)
__global__ void __launch_bounds__(256) loss_coef_kernel(int n, int cap, const double* a, const double* W,
                                                        LossScratch s) {
    const int b = blockIdx.x;
    const EnvIdx ix{n, cap};
    const double* Wb = W + (size_t)b * n * n;
    const double* ab = a + (size_t)b * n;
    double* coef = s.coef + (size_t)b * (n + 3);
    const double Z = s.L0[ix.v(b, n)];
    const double iz = Z != 0.0 ? 1.0 / Z : 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double acc = ab[i];
        for (int j = 0; j < n; ++j)
            if (j != i) acc -= Wb[(size_t)i * n + j] * s.L1[ix.w(b, n, j)] * iz;
        coef[i] = acc;
    }
    if (threadIdx.x == 0) {
        double lin = 0.0, prod = 0.0;
        for (int i = 0; i < n; ++i) {
            const double ei = s.L1[ix.w(b, n, i)] * iz;
            lin += ab[i] * ei;
            for (int j = i + 1; j < n; ++j) prod += Wb[(size_t)i * n + j] * ei * s.L1[ix.w(b, n, j)] * iz;
        }
        const double pair = s.L2[ix.v(b, n)] * iz;
        coef[n] = lin + pair - 2.0 * prod;
        coef[n + 1] = Z;
        coef[n + 2] = lin + pair - prod;
    }
}

// sbar site k of instance b: slices I and Z (X, Y zero), divided by Z
__global__ void __launch_bounds__(LT) loss_assemble_kernel(const int* dims, int n, int cap, const double* W,
                                                           LossScratch s, double* sbar) {
    const int k = blockIdx.x, b = blockIdx.y;
    const int* dm = dims + (size_t)b * (n + 1);
    const int cl = dm[k], cr = dm[k + 1];
    const EnvIdx ix{n, cap};
    const double* Wb = W + (size_t)b * n * n;
    const double* coef = s.coef + (size_t)b * (n + 3);
    const double Z = coef[n + 1];
    const double iz = Z != 0.0 ? 1.0 / Z : 0.0;
    const double cc = coef[n];
    __shared__ double lz[kMaxChi], li[kMaxChi], l0[kMaxChi], rz[kMaxChi], ri[kMaxChi], r0[kMaxChi];
    double* T = s.T + (((size_t)b * n + k) * n) * cap;   // T[j][l], j > k
    for (int l = threadIdx.x; l < cl; l += blockDim.x) {
        const double v0 = s.L0[ix.v(b, k) + l];
        double az = coef[k] * v0, ai = -cc * v0 + s.L2[ix.v(b, k) + l];
        for (int i = 0; i < k; ++i) {
            const double v1 = s.L1[ix.w(b, k, i) + l];
            az = fma(Wb[(size_t)i * n + k], v1, az);
            ai = fma(coef[i], v1, ai);
        }
        l0[l] = v0;
        lz[l] = az;
        li[l] = ai;
    }
    for (int r = threadIdx.x; r < cr; r += blockDim.x) {
        double az = 0.0, ai = s.R2[ix.v(b, k + 1) + r];
        for (int j = k + 1; j < n; ++j) {
            const double v1 = s.R1[ix.w(b, k + 1, j) + r];
            az = fma(Wb[(size_t)k * n + j], v1, az);
            ai = fma(coef[j], v1, ai);
        }
        r0[r] = s.R0[ix.v(b, k + 1) + r];
        rz[r] = az;
        ri[r] = ai;
    }
    const int nj = n - k - 1;
    for (int e = threadIdx.x; e < nj * cl; e += blockDim.x) {
        const int j = k + 1 + e / cl, l = e % cl;
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc = fma(Wb[(size_t)i * n + j], s.L1[ix.w(b, k, i) + l], acc);
        T[(size_t)j * cap + l] = acc;
    }
    __syncthreads();
    double* S = sbar + ((size_t)b * n + k) * (size_t)cap * 4 * cap;
    for (int e = threadIdx.x; e < cl * cr; e += blockDim.x) {
        const int l = e / cr, r = e % cr;
        double vi = fma(li[l], r0[r], l0[l] * ri[r]);
        for (int j = k + 1; j < n; ++j) vi = fma(T[(size_t)j * cap + l], s.R1[ix.w(b, k + 1, j) + r], vi);
        const double vz = fma(lz[l], r0[r], l0[l] * rz[r]);
        double* row = S + (size_t)l * 4 * cap + r;
        row[0] = vi * iz;
        row[(size_t)cap] = 0.0;
        row[(size_t)2 * cap] = 0.0;
        row[(size_t)3 * cap] = vz * iz;
    }
}

// ---------------------------------------------------------------------------
// parameter gradient
// ---------------------------------------------------------------------------
constexpr int kContrib = 14;   // qa: 6 on-site, qb: 6 on-site, J, Jz

__global__ void __launch_bounds__(1024) frechet_kernel(const GateSpec* specs, int n, int nb, const double* params,
                                                       const double* gacc, double* contrib) {
    const int id = blockIdx.x;
    const GateSpec sp = specs[id];
    const int t = threadIdx.x, row = t >> 5, col = t & 31;
    double* out = contrib + (size_t)id * kContrib;
    if (sp.kind == 1) {
        if (t < kContrib) out[t] = 0.0;
        return;
    }
    __shared__ double X[256], Gb[256], Lb[256];
    __shared__ double A[1024], E[1024], T[1024];
    __shared__ double colsum[32];
    __shared__ double s_gamma;
    __shared__ int s_shift;
    const double* P = params + (size_t)sp.b * (6 * n + 2 * nb);
    if (t < 256) {
        X[t] = sp.tau * op_generator(P, n, nb, sp, t >> 4, t & 15);
        Gb[t] = gacc[(size_t)id * 256 + t];
    }
    __syncthreads();
    // ||X^T||_1 (row sums of X) and ||G-bar||_1 (column sums)
    if (t < 16) {
        double s = 0.0;
        for (int c = 0; c < 16; ++c) s += fabs(X[t * 16 + c]);
        colsum[t] = s;
    } else if (t < 32) {
        double s = 0.0;
        for (int r = 0; r < 16; ++r) s += fabs(Gb[r * 16 + (t - 16)]);
        colsum[t] = s;
    }
    __syncthreads();
    if (t == 0) {
        double nx = 0.0, ng = 0.0;
        for (int c = 0; c < 16; ++c) {
            nx = fmax(nx, colsum[c]);
            ng = fmax(ng, colsum[16 + c]);
        }
        // G-bar enters linearly: scale it to the size of X (or 1) and undo after
        const double target = nx > 0.0 ? nx : 1.0;
        s_gamma = ng > 0.0 ? ng / target : 0.0;
        double nrm = nx + (ng > 0.0 ? target : 0.0);
        int s = 0;
        while (nrm > 0.25 && s < 60) {
            nrm *= 0.5;
            ++s;
        }
        s_shift = s;
    }
    __syncthreads();
    const double gamma = s_gamma;
    if (gamma == 0.0) {
        if (t < kContrib) out[t] = 0.0;
        return;
    }
    // M = [[X^T, G-bar / gamma], [0, X^T]] scaled by 2^-s
    {
        double v = 0.0;
        if (row < 16 && col < 16) v = X[col * 16 + row];
        else if (row < 16) v = Gb[row * 16 + (col - 16)] / gamma;
        else if (col >= 16) v = X[(col - 16) * 16 + (row - 16)];
        A[t] = ldexp(v, -s_shift);
    }
    const double id1 = (row == col) ? 1.0 : 0.0;
    constexpr int kTerms = 14;
    __syncthreads();
    E[t] = id1 + A[t] / kTerms;   // Horner: E = I + A/k (I + A/(k+1)(...))
    __syncthreads();
    for (int k = kTerms - 1; k >= 1; --k) {
        double acc = 0.0;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) acc = fma(A[row * 32 + q], E[q * 32 + col], acc);
        __syncthreads();
        E[t] = id1 + acc / k;
        __syncthreads();
    }
    for (int r = 0; r < s_shift; ++r) {
        double acc = 0.0;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) acc = fma(E[row * 32 + q], E[q * 32 + col], acc);
        T[t] = acc;
        __syncthreads();
        E[t] = T[t];
        __syncthreads();
    }
    if (row < 16 && col >= 16) Lb[row * 16 + (col - 16)] = sp.tau * gamma * E[t];
    __syncthreads();
    // <L-bar, dL_op/dtheta> for the 14 parameters the op depends on
    const int warp = t >> 5, lane = t & 31;
    if (warp < kContrib) {
        double acc = 0.0;
        for (int e = lane; e < 256; e += 32) {
            const int a1 = e >> 6, a2 = (e >> 4) & 3, b1 = (e >> 2) & 3, b2 = e & 3;
            double u;
            if (warp < 6)
                u = (a2 == b2) ? sp.wa * site_gen_unit(warp, a1, b1) : 0.0;
            else if (warp < 12)
                u = (a1 == b1) ? sp.wb * site_gen_unit(warp - 6, a2, b2) : 0.0;
            else
                u = bond_gen(warp == 12 ? 1.0 : 0.0, warp == 13 ? 1.0 : 0.0, a1, a2, b1, b2);
            acc = fma(Lb[e], u, acc);
        }
        acc = warp_sum_d(acc);
        if (lane == 0) out[warp] = acc;
    }
}

// grad[b][q] = sum over the ops of instance b (in op order) of the contributions to q
__global__ void __launch_bounds__(256) param_reduce_kernel(const GateSpec* specs, int n, int nb, int n_ops,
                                                           const double* contrib, double* grad) {
    const int b = blockIdx.x;
    const int P = 6 * n + 2 * nb;
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        double acc = 0.0;
        for (int op = 0; op < n_ops; ++op) {
            const size_t id = (size_t)b * n_ops + op;
            const GateSpec& sp = specs[id];
            if (sp.kind == 1) continue;
            const double* cb = contrib + id * kContrib;
            if (q < 6 * n) {
                const int u = q / n, qq = q % n;
                if (sp.qa == qq) acc += cb[u];
                if (sp.qb == qq) acc += cb[6 + u];
            } else if (q < 6 * n + nb) {
                if (sp.bond == q - 6 * n) acc += cb[12];
            } else if (sp.bond == q - 6 * n - nb) {
                acc += cb[13];
            }
        }
        grad[(size_t)b * P + q] = acc;
    }
}

}  // namespace

cudaError_t launch_copy2d(const Copy2D* d_desc, int count, int max_rows, cudaStream_t st) {
    if (count <= 0 || max_rows <= 0) return cudaSuccess;
    const int gx = std::min((max_rows + CT / 32 - 1) / (CT / 32), 128);
    for (int c0 = 0; c0 < count; c0 += 65535) {
        const int cnt = std::min(count - c0, 65535);
        copy2d_kernel<<<dim3(gx, cnt), CT, 0, st>>>(d_desc + c0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_svd_bwd_coeffs(const BwdDesc* d_desc, int nops, double rel_broadening, double rel_degenerate,
                                  cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    svd_bwd_coeffs_kernel<<<dim3(256, nops), CT, 0, st>>>(d_desc, rel_broadening, rel_degenerate);
    return cudaGetLastError();
}

cudaError_t launch_lambda_bwd(const BwdDesc* d_desc, int nops, int max_cl, cudaStream_t st) {
    if (nops <= 0 || max_cl <= 0) return cudaSuccess;
    const int gx = std::min((max_cl + CT / 32 - 1) / (CT / 32), 64);
    lambda_bwd_kernel<<<dim3(gx, nops), CT, 0, st>>>(d_desc);
    return cudaGetLastError();
}

cudaError_t launch_gate_bwd(const BwdDesc* d_desc, int nops, int parts, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    gate_bwd_kernel<<<dim3(parts, nops), CT, 0, st>>>(d_desc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gbar_reduce_kernel<<<nops, 256, 0, st>>>(d_desc, parts);
    return cudaGetLastError();
}

cudaError_t launch_loss_cotangent(const double* sites, const int* dims, int n, int B, int chi_cap, const double* a,
                                  const double* W, const LossScratch& s, double* sbar, cudaStream_t st) {
    env0_kernel<<<dim3(B, 2), LT, 0, st>>>(sites, dims, n, chi_cap, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    env1_kernel<<<dim3(n, B, 2), LT, 0, st>>>(sites, dims, n, chi_cap, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    env2_kernel<<<dim3(B, 2), LT, 0, st>>>(sites, dims, n, chi_cap, W, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    loss_coef_kernel<<<B, 256, 0, st>>>(n, chi_cap, a, W, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    loss_assemble_kernel<<<dim3(n, B), LT, 0, st>>>(dims, n, chi_cap, W, s, sbar);
    return cudaGetLastError();
}

cudaError_t launch_param_grad(const GateSpec* d_specs, int count, int n, int nb, const double* d_params,
                              const double* gacc, double* contrib, int B, int n_ops, double* grad, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    frechet_kernel<<<count, 1024, 0, st>>>(d_specs, n, nb, d_params, gacc, contrib);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    param_reduce_kernel<<<B, 256, 0, st>>>(d_specs, n, nb, n_ops, contrib, grad);
    return cudaGetLastError();
}

}  // namespace mpdo
