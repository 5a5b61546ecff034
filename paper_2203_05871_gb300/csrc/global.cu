// Global characteristics of the state (Sec. 2.3): the second Renyi entropy
// S2 = -ln tr(rho^2) (Eq. (S_2)) and the operator space entanglement entropy
// of the vectorised state |rho>> for a cut of the MPO path (Eq. (OSEE)).
//
// The basis P_a/sqrt2 is orthonormal for the trace inner product, so
// tr(rho^2) = sum_a r_a^2 = <<rho|rho>>, the squared norm of the coefficient
// MPS, and for the normalised rho tr(rho^2) = <<rho|rho>> / (tr rho)^2.
//
// Gram matrices of the two halves of the chain at bond p (between positions
// p and p+1), both chi x chi with chi = dims[p+1]:
//   X_0 = [1],      X_{q+1} = sum_s B_q[s]^T X_q B_q[s]      (q = 0 .. p)
//   Y_N = [1],      Y_q     = sum_s B_q[s] Y_{q+1} B_q[s]^T  (q = N-1 .. p+1)
// With r = M_L M_R through the bond index, X = M_L^T M_L and Y = M_R M_R^T, and
// the squared Schmidt values of |rho>> at the cut are the eigenvalues of X Y.
// Each Gram matrix is factored by the one-sided Jacobi SVD of its rows
// (X = V diag(x) V^T, rows w_j = x_j v_j^T after convergence), F_X = rows
// w_j / sqrt(x_j) with F_X^T F_X = X, and likewise F_Y; then eig(X Y) =
// sv(F_X F_Y^T)^2, so a third Jacobi SVD, of C = F_X F_Y^T, gives the Schmidt
// values s_k and OSEE = -sum_k p_k ln p_k with p_k = s_k^2 / sum s^2.
// FP64 throughout: the Gram sweeps are batched FP64 GEMMs (gemm.cu), the SVDs
// the FP64 pass of jacobi.cu at its strict tolerance sqrt(L) eps.  Squaring
// the bond matrix into X and Y costs accuracy only on the smallest p_k, at the
// 1e-16 level of the largest, which moves the entropy by ~1e-14.
#include <mpdo.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ctx.h"
#include "internal.h"

using namespace mpdo;

namespace mpdo {

namespace {

// X and Y of instance i of a chunk: W slots 2i and 2i+1; [0][0] = 1
__global__ void gram_unit_kernel(double* W, size_t mat, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * m) return;
    W[(size_t)i * mat] = 1.0;
}

// norms[s * 2 ld + j] = |row j| of the matrix in slot s (rows j < chi[s])
__global__ void row_norms_kernel(const double* W, size_t mat, int ld, const int* chi, double* norms) {
    const int s = blockIdx.y;
    const int n = chi[s];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* M = W + (size_t)s * mat;
    for (int j = blockIdx.x * 8 + warp; j < n; j += gridDim.x * 8) {
        double a = 0.0;
        for (int k = lane; k < n; k += 32) a = fma(M[(size_t)j * ld + k], M[(size_t)j * ld + k], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) norms[(size_t)s * 2 * ld + j] = sqrt(a);
    }
}

// C_i[j][k] /= sqrt(|x_j| |y_k|) (0 where either norm is 0): C = F_X F_Y^T
__global__ void scale_kernel(double* C, size_t mat, int ld, const int* chi, const double* norms) {
    const int i = blockIdx.y;
    const int n = chi[2 * i];
    const double* nx = norms + (size_t)(2 * i) * 2 * ld;
    const double* ny = norms + (size_t)(2 * i + 1) * 2 * ld;
    double* M = C + (size_t)(2 * i) * mat;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
        const int j = e / n, k = e % n;
        const double d = nx[j] * ny[k];
        M[(size_t)j * ld + k] = d > 0.0 ? M[(size_t)j * ld + k] / sqrt(d) : 0.0;
    }
}

// out[b0 + i] = OSEE from the row norms s_k of C_i after its Jacobi SVD
__global__ void osee_kernel(const double* C, size_t mat, int ld, const int* chi, int b0, double* out) {
    const int i = blockIdx.x;
    const int n = chi[2 * i];
    const double* M = C + (size_t)(2 * i) * mat;
    __shared__ double s2[4 * kMaxChi];
    __shared__ double red[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < n; j += nw) {
        double a = 0.0;
        for (int k = lane; k < n; k += 32) a = fma(M[(size_t)j * ld + k], M[(size_t)j * ld + k], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s2[j] = a;
    }
    __syncthreads();
    double t = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) t += s2[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[warp] = t;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < nw; ++w) tot += red[w];
    __syncthreads();
    double h = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double p = tot > 0.0 ? s2[j] / tot : 0.0;
        if (p > 0.0) h -= p * log(p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if (lane == 0) red[warp] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        for (int w = 0; w < nw; ++w) e += red[w];
        out[b0 + i] = e;
    }
}

// out[b0 + i] = -ln(X_i[0][0] / (2^{N/2} E0_b)^2), X_i = <<rho|rho>> after the full left sweep
__global__ void renyi2_kernel(const double* W, size_t mat, const double* envL, int n, int cap, int b0, int m,
                              double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int b = b0 + i;
    const double nrm2 = W[(size_t)(2 * i) * mat];
    const double tr = exp2(0.5 * n) * envL[((size_t)b * (n + 1) + n) * cap];
    out[b] = -log(nrm2 / (tr * tr));
}

struct GqPlan {
    std::vector<GemmDesc> g;
    struct Launch {
        size_t first;
        int count, max_m, max_n;
    };
    std::vector<Launch> launches;
    void begin() { launches.push_back(Launch{g.size(), 0, 1, 1}); }
    void add(const GemmDesc& d) {
        g.push_back(d);
        Launch& L = launches.back();
        ++L.count;
        L.max_m = std::max(L.max_m, d.M);
        L.max_n = std::max(L.max_n, d.N);
    }
};

// Left Gram sweep over sites 0..last of the chunk's instances: X (slot 2i) is
// chi x chi with chi = dims[last + 1] at the end.  T (thetap slot 2i) holds X B.
void plan_left(mpdo_ctx* c, int b0, int m, int last, GqPlan& P) {
    const int N = c->N, cap = c->cap, ld = c->ld;
    const size_t mat = (size_t)ld * ld;
    const int f32 = sites_f32(c);
    for (int q = 0; q <= last; ++q) {
        P.begin();
        for (int i = 0; i < m; ++i) {
            const int b = b0 + i;
            const int l = c->h_dims[(size_t)b * (N + 1) + q], r = c->h_dims[(size_t)b * (N + 1) + q + 1];
            double* X = c->d_W + (size_t)(2 * i) * mat;
            double* T = c->d_thetap + (size_t)(2 * i) * mat;
            // T[l][(s, r)] = sum_l' X[l][l'] B[l'][s][r]
            P.add(GemmDesc{l, 3 * cap + r, l, X, ld, 0, site_v(c, b, q), 4 * cap, f32, 0, T, 4 * cap, 1.0, 0.0,
                           nullptr, 0, 0, 0, 0, 0});
        }
        P.begin();
        for (int i = 0; i < m; ++i) {
            const int b = b0 + i;
            const int l = c->h_dims[(size_t)b * (N + 1) + q], r = c->h_dims[(size_t)b * (N + 1) + q + 1];
            double* X = c->d_W + (size_t)(2 * i) * mat;
            double* T = c->d_thetap + (size_t)(2 * i) * mat;
            // X'[r][r'] = sum_{(l, s)} B[(l, s)][r] T[(l, s)][r']  (both (4 l) x r with row stride cap)
            P.add(GemmDesc{r, r, 4 * l, site_v(c, b, q), cap, f32, T, cap, 0, 0, X, ld, 1.0, 0.0, nullptr, 0, 0, 0, 1,
                           1});
        }
    }
}

// Right Gram sweep over sites N-1..first: Y (slot 2i + 1), U (thetap slot 2i + 1) holds B Y.
void plan_right(mpdo_ctx* c, int b0, int m, int first, GqPlan& P) {
    const int N = c->N, cap = c->cap, ld = c->ld;
    const size_t mat = (size_t)ld * ld;
    const int f32 = sites_f32(c);
    for (int q = N - 1; q >= first; --q) {
        P.begin();
        for (int i = 0; i < m; ++i) {
            const int b = b0 + i;
            const int l = c->h_dims[(size_t)b * (N + 1) + q], r = c->h_dims[(size_t)b * (N + 1) + q + 1];
            double* Y = c->d_W + (size_t)(2 * i + 1) * mat;
            double* U = c->d_thetap + (size_t)(2 * i + 1) * mat;
            // U[(l, s)][r'] = sum_r B[(l, s)][r] Y[r][r']
            P.add(GemmDesc{4 * l, r, r, site_v(c, b, q), cap, f32, Y, ld, 0, 0, U, cap, 1.0, 0.0, nullptr, 0, 0, 0, 0,
                           0});
        }
        for (int s = 0; s < 4; ++s) {
            P.begin();
            for (int i = 0; i < m; ++i) {
                const int b = b0 + i;
                const int l = c->h_dims[(size_t)b * (N + 1) + q], r = c->h_dims[(size_t)b * (N + 1) + q + 1];
                double* Y = c->d_W + (size_t)(2 * i + 1) * mat;
                double* U = c->d_thetap + (size_t)(2 * i + 1) * mat;
                const void* Bs = static_cast<const char*>(site_v(c, b, q)) + (size_t)s * cap * site_esize(c);
                // Y'[l][l'] (+)= sum_r U[(l, s)][r] B[(l', s)][r]
                P.add(GemmDesc{l, l, r, U + (size_t)s * cap, 4 * cap, 0, Bs, 4 * cap, f32, 1, Y, ld, 1.0,
                               s > 0 ? 1.0 : 0.0, s > 0 ? Y : nullptr, ld, 0, 0, 0, 0});
            }
        }
    }
}

int run_plan(mpdo_ctx* c, GqPlan& P) {
    if (P.g.empty()) return MPDO_OK;
    if (c->gq_cap < P.g.size()) {
        if (c->d_gq) cudaFree(c->d_gq);
        c->d_gq = nullptr;
        c->gq_cap = 0;
        CU(dalloc(&c->d_gq, P.g.size()));
        c->gq_cap = P.g.size();
    }
    CU(cudaMemcpyAsync(c->d_gq, P.g.data(), sizeof(GemmDesc) * P.g.size(), cudaMemcpyHostToDevice, c->st));
    for (const auto& L : P.launches)
        if (L.count > 0) CU(launch_gemm(c->d_gq + L.first, L.count, L.max_m, L.max_n, false, c->st));
    CU(cudaStreamSynchronize(c->st));   // the host descriptors are rebuilt by the next plan
    return MPDO_OK;
}

// FP64 Jacobi SVD (strict tolerance, every pair) of the chi x chi matrices in
// W + slot * mat for the listed slots (rows j < chi of length chi).
int run_svd(mpdo_ctx* c, double* W, const std::vector<int>& slots, const std::vector<int>& chis,
            const std::vector<int>& inst) {
    const int ld = c->ld;
    const size_t mat = (size_t)ld * ld;
    const int nops = (int)slots.size();
    for (int k = 0; k < nops; ++k) {
        OpDesc d{};
        const int s = slots[k], n = chis[k];
        d.b = inst[k];
        d.c = n;
        d.L = n;
        d.m = n;
        d.n = n;
        d.chi_max = n;
        d.W = W + (size_t)s * mat;
        d.W0 = d.W;
        d.snorm = c->d_snorm + (size_t)s * 2 * ld;
        d.status = c->d_status + inst[k];
        d.sweeps_out = c->d_sweeps + s;
        d.full_svd = 1;
        d.jb = jacobi_block_rows(n, n, 8);
        d.jb32 = 1;
        c->h_desc[k] = d;
    }
    CU(cudaMemcpyAsync(c->d_desc, c->h_desc, sizeof(OpDesc) * nops, cudaMemcpyHostToDevice, c->st));
    int total = 0;
    int rc = plan_jacobi(c, c->h_desc, nops, false, c->h_cta, total);
    if (rc) return rc;
    CU(cudaMemcpyAsync(c->d_cta, c->h_cta, sizeof(int) * (2 * total + nops), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemsetAsync(c->d_sync, 0, sizeof(unsigned) * jacobi_sync_words(nops), c->st));
    const unsigned long long timeout_ns = (unsigned long long)c->cfg.barrier_timeout_ms * 1000000ull;
    CU(launch_jacobi(c->d_desc, nops, c->d_cta, c->d_cta + total, c->d_cta + 2 * total, c->d_sync, total,
                     c->cfg.jacobi_max_sweeps, 0.0, timeout_ns, ld, false, c->st));
    CU(cudaStreamSynchronize(c->st));   // h_desc / h_cta are reused by the next call
    return MPDO_OK;
}

int global_prepare(mpdo_ctx* c, double* out) {
    if (!c || !out) return fail(MPDO_EINVAL, "NULL argument");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (c->slots < 2) return fail(MPDO_ECAPACITY, "needs at least two workspace slots");
    CU(cudaMemcpyAsync(c->h_dims.data(), c->d_dims, sizeof(int) * c->h_dims.size(), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return MPDO_OK;
}

int finish(mpdo_ctx* c, double* out, int out_on_device) {
    if (!out_on_device) {
        CU(cudaMemcpyAsync(out, c->d_out, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
    }
    return MPDO_OK;
}

}  // namespace

}  // namespace mpdo

extern "C" int mpdo_renyi2(mpdo_ctx* c, double* out, int out_on_device) {
    int rc = global_prepare(c, out);
    if (rc) return rc;
    const int N = c->N, B = c->B;
    const size_t mat = (size_t)c->ld * c->ld;
    double* dst = out_on_device ? out : c->d_out;
    CU(launch_environments(c->d_sites, sites_f32(c), c->d_dims, N, B, c->cap, c->d_envL, c->d_envR, c->st));
    const int per = std::max(1, c->slots / 2);
    for (int b0 = 0; b0 < B; b0 += per) {
        const int m = std::min(per, B - b0);
        gram_unit_kernel<<<(2 * m + 127) / 128, 128, 0, c->st>>>(c->d_W, mat, m);
        CU(cudaGetLastError());
        GqPlan P;
        plan_left(c, b0, m, N - 1, P);
        rc = run_plan(c, P);
        if (rc) return rc;
        renyi2_kernel<<<(m + 127) / 128, 128, 0, c->st>>>(c->d_W, mat, c->d_envL, N, c->cap, b0, m, dst);
        CU(cudaGetLastError());
    }
    return finish(c, out, out_on_device);
}

extern "C" int mpdo_osee(mpdo_ctx* c, int bond, double* out, int out_on_device) {
    int rc = global_prepare(c, out);
    if (rc) return rc;
    const int N = c->N, B = c->B, ld = c->ld;
    if (bond < 0 || bond > N - 2) return fail(MPDO_EINVAL, "bond must be in [0, N-2]");
    const size_t mat = (size_t)ld * ld;
    double* dst = out_on_device ? out : c->d_out;
    const int per = std::max(1, c->slots / 2);
    int* d_chi = c->d_q;   // [2 m] chi of each slot (ints; N >= 2 m is not guaranteed, so chunk by it too)
    const int per_chi = std::max(1, N / 2);
    for (int b0 = 0; b0 < B; b0 += std::min(per, per_chi)) {
        const int m = std::min(std::min(per, per_chi), B - b0);
        gram_unit_kernel<<<(2 * m + 127) / 128, 128, 0, c->st>>>(c->d_W, mat, m);
        CU(cudaGetLastError());
        GqPlan P;
        plan_left(c, b0, m, bond, P);
        plan_right(c, b0, m, bond + 1, P);
        rc = run_plan(c, P);
        if (rc) return rc;
        std::vector<int> slots, chis, inst, chi2(2 * m);
        for (int i = 0; i < m; ++i) {
            const int b = b0 + i;
            const int chi = c->h_dims[(size_t)b * (N + 1) + bond + 1];
            for (int h = 0; h < 2; ++h) {
                slots.push_back(2 * i + h);
                chis.push_back(chi);
                inst.push_back(b);
                chi2[2 * i + h] = chi;
            }
        }
        CU(cudaMemcpyAsync(d_chi, chi2.data(), sizeof(int) * 2 * m, cudaMemcpyHostToDevice, c->st));
        rc = run_svd(c, c->d_W, slots, chis, inst);   // X and Y factored
        if (rc) return rc;
        int maxchi = 1;
        for (int v : chis) maxchi = std::max(maxchi, v);
        row_norms_kernel<<<dim3((maxchi + 7) / 8, 2 * m), 256, 0, c->st>>>(c->d_W, mat, ld, d_chi, c->d_snorm);
        CU(cudaGetLastError());
        // C_i = (rows of X) (rows of Y)^T into thetap slot 2i, then scaled to F_X F_Y^T
        GqPlan Pc;
        Pc.begin();
        for (int i = 0; i < m; ++i) {
            const int n = chi2[2 * i];
            Pc.add(GemmDesc{n, n, n, c->d_W + (size_t)(2 * i) * mat, ld, 0, c->d_W + (size_t)(2 * i + 1) * mat, ld, 0,
                            1, c->d_thetap + (size_t)(2 * i) * mat, ld, 1.0, 0.0, nullptr, 0, 0, 0, 0, 0});
        }
        rc = run_plan(c, Pc);
        if (rc) return rc;
        scale_kernel<<<dim3(64, m), 256, 0, c->st>>>(c->d_thetap, mat, ld, d_chi, c->d_snorm);
        CU(cudaGetLastError());
        std::vector<int> s1, c1, i1;
        for (int i = 0; i < m; ++i) {
            s1.push_back(2 * i);
            c1.push_back(chi2[2 * i]);
            i1.push_back(b0 + i);
        }
        rc = run_svd(c, c->d_thetap, s1, c1, i1);
        if (rc) return rc;
        osee_kernel<<<m, 512, 0, c->st>>>(c->d_thetap, mat, ld, d_chi, b0, dst);
        CU(cudaGetLastError());
    }
    return finish(c, out, out_on_device);
}
