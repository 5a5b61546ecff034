// Truncation of one bond after the Jacobi SVD (App. B).
//
// s_j = |w_j| (row norms after Jacobi), sorted descending with ties kept in
// row order.  k_cut = smallest k >= 1 whose discarded weight
// sum_{i>=k} s_i^2 is <= cutoff * sum_i s_i^2 (the tail is summed from the
// smallest value up); k = min(chi_max, k_cut).  Writes lambda_p = s[:k],
// Yk[j] = v_j^T (rows of W normalised, or rows of Z), the new site p+1
// B'[j][s2][r] = Yk[j][s2*cr + r] and the new bond dimension.  A forced rank
// (replay of a recorded run) replaces k_cut, still capped by chi_max and c.
// When the adjoint records a tape, all c sorted singular values and
// normalised rows are written as well.
#include <mpdo.h>

#include "internal.h"

namespace mpdo {

namespace {

constexpr int TT = 1024;
constexpr int kMaxRows = 4 * kMaxChi;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(TT) truncate_kernel(const OpDesc* descs, int chi_cap) {
    const OpDesc& d = descs[blockIdx.x];
    const int c = d.c, L = d.L, ld = 4 * chi_cap;
    __shared__ double s[kMaxRows];
    __shared__ int perm[kMaxRows];
    __shared__ int s_k, s_bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int j = warp; j < c; j += TT / 32) {
        const double* w = d.W + (size_t)j * ld;
        double a = 0.0;
        for (int i = lane; i < L; i += 32) {
            const double x = w[i];
            a = fma(x, x, a);
        }
        a = warp_sum(a);
        if (lane == 0) {
            const double v = sqrt(a);
            if (!isfinite(v)) s_bad = 1;
            s[j] = v;
        }
    }
    __syncthreads();
    const int bad = s_bad;
    for (int j = threadIdx.x; j < c; j += TT) {
        if (bad) {
            perm[j] = j;
            continue;
        }
        const double sj = s[j];
        int r = 0;
        for (int i = 0; i < c; ++i) {
            const double si = s[i];
            r += (si > sj) || (si == sj && i < j);
        }
        perm[r] = j;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int k = 1;
        double disc = 0.0;
        if (!bad) {
            // tail[k] = sum_{i>=k} s_perm(i)^2, accumulated from the smallest
            double tail = 0.0;
            double total = 0.0;
            for (int i = c - 1; i >= 0; --i) {
                const double v = s[perm[i]];
                total += v * v;
            }
            // find the smallest k with tail(k) <= cutoff*total by walking up from the end
            // (tail(k) is non-increasing in k, so scan k = c, c-1, ... while it holds)
            const double thr = d.cutoff * total;
            int kcut = c;
            tail = 0.0;
            for (int kk = c; kk >= 1; --kk) {
                // tail currently = sum_{i>=kk} w_i
                if (tail <= thr)
                    kcut = kk;
                else
                    break;
                const double v = s[perm[kk - 1]];
                tail += v * v;
            }
            k = kcut;
            if (k > d.chi_max) k = d.chi_max;
            if (d.forced_k > 0) k = d.forced_k < d.chi_max ? d.forced_k : d.chi_max;
            if (k > c) k = c;
            if (k < 1) k = 1;
            double dsum = 0.0;
            for (int i = c - 1; i >= k; --i) {
                const double v = s[perm[i]];
                dsum += v * v;
            }
            disc = total > 0.0 ? dsum / total : 0.0;
        } else {
            atomicOr(d.status, (int)MPDO_ST_NONFINITE);
        }
        s_k = k;
        *d.k_out = k;
        if (d.rank_log) *d.rank_log = k;
        atomicMax((unsigned long long*)d.max_disc, (unsigned long long)__double_as_longlong(disc));
    }
    __syncthreads();
    const int k = s_k;
    for (int j = threadIdx.x; j < k; j += TT) d.lam_out[j] = bad ? 0.0 : s[perm[j]];
    if (d.tape_V) {
        // every sorted right singular vector (zero rows stay zero) for the adjoint
        for (int j = threadIdx.x; j < c; j += TT) d.tape_s[j] = bad ? 0.0 : s[perm[j]];
        for (int j = warp; j < c; j += TT / 32) {
            const int src = perm[j];
            const double sv = s[src];
            const double inv = (sv > 0.0 && !bad) ? 1.0 / sv : 0.0;
            const double* wr = d.W + (size_t)src * ld;
            double* v = d.tape_V + (size_t)j * d.n;
            for (int i = lane; i < d.n; i += 32) v[i] = wr[i] * inv;
        }
    }
    const int n = d.n, cr = d.cr;
    for (int j = warp; j < k; j += TT / 32) {
        const int src = perm[j];
        double* y = d.Yk + (size_t)j * ld;
        const size_t bnew = (size_t)j * 4 * chi_cap;   // row j of the new site p+1
        if (d.transposed) {
            const double* zr = d.Z + (size_t)src * ld;
            for (int i = lane; i < n; i += 32) {
                const double v = zr[i];
                y[i] = v;
                site_st(d.B, bnew + (i / cr) * chi_cap + (i % cr), v, d.site_f32);
            }
        } else {
            const double* wr = d.W + (size_t)src * ld;
            const double sv = s[src];
            const double inv = (sv > 0.0 && !bad) ? 1.0 / sv : 0.0;
            for (int i = lane; i < n; i += 32) {
                const double v = wr[i] * inv;
                y[i] = v;
                site_st(d.B, bnew + (i / cr) * chi_cap + (i % cr), v, d.site_f32);
            }
        }
    }
}

}  // namespace

cudaError_t launch_truncate(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    truncate_kernel<<<nops, TT, 0, st>>>(d_desc, chi_cap);
    return cudaGetLastError();
}

}  // namespace mpdo
