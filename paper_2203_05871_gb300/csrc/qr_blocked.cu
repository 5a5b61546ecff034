// Blocked Householder QR with panel pivoting: the QR preconditioner of the
// mixed path's Jacobi SVD (a7), with its trailing updates on the tensor cores.
//
// Same factorisation as qr.cu (theta~ P = Q R, only the rows of R P^T are
// kept, graded rows for the Jacobi passes), organised in panels of nb
// columns (16, or 8 when rows are longer than 1024):
//   1. window pivoting: the nb remaining columns of largest norm below row k0
//      form the panel, in order of decreasing norm (Quintana-Orti, Sun &
//      Bischof's windowed pivoting; exact QRCP pivots column by column);
//   2. the panel (m' = m - k0 rows) is factored in one CTA's shared memory by
//      Householder reflections, y <- y - beta v (v . y), with column pivoting
//      inside the panel on downdated norms; the reflectors go out as rows of V
//      (nb x m') with their beta, and the compact-WY factor T (upper
//      triangular, H_1 ... H_nb = I - V^T T V in this row convention) is
//      built by the forward recurrence T[0:j, j] = -beta_j T[0:j, 0:j] (V v_j);
//   3. the trailing columns A_t (m' x n') are updated with the block
//      reflector: A_t <- A_t - V^T (T^T (V A_t)), as two tensor-core products
//      with FP64-class accuracy (oz_gemm.cu): Wt = A_t^T V^T (n' x nb), then
//      A_t^T <- A_t^T - (Wt T) V, where the rows of A_t^T are the trailing
//      columns gathered through the permutation (columns never move in memory);
//   4. the trailing columns' norms below row k0 + nb are recomputed exactly.
// The products' errors are relative to each trailing column's norm (its row of
// A_t^T is scaled on its own), the normwise accuracy of an FP64 Householder QR.
// Column-major input in d.Acm (column k at Acm + k * ld); output the r rows of
// R P^T (r = min(m, n)) row-major in d.W0.  Scratch per op: d.snorm holds the
// squared column norms and, from d.snorm + ld, the permutation (logical column
// -> physical column); d.W holds V, T, Wt and Wt T (dead until the Jacobi
// passes); the op's slice buffers carry the products.
#include <mpdo.h>

#include <algorithm>

#include "internal.h"

namespace mpdo {

namespace {

constexpr int kThreads = 512;
constexpr int kMaxNb = 16;
constexpr int kPanelBytes = 128 * 1024;   // shared memory of the panel (m' x nb doubles)

struct Scratch {
    double* cn;    // squared norms below the current row, by physical column
    int* perm;     // logical -> physical column
    double* V;     // nb rows of stride ld: reflector j = V[j * ld + i], i < m'
    double* T;     // nb x nb, row-major
    double* Wt;    // n' x kMaxNb, row-major
    double* W2t;   // n' x kMaxNb, row-major
};

__device__ __forceinline__ Scratch scratch(const OpDesc& d, int ld) {
    Scratch s;
    s.cn = d.snorm;
    s.perm = reinterpret_cast<int*>(d.snorm + ld);
    s.V = d.W;
    s.T = d.W + (size_t)kMaxNb * ld;
    s.Wt = s.T + kMaxNb * kMaxNb;
    s.W2t = s.Wt + (size_t)kMaxNb * ld;
    return s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// identity permutation and squared column norms of the whole matrix
__global__ void __launch_bounds__(256) qrb_start_kernel(const OpDesc* descs, int ld) {
    const OpDesc& d = descs[blockIdx.x];
    const Scratch s = scratch(d, ld);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = threadIdx.x; k < d.n; k += blockDim.x) s.perm[k] = k;
    for (int k = warp; k < d.n; k += blockDim.x >> 5) {
        const double* y = d.Acm + (size_t)k * ld;
        double a = 0.0;
        for (int i = lane; i < d.m; i += 32) a = fma(y[i], y[i], a);
        a = warp_sum(a);
        if (lane == 0) s.cn[k] = a;
    }
}

constexpr int kSums = 2 * kMaxNb + 1;   // per column: x . y_q (q > j), |x|^2, v_t . v_j (t < j)

// Reduce kSums per-thread partial sums over the block in one pass: after the
// call out[0..kSums) hold the block sums (every thread may read them).
__device__ __forceinline__ void block_sums(double* v, double (*red)[kSums], double* out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < kSums; ++q) {
        const double t = warp_sum(v[q]);
        if (lane == 0) red[warp][q] = t;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) t += red[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// panel k0 of every op: window selection, factorisation with in-panel pivoting,
// reflectors V and beta, the compact-WY T, and the panel's columns of R.  Every
// column's reductions (its norm, its inner products with the later panel
// columns, their norm updates) share one block-wide reduction.
__global__ void __launch_bounds__(kThreads, 1) qrb_panel_kernel(const OpDesc* descs, int k0, int nb, int ld) {
    extern __shared__ double P[];   // panel, column-major: P[j * mp + i]; then the window's norms
    __shared__ double red[kThreads / 32][kSums];
    __shared__ double s_sum[kSums];
    __shared__ double s_pn[kMaxNb], s_w[kMaxNb], s_z[kMaxNb];
    __shared__ double s_best[kThreads / 32];
    __shared__ int s_bidx[kThreads / 32];
    __shared__ int s_piv, s_redo;
    const OpDesc& d = descs[blockIdx.x];
    const int m = d.m, n = d.n, r = min(m, n);
    if (k0 >= r) return;
    const int jb = min(nb, r - k0), mp = m - k0, nw = n - k0;
    const Scratch s = scratch(d, ld);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double* wn = P + (size_t)nb * ld;          // norms of logical columns k0 .. n-1 (window)
    int* wp = reinterpret_cast<int*>(wn + ld);  // their physical columns

    // 1. window: the jb largest norms among logical columns [k0, n), in order
    for (int k = tid; k < nw; k += kThreads) {
        wp[k] = s.perm[k0 + k];
        wn[k] = s.cn[wp[k]];
    }
    __syncthreads();
    for (int t = 0; t < jb; ++t) {
        double best = -1.0;
        int bidx = t;
        for (int k = t + tid; k < nw; k += kThreads)
            if (wn[k] > best) {
                best = wn[k];
                bidx = k;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ob > best || (ob == best && oi < bidx)) {
                best = ob;
                bidx = oi;
            }
        }
        if (lane == 0) {
            s_best[warp] = best;
            s_bidx[warp] = bidx;
        }
        __syncthreads();
        if (tid == 0) {
            double b = s_best[0];
            int bi = s_bidx[0];
            for (int w = 1; w < kThreads / 32; ++w)
                if (s_best[w] > b || (s_best[w] == b && s_bidx[w] < bi)) {
                    b = s_best[w];
                    bi = s_bidx[w];
                }
            const double tn = wn[t];
            wn[t] = wn[bi];
            wn[bi] = tn;
            const int tp = wp[t];
            wp[t] = wp[bi];
            wp[bi] = tp;
        }
        __syncthreads();
    }
    for (int k = tid; k < nw; k += kThreads) s.perm[k0 + k] = wp[k];
    // 2. load the panel and its norms
    for (int e = tid; e < jb * mp; e += kThreads) {
        const int j = e / mp, i = e % mp;
        P[e] = d.Acm[(size_t)wp[j] * ld + k0 + i];
    }
    if (tid < jb) s_pn[tid] = wn[tid];
    __syncthreads();
    // 3. Householder reflections with pivoting inside the panel
    for (int j = 0; j < jb; ++j) {
        if (tid == 0) {
            int c = j;
            for (int q = j + 1; q < jb; ++q)
                if (s_pn[q] > s_pn[c]) c = q;
            s_piv = c;
            if (c != j) {
                const double t = s_pn[c];
                s_pn[c] = s_pn[j];
                s_pn[j] = t;
                const int p = s.perm[k0 + c];
                s.perm[k0 + c] = s.perm[k0 + j];
                s.perm[k0 + j] = p;
            }
        }
        __syncthreads();
        const int c = s_piv;
        if (c != j)
            for (int i = tid; i < mp; i += kThreads) {
                const double t = P[c * mp + i];
                P[c * mp + i] = P[j * mp + i];
                P[j * mp + i] = t;
            }
        __syncthreads();
        double* x = P + j * mp;
        // one reduction: x.y_q below row j (slot q > j), |x below row j|^2 (slot
        // kMaxNb) and, for T, x.v_t below row j (slot kMaxNb + 1 + t, t < j; the
        // earlier reflectors are read back from V); v_t . v_j then follows from
        // v_j = (v0 at row j, x below)
        double acc[kSums];
#pragma unroll
        for (int q = 0; q < kSums; ++q) acc[q] = 0.0;
        for (int i = j + 1 + tid; i < mp; i += kThreads) {
            const double xi = x[i];
            acc[kMaxNb] = fma(xi, xi, acc[kMaxNb]);
#pragma unroll
            for (int q = 0; q < kMaxNb; ++q) {
                if (q > j && q < jb) acc[q] = fma(xi, P[q * mp + i], acc[q]);
                if (q < j) acc[kMaxNb + 1 + q] = fma(xi, s.V[(size_t)q * ld + i], acc[kMaxNb + 1 + q]);
            }
        }
        block_sums(acc, red, s_sum);
        const double ss = s_sum[kMaxNb];
        const double x0 = x[j];
        const double nrm = sqrt(fma(x0, x0, ss));
        const double alpha = x0 > 0.0 ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double vtv = 2.0 * alpha * (alpha - x0);
        const double beta = (ss == 0.0 || !(vtv > 0.0)) ? 0.0 : 2.0 / vtv;
        // reflector j as row j of V (zeros above its pivot row)
        double* vr = s.V + (size_t)j * ld;
        for (int i = tid; i < mp; i += kThreads) vr[i] = i < j ? 0.0 : (i == j ? v0 : x[i]);
        if (tid > j && tid < jb) s_w[tid] = fma(v0, P[tid * mp + j], s_sum[tid]);   // w_q = v . y_q
        // T column j: z_t = v_t . v_j = v_t[j] v0 + (x . v_t below row j), then
        // T[t][j] = -beta_j sum_{t <= l < j} T[t][l] z_l, T[j][j] = beta_j
        if (tid < j) s_z[tid] = fma(s.V[(size_t)tid * ld + j], v0, s_sum[kMaxNb + 1 + tid]);
        __syncthreads();
        if (tid < j) {
            double accT = 0.0;
            for (int l = tid; l < j; ++l) accT = fma(s.T[tid * kMaxNb + l], s_z[l], accT);
            s.T[tid * kMaxNb + j] = -beta * accT;
        }
        if (tid == j) s.T[j * kMaxNb + j] = beta;
        if (tid > j && tid < kMaxNb) s.T[tid * kMaxNb + j] = 0.0;
        if (beta != 0.0)
            for (int i = j + tid; i < mp; i += kThreads) {
                const double vi = i == j ? v0 : x[i];
#pragma unroll
                for (int q = 0; q < kMaxNb; ++q)
                    if (q > j && q < jb) P[q * mp + i] = fma(-beta * s_w[q], vi, P[q * mp + i]);
            }
        __syncthreads();
        // column j of R; downdate the norms of the later panel columns
        if (tid == 0) x[j] = (ss == 0.0) ? x0 : alpha;
        for (int i = j + 1 + tid; i < mp; i += kThreads) x[i] = 0.0;
        if (tid == 0) s_redo = 0;
        __syncthreads();
        if (tid > j && tid < jb) {
            const double y = P[tid * mp + j];
            const double nv = s_pn[tid] - y * y;
            if (nv > 0.05 * s_pn[tid])
                s_pn[tid] = nv;
            else
                s_redo = 1;   // heavy cancellation: recomputed below row j
        }
        __syncthreads();
        if (s_redo) {
#pragma unroll
            for (int q = 0; q < kSums; ++q) acc[q] = 0.0;
            for (int i = j + 1 + tid; i < mp; i += kThreads)
#pragma unroll
                for (int q = 0; q < kMaxNb; ++q)
                    if (q > j && q < jb) acc[q] = fma(P[q * mp + i], P[q * mp + i], acc[q]);
            block_sums(acc, red, s_sum);
            if (tid > j && tid < jb) {
                const double y = P[tid * mp + j];
                const double nv = s_pn[tid] - y * y;
                if (!(nv > 0.05 * s_pn[tid])) s_pn[tid] = s_sum[tid];
            }
            __syncthreads();
        }
    }
    // 4. the panel's columns of R back in place
    for (int e = tid; e < jb * mp; e += kThreads) {
        const int j = e / mp, i = e % mp;
        d.Acm[(size_t)s.perm[k0 + j] * ld + k0 + i] = P[e];
    }
}

// The two products of the trailing update of panel k0, built per op:
// which = 0: Wt = A_t^T V^T (n' x jb); which = 1: A_t^T <- A_t^T - W2t V.
__global__ void qrb_prep_kernel(const OpDesc* descs, int nops, int k0, int nb, int which, OzProblem* out, int ld,
                                int bf16) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nops) return;
    const OpDesc& d = descs[o];
    const Scratch s = scratch(d, ld);
    const int m = d.m, n = d.n, r = min(m, n);
    const int jb = k0 < r ? min(nb, r - k0) : 0;
    const int mp = m - k0, np = k0 < r ? n - k0 - jb : 0;
    OzProblem P{};
    const OzOperand trail{d.Acm + k0, 0, ld, 1, 0, 1, 1, s.perm + k0 + jb};   // row q: trailing column q
    if (which == 0) {
        P.M = np;
        P.N = jb;
        P.K = mp;
        P.A = trail;
        P.B = OzOperand{s.V, 0, ld, 1, 0, 1, 1, nullptr};
        P.C = s.Wt;
        P.ldc = kMaxNb;
        P.alpha = 1.0;
    } else {
        P.M = np;
        P.N = mp;
        P.K = jb;
        P.A = OzOperand{s.W2t, 0, kMaxNb, 1, 0, 1, 1, nullptr};
        P.B = OzOperand{s.V, 0, 1, ld, 0, 1, 1, nullptr};   // (i, t) = V[t][i]
        P.C = d.Acm + k0;
        P.ldc = ld;
        P.c_gather = s.perm + k0 + jb;
        P.alpha = -1.0;
        P.beta = 1.0;
        P.D = d.Acm + k0;
        P.ldd = ld;
    }
    if (P.M <= 0 || P.N <= 0 || P.K <= 0) P.M = P.N = P.K = 0;
    P.as = d.oz_as;
    P.bs = d.oz_bs;
    P.ea = d.oz_ea;
    P.eb = d.oz_eb;
    P.status = d.status;
    oz_set_tiles(P, bf16 != 0);
    out[o] = P;
}

// W2t = Wt T (T upper triangular): W2t[q][j] = sum_{t <= j} Wt[q][t] T[t][j]
__global__ void qrb_wt_kernel(const OpDesc* descs, int k0, int nb, int ld) {
    const OpDesc& d = descs[blockIdx.y];
    const int m = d.m, n = d.n, r = min(m, n);
    if (k0 >= r) return;
    const int jb = min(nb, r - k0), np = n - k0 - jb;
    const Scratch s = scratch(d, ld);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= np * jb) return;
    const int q = e / jb, j = e % jb;
    double acc = 0.0;
    for (int t = 0; t <= j; ++t) acc = fma(s.Wt[q * kMaxNb + t], s.T[t * kMaxNb + j], acc);
    s.W2t[q * kMaxNb + j] = acc;
}

// squared norms of the trailing columns below row k0 + jb
__global__ void __launch_bounds__(256) qrb_norms_kernel(const OpDesc* descs, int k0, int nb, int ld) {
    const OpDesc& d = descs[blockIdx.y];
    const int m = d.m, n = d.n, r = min(m, n);
    if (k0 >= r) return;
    const int jb = min(nb, r - k0), row0 = k0 + jb;
    const Scratch s = scratch(d, ld);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = row0 + blockIdx.x * 8 + warp; k < n; k += gridDim.x * 8) {
        const int pk = s.perm[k];
        const double* y = d.Acm + (size_t)pk * ld;
        double a = 0.0;
        for (int i = row0 + lane; i < m; i += 32) a = fma(y[i], y[i], a);
        a = warp_sum(a);
        if (lane == 0) s.cn[pk] = a;
    }
}

// rows of R P^T into W0: W0[i][perm[k]] = R[i][k] for k >= i, 0 below
__global__ void __launch_bounds__(256) qrb_finish_kernel(const OpDesc* descs, int ld) {
    const OpDesc& d = descs[blockIdx.y];
    const int m = d.m, n = d.n, r = min(m, n);
    const Scratch s = scratch(d, ld);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * 8 + warp; i < r; i += gridDim.x * 8) {
        double* out = d.W0 + (size_t)i * ld;
        for (int k = lane; k < n; k += 32) {
            const int pk = s.perm[k];
            out[pk] = k >= i ? d.Acm[(size_t)pk * ld + i] : 0.0;
        }
    }
}

}  // namespace

int qrb_panel_width(int chi_cap) {
    const int ld = 4 * chi_cap;
    int nb = kPanelBytes / (8 * ld);
    return std::max(4, std::min(kMaxNb, nb));
}

// dynamic shared memory of the panel kernel: the panel (nb x ld doubles) and
// the window's norms and physical columns (ld doubles + ld ints)
static size_t panel_smem(int chi_cap) {
    const int ld = 4 * chi_cap;
    return ((size_t)qrb_panel_width(chi_cap) * ld + ld) * sizeof(double) + (size_t)ld * sizeof(int);
}

cudaError_t qrb_prepare() {
    return cudaFuncSetAttribute(qrb_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)panel_smem(kMaxChi));
}

int qrb_kernels(int chi_cap, int r_max) {
    const int ld = 4 * chi_cap, nb = qrb_panel_width(chi_cap);
    if (r_max <= 0 || r_max > ld) r_max = ld;
    // start and finish, and per panel: the panel, two operand set-ups, two
    // products (slicing + slice products each), W^T and the norms
    return 2 + ((r_max + nb - 1) / nb) * 9;
}

cudaError_t launch_qr_blocked(const OpDesc* d_desc, int nops, int chi_cap, OzProblem* probs, bool bf16,
                              unsigned long long timeout_ns, cudaStream_t st, int r_max) {
    if (nops <= 0) return cudaSuccess;
    const int ld = 4 * chi_cap, nb = qrb_panel_width(chi_cap);
    if (r_max <= 0 || r_max > ld) r_max = ld;
    qrb_start_kernel<<<nops, 256, 0, st>>>(d_desc, ld);
    cudaError_t e = cudaGetLastError();
    const size_t smem = panel_smem(chi_cap);
    for (int k0 = 0; k0 < r_max && e == cudaSuccess; k0 += nb) {
        qrb_panel_kernel<<<nops, kThreads, smem, st>>>(d_desc, k0, nb, ld);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        qrb_prep_kernel<<<(nops + 127) / 128, 128, 0, st>>>(d_desc, nops, k0, nb, 0, probs, ld, bf16 ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = launch_oz_gemm(probs, nops, ld, nb, ld, bf16, timeout_ns, st)) != cudaSuccess) break;
        qrb_wt_kernel<<<dim3((ld * kMaxNb + 255) / 256, nops), 256, 0, st>>>(d_desc, k0, nb, ld);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        qrb_prep_kernel<<<(nops + 127) / 128, 128, 0, st>>>(d_desc, nops, k0, nb, 1, probs, ld, bf16 ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = launch_oz_gemm(probs, nops, ld, ld, ld, bf16, timeout_ns, st)) != cudaSuccess) break;
        qrb_norms_kernel<<<dim3((ld + 63) / 64, nops), 256, 0, st>>>(d_desc, k0, nb, ld);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    qrb_finish_kernel<<<dim3((ld + 63) / 64, nops), 256, 0, st>>>(d_desc, ld);
    return cudaGetLastError();
}

}  // namespace mpdo
