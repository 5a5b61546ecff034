// Householder QR of the weighted bond matrices, the preconditioner of the
// Jacobi SVD.
//
// theta~ = Q R with Q orthogonal, so theta~ and R have the same singular
// values and the same right singular vectors: the truncation needs only R.
// One-sided Jacobi on the rows of R converges in far fewer sweeps than on
// the rows of theta~ itself (R's rows are graded), which is the point of
// the QR step (Drmac & Veselic, "New fast and accurate Jacobi SVD
// algorithm", preconditioning by QR).  Q is never formed.
//
// Column pivoting (theta~ P = Q R, P a permutation): at step j the remaining
// column of largest norm below row j is moved to position j, which makes
// |R_jj| decrease and R graded row by row, the property that lets the
// Jacobi sweeps converge at the rate of the well-conditioned part.
// Input: theta~ (m x n) column-major in d.Acm (column k at Acm + k*ld).
// For j = 0 .. r-1 (r = min(m, n)): x = pivot column below the diagonal,
// alpha = -sign(x_0) |x|, v = x - alpha e_0, and every later column is
// reflected, y <- y - 2 v (v.y) / (v.v), with v.v = 2 alpha (alpha - x_0);
// column norms are downdated (recomputed after heavy cancellation).
// The CTAs of an op share the columns of each step and meet in a bounded
// barrier after it (cooperative launch; a wait that gives up records
// MPDO_ST_TIMEOUT); every CTA finds the same pivot from the same norms.
// Output: the r rows of R P^T (columns back in their original order),
// row-major in d.W0: theta~ and R P^T share their right singular vectors.
// FP64 throughout; shared data is read and written through L2 (.cg).
#include <mpdo.h>

#include "coop.cuh"
#include "internal.h"

namespace mpdo {

namespace {

constexpr int QW = kQrWarps;   // warps per CTA
constexpr int QT = QW * 32;
constexpr int kMaxRowsQR = 4 * kMaxChi;

__global__ void __launch_bounds__(QT, 1) qr_kernel(const OpDesc* descs, const int* cta_op, const int* cta_rank,
                                                   const int* group, unsigned* sync, unsigned long long timeout_ns,
                                                   int ld) {
    const int op = cta_op[blockIdx.x];
    if (op < 0) return;   // a CTA the plan left unused (graph step)
    const int g = cta_rank[blockIdx.x];
    const int G = group[op];
    const OpDesc& d = descs[op];
    unsigned* sw = sync + (size_t)op * kSyncWords;
    const int m = d.m, n = d.n, r = m < n ? m : n;
    double* A = d.Acm;
    double* rdiag = d.snorm;          // R[j][j]
    double* cn = d.snorm + ld;   // squared norms of the physical columns below the current row (slot has 2 ld)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = g * QW + warp, NW = G * QW;
    unsigned gen = 0;
    __shared__ int perm[kMaxRowsQR];   // logical column -> physical column (same in every CTA)
    __shared__ double s_v0, s_beta;
    __shared__ double s_best[QW];
    __shared__ int s_bidx[QW];
    for (int k = threadIdx.x; k < n; k += QT) perm[k] = k;
    for (int k = gw; k < n; k += NW) {
        const double* y = A + (size_t)k * ld;
        double ss = 0.0;
        for (int i = lane; i < m; i += 32) {
            const double t = __ldcg(y + i);
            ss = fma(t, t, ss);
        }
        ss = warp_sum(ss);
        if (lane == 0) __stcg(cn + k, ss);
    }
    if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
    for (int j = 0; j < r; ++j) {
        // pivot: the remaining column of largest norm (ties: smallest logical index)
        {
            double best = -1.0;
            int bidx = j;
            for (int k = j + threadIdx.x; k < n; k += QT) {
                const double v = __ldcg(cn + perm[k]);
                if (v > best) {
                    best = v;
                    bidx = k;
                }
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
            if (threadIdx.x == 0) {
                double b = s_best[0];
                int bi = s_bidx[0];
                for (int w = 1; w < QW; ++w)
                    if (s_best[w] > b || (s_best[w] == b && s_bidx[w] < bi)) {
                        b = s_best[w];
                        bi = s_bidx[w];
                    }
                const int t = perm[j];
                perm[j] = perm[bi];
                perm[bi] = t;
            }
            __syncthreads();
        }
        const double* col = A + (size_t)perm[j] * ld;
        if (warp == 0) {
            double ss = 0.0;
            for (int i = j + 1 + lane; i < m; i += 32) ss = fma(__ldcg(col + i), __ldcg(col + i), ss);
            ss = warp_sum(ss);
            if (lane == 0) {
                const double x0 = __ldcg(col + j);
                const double nrm = sqrt(fma(x0, x0, ss));
                const double alpha = x0 > 0.0 ? -nrm : nrm;
                s_v0 = x0 - alpha;
                const double vtv = 2.0 * alpha * (alpha - x0);
                s_beta = (ss == 0.0 || !(vtv > 0.0)) ? 0.0 : 2.0 / vtv;
                if (g == 0) rdiag[j] = (ss == 0.0) ? x0 : alpha;
            }
        }
        __syncthreads();
        const double v0 = s_v0, beta = s_beta;
        for (int k = j + 1 + gw; k < n; k += NW) {
            const int pk = perm[k];
            double* y = A + (size_t)pk * ld;
            if (beta != 0.0) {
                double w = 0.0;
                for (int i = j + 1 + lane; i < m; i += 32) w = fma(__ldcg(col + i), __ldcg(y + i), w);
                w = warp_sum(w);
                w = fma(v0, __ldcg(y + j), w);
                const double s = beta * w;
                for (int i = j + 1 + lane; i < m; i += 32) __stcg(y + i, fma(-s, __ldcg(col + i), __ldcg(y + i)));
                if (lane == 0) __stcg(y + j, fma(-s, v0, __ldcg(y + j)));
                __syncwarp();
            }
            // squared norm of the column below row j: downdate, or recompute when
            // more than 95% of it cancelled
            double nv = 0.0;
            int redo = 0;
            if (lane == 0) {
                const double old = __ldcg(cn + pk);
                const double yj = __ldcg(y + j);
                nv = old - yj * yj;
                redo = !(nv > 0.05 * old);
            }
            redo = __shfl_sync(0xffffffffu, redo, 0);
            if (redo) {
                double ss = 0.0;
                for (int i = j + 1 + lane; i < m; i += 32) {
                    const double t = __ldcg(y + i);
                    ss = fma(t, t, ss);
                }
                nv = warp_sum(ss);
            }
            if (lane == 0) __stcg(cn + pk, nv);
        }
        if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
    }
    // rows of R P^T (columns back in their physical order)
    for (int i = gw; i < r; i += NW) {
        double* out = d.W0 + (size_t)i * ld;
        for (int k = lane; k < n; k += 32) {
            const int c = perm[k];
            out[c] = k > i ? __ldcg(A + (size_t)c * ld + i) : (k == i ? rdiag[i] : 0.0);
        }
    }
    return;
timeout:
    if (threadIdx.x == 0) atomicOr(d.status, (int)MPDO_ST_TIMEOUT);
}

}  // namespace

int qr_threads() { return QT; }

cudaError_t qr_max_resident(int* blocks) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, qr_kernel, QT, 0)) != cudaSuccess) return e;
    *blocks = sms * per;
    return cudaSuccess;
}

cudaError_t launch_qr(const OpDesc* d_desc, const int* d_cta_op, const int* d_cta_rank, const int* d_group,
                      unsigned* d_sync, int grid, unsigned long long timeout_ns, int ld, cudaStream_t st) {
    if (grid <= 0) return cudaSuccess;
    void* args[] = {(void*)&d_desc, (void*)&d_cta_op, (void*)&d_cta_rank, (void*)&d_group, (void*)&d_sync,
                    (void*)&timeout_ns, (void*)&ld};
    return cudaLaunchCooperativeKernel((const void*)qr_kernel, dim3(grid), dim3(QT), args, 0, st);
}

}  // namespace mpdo
