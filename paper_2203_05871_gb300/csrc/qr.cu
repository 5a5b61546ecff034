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
// Input: theta~ (m x n) column-major in d.Acm (column k at Acm + k*ld).
// For j = 0 .. r-1 (r = min(m, n)): x = column j below the diagonal,
// alpha = -sign(x_0) |x|, v = x - alpha e_0, and every later column is
// reflected, y <- y - 2 v (v.y) / (v.v), with v.v = 2 alpha (alpha - x_0).
// The CTAs of an op share the columns of each step and meet in a bounded
// barrier after it (cooperative launch; a wait that gives up records
// MPDO_ST_TIMEOUT).  Output: the r rows of R, row-major in d.W0
// (R[i][k] = 0 for k < i).  FP64 throughout.
#include <mpdo.h>

#include "coop.cuh"
#include "internal.h"

namespace mpdo {

namespace {

constexpr int QW = 8;   // warps per CTA
constexpr int QT = QW * 32;

__global__ void __launch_bounds__(QT, 1) qr_kernel(const OpDesc* descs, const int* cta_op, const int* cta_rank,
                                                   const int* group, unsigned* sync, unsigned long long timeout_ns,
                                                   int ld) {
    const int op = cta_op[blockIdx.x];
    const int g = cta_rank[blockIdx.x];
    const int G = group[op];
    const OpDesc& d = descs[op];
    unsigned* sw = sync + (size_t)op * kSyncWords;
    const int m = d.m, n = d.n, r = m < n ? m : n;
    double* A = d.Acm;
    double* rdiag = d.snorm;   // R[j][j]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = g * QW + warp, NW = G * QW;
    unsigned gen = 0;
    __shared__ double s_v0, s_beta;
    for (int j = 0; j < r; ++j) {
        const double* col = A + (size_t)j * ld;
        if (warp == 0) {
            double ss = 0.0;
            for (int i = j + 1 + lane; i < m; i += 32) ss = fma(col[i], col[i], ss);
            ss = warp_sum(ss);
            if (lane == 0) {
                const double x0 = col[j];
                const double nrm = sqrt(fma(x0, x0, ss));
                const double alpha = x0 > 0.0 ? -nrm : nrm;
                const double v0 = x0 - alpha;
                const double vtv = 2.0 * alpha * (alpha - x0);
                s_v0 = v0;
                s_beta = (vtv > 0.0) ? 2.0 / vtv : 0.0;
                if (g == 0) rdiag[j] = (ss == 0.0) ? x0 : alpha;
                if (ss == 0.0) s_beta = 0.0;   // already upper triangular here: no reflection
            }
        }
        __syncthreads();
        const double v0 = s_v0, beta = s_beta;
        if (beta != 0.0) {
            for (int k = j + 1 + gw; k < n; k += NW) {
                double* y = A + (size_t)k * ld;
                double w = 0.0;
                for (int i = j + 1 + lane; i < m; i += 32) w = fma(col[i], y[i], w);
                w = warp_sum(w);
                w = fma(v0, y[j], w);
                const double s = beta * w;
                if (lane == 0) y[j] = fma(-s, v0, y[j]);
                for (int i = j + 1 + lane; i < m; i += 32) y[i] = fma(-s, col[i], y[i]);
            }
        }
        if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
    }
    // rows of R
    for (int i = gw; i < r; i += NW) {
        double* out = d.W0 + (size_t)i * ld;
        for (int k = lane; k < n; k += 32) out[k] = k > i ? A[(size_t)k * ld + i] : (k == i ? rdiag[i] : 0.0);
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
