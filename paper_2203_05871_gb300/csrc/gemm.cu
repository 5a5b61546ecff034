// Batched small dense GEMMs of the mixed-precision SVD preconditioner.
//
//   C = alpha * op(A) op(B) + beta * D  (- I if sub_identity)
// with A (M x K, or K x M when a_trans) and B (K x N, or N x K when b_trans)
// row-major, stored as
// float or double (converted on load), accumulated in TC (double or float),
// written as double.  One launch serves a list of problems of different
// sizes (grid.z = problem); CTAs outside a problem's tiles return at once.
// 64 x 64 tiles, k-step 16, 256 threads with a 4 x 4 register tile each.
// A symmetric product (sym: E = U U^T) computes the tiles on and above the
// diagonal only and writes each strictly upper tile to both triangles; entry
// (j, i) is then the same products summed in the same order as (i, j), so
// the result is bitwise that of the full product.
#include "internal.h"

namespace mpdo {

namespace {

constexpr int GT = 64;
constexpr int GK = 16;

template <typename TC>
__device__ __forceinline__ TC load_as(const void* p, int is_f32, size_t i) {
    return is_f32 ? (TC)(static_cast<const float*>(p)[i]) : (TC)(static_cast<const double*>(p)[i]);
}

template <typename TC>
__global__ void __launch_bounds__(256) gemm_kernel(const GemmDesc* descs) {
    const GemmDesc& g = descs[blockIdx.z];
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    if (i0 >= g.M || j0 >= g.N) return;
    if (g.sym && i0 > j0) return;   // the mirror of a tile above the diagonal
    __shared__ TC As[GK][GT + 1];
    __shared__ TC Bs[GK][GT + 1];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    TC acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = (TC)0;
    for (int k0 = 0; k0 < g.K; k0 += GK) {
        if (g.a_trans) {   // A stored K x M row-major
            for (int e = t; e < GT * GK; e += 256) {
                const int kk = e / GT, ii = e % GT;
                const int gi = i0 + ii, gk = k0 + kk;
                As[kk][ii] = (gi < g.M && gk < g.K) ? load_as<TC>(g.A, g.a_f32, (size_t)gk * g.lda + gi) : (TC)0;
            }
        } else {
            for (int e = t; e < GT * GK; e += 256) {
                const int ii = e / GK, kk = e % GK;
                const int gi = i0 + ii, gk = k0 + kk;
                As[kk][ii] = (gi < g.M && gk < g.K) ? load_as<TC>(g.A, g.a_f32, (size_t)gi * g.lda + gk) : (TC)0;
            }
        }
        if (g.b_trans) {
            for (int e = t; e < GT * GK; e += 256) {
                const int jj = e / GK, kk = e % GK;
                const int gj = j0 + jj, gk = k0 + kk;
                Bs[kk][jj] = (gj < g.N && gk < g.K) ? load_as<TC>(g.B, g.b_f32, (size_t)gj * g.ldb + gk) : (TC)0;
            }
        } else {
            for (int e = t; e < GT * GK; e += 256) {
                const int kk = e / GT, jj = e % GT;
                const int gj = j0 + jj, gk = k0 + kk;
                Bs[kk][jj] = (gj < g.N && gk < g.K) ? load_as<TC>(g.B, g.b_f32, (size_t)gk * g.ldb + gj) : (TC)0;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GK; ++kk) {
            TC a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty * 4 + u];
                b[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int gi = i0 + ty * 4 + u;
        if (gi >= g.M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gj = j0 + tx * 4 + v;
            if (gj >= g.N) continue;
            double r = g.alpha * (double)acc[u][v];
            if (g.D) r += g.beta * load_as<double>(g.D, g.d_f32, (size_t)gi * g.ldd + gj);
            if (g.sub_identity && gi == gj) r -= 1.0;
            g.C[(size_t)gi * g.ldc + gj] = r;
            if (g.sym && i0 < j0) g.C[(size_t)gj * g.ldc + gi] = r;
        }
    }
}

}  // namespace

cudaError_t launch_gemm(const GemmDesc* d_desc, int count, int max_m, int max_n, bool fp32_compute,
                        cudaStream_t st) {
    if (count <= 0 || max_m <= 0 || max_n <= 0) return cudaSuccess;
    dim3 grid((max_n + GT - 1) / GT, (max_m + GT - 1) / GT, count);
    if (fp32_compute)
        gemm_kernel<float><<<grid, 256, 0, st>>>(d_desc);
    else
        gemm_kernel<double><<<grid, 256, 0, st>>>(d_desc);
    return cudaGetLastError();
}

}  // namespace mpdo
