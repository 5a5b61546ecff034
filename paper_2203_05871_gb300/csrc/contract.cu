// FP64 two-site contractions of one op (App. B update of |rho>> per bond):
//   merge + gate + weight:
//     Theta [l,s1,s2,r] = sum_m A[l,s1,m] B[m,s2,r]
//     Theta'[l,s1',s2',r] = sum_{s1,s2} G[s1's2', s1s2] Theta[l,s1,s2,r]
//     theta~ = lambda_{p-1}[l] * Theta'   (rows (l,s1'), cols (s2',r)), stored
//     column-major for the QR step
//   reconstruct:
//     B_p'[(l,s1), j] = sum_c Theta'[(l,s1), c] Yk[j, c]
// Site tensors are stored [chi_l][4][chi_cap] (row (l,s) of length chi_cap).
// Workspace matrices are row-major with ld = 4*chi_cap; Theta' columns are
// compact: c = s2*cr + r.
#include "internal.h"

namespace mpdo {

namespace {

constexpr int TL = 16;   // l per tile
constexpr int TR = 16;   // r per tile
constexpr int KT = 16;   // m per k-step

// One thread owns one (l, r) pair and its 16 (s1, s2) outputs, so the gate
// (a 16x16 matrix on (s1, s2)) is applied in registers.
__global__ void __launch_bounds__(256) merge_gate_kernel(const OpDesc* descs, int chi_cap) {
    const OpDesc& d = descs[blockIdx.z];
    const int l0 = blockIdx.y * TL, r0 = blockIdx.x * TR;
    if (l0 >= d.cl || r0 >= d.cr) return;
    const int ld = 4 * chi_cap;
    __shared__ double As[TL][4][KT + 1];
    __shared__ double Bs[KT][4][TR];
    __shared__ double Gs[256];
    const int t = threadIdx.x, tl = t >> 4, tr = t & 15;
    Gs[t] = d.G[t];
    double acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.0;
    for (int m0 = 0; m0 < d.cm; m0 += KT) {
        for (int e = t; e < TL * 4 * KT; e += 256) {
            const int l = e / (4 * KT), s = (e / KT) & 3, kk = e % KT;
            const int gl = l0 + l, gm = m0 + kk;
            As[l][s][kk] = (gl < d.cl && gm < d.cm) ? site_ld(d.A, ((size_t)gl * 4 + s) * chi_cap + gm, d.site_f32) : 0.0;
        }
        for (int e = t; e < KT * 4 * TR; e += 256) {
            const int kk = e / (4 * TR), s = (e / TR) & 3, r = e % TR;
            const int gm = m0 + kk, gr = r0 + r;
            Bs[kk][s][r] = (gm < d.cm && gr < d.cr) ? site_ld(d.B, ((size_t)gm * 4 + s) * chi_cap + gr, d.site_f32) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KT; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                a[s] = As[tl][s][kk];
                b[s] = Bs[kk][s][tr];
            }
#pragma unroll
            for (int s1 = 0; s1 < 4; ++s1)
#pragma unroll
                for (int s2 = 0; s2 < 4; ++s2) acc[s1 * 4 + s2] = fma(a[s1], b[s2], acc[s1 * 4 + s2]);
        }
        __syncthreads();
    }
    const int l = l0 + tl, r = r0 + tr;
    if (l >= d.cl || r >= d.cr) return;
    const double lam = d.lam_left ? d.lam_left[l] : 1.0;
    for (int o = 0; o < 16; ++o) {
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < 16; ++i) v = fma(Gs[o * 16 + i], acc[i], v);
        const int s1 = o >> 2, s2 = o & 3;
        const int row = l * 4 + s1, col = s2 * d.cr + r;
        d.thetap[(size_t)row * ld + col] = v;
        d.Acm[(size_t)col * ld + row] = lam * v;
    }
}

constexpr int RT = 64;   // reconstruct tile (rows and cols)
constexpr int RK = 16;

__global__ void __launch_bounds__(256) reconstruct_kernel(const OpDesc* descs, int chi_cap) {
    const OpDesc& d = descs[blockIdx.z];
    const int k = *d.k_out;
    const int i0 = blockIdx.y * RT, j0 = blockIdx.x * RT;
    if (i0 >= d.m || j0 >= k) return;
    const int ld = 4 * chi_cap;
    __shared__ double As[RK][RT + 1];
    __shared__ double Bs[RK][RT + 1];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    double acc[4][4] = {};
    for (int c0 = 0; c0 < d.n; c0 += RK) {
        for (int e = t; e < RT * RK; e += 256) {
            const int ii = e / RK, kk = e % RK;
            const int gi = i0 + ii, gc = c0 + kk;
            As[kk][ii] = (gi < d.m && gc < d.n) ? d.thetap[(size_t)gi * ld + gc] : 0.0;
            const int gj = j0 + ii;
            Bs[kk][ii] = (gj < k && gc < d.n) ? d.Yk[(size_t)gj * ld + gc] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < RK; ++kk) {
            double a[4], b[4];
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
        if (gi >= d.m) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gj = j0 + tx * 4 + v;
            if (gj < k) site_st(d.A, (size_t)gi * chi_cap + gj, acc[u][v], d.site_f32);
        }
    }
}

}  // namespace

cudaError_t launch_merge_gate(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    dim3 grid((chi_cap + TR - 1) / TR, (chi_cap + TL - 1) / TL, nops);
    merge_gate_kernel<<<grid, 256, 0, st>>>(d_desc, chi_cap);
    return cudaGetLastError();
}

cudaError_t launch_reconstruct(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    dim3 grid((chi_cap + RT - 1) / RT, (4 * chi_cap + RT - 1) / RT, nops);
    reconstruct_kernel<<<grid, 256, 0, st>>>(d_desc, chi_cap);
    return cudaGetLastError();
}

}  // namespace mpdo
