// Trace forcing and Pauli observables from the MPO (Sec. 2.3-2.4, App. A).
//
// With r_{a1..aN} = B_0[a1] ... B_{N-1}[aN] the coefficients of rho in the
// normalised Pauli basis, Tr(P_a/sqrt2) = sqrt2 delta_{a,I} per site gives
//   tr rho = 2^{N/2} E(I...I),   Tr(sigma^a_i rho) = 2^{N/2} E(..a at i..),
// E(string) = product over sites of the selected a-slices of the B's.  So
//   <sigma^a_i> = E(a at i)/E(I..I),  <sigma^a_i sigma^b_j> = E(a at i, b at j)/E(I..I).
// Left environments L_p = E-prefix over sites < p (row vectors), right
// environments R_p = suffix over sites >= p (column vectors), all with I.
#include <mpdo.h>

#include "internal.h"

namespace mpdo {

namespace {

constexpr int MT = 512;

// one site tensor, read as double whatever the storage (f64 or f32)
struct SiteRef {
    const void* p;
    int f32;
    __device__ double operator[](size_t i) const { return site_ld(p, i, f32); }
};

__device__ __forceinline__ SiteRef site_ptr(const void* sites, int f32, int b, int p, int n, int cap) {
    const size_t off = ((size_t)b * n + p) * (size_t)cap * 4 * cap;
    return SiteRef{f32 ? (const void*)(static_cast<const float*>(sites) + off)
                       : (const void*)(static_cast<const double*>(sites) + off),
                   f32};
}

// v_out[r] = sum_l v_in[l] S[l][a][r]   (row vector times one Pauli slice)
__device__ void vec_slice(SiteRef S, int a, int cl, int cr, int cap, const double* vin, double* vout) {
    for (int r = threadIdx.x; r < cr; r += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < cl; ++l) acc = fma(vin[l], S[((size_t)l * 4 + a) * cap + r], acc);
        vout[r] = acc;
    }
}

__global__ void __launch_bounds__(MT) trace_kernel(void* sites, int f32, const int* dims, int n, int cap, int force,
                                                   double* trace_out, int* status) {
    const int b = blockIdx.x;
    const int* dm = dims + (size_t)b * (n + 1);
    __shared__ double v0[kMaxChi], v1[kMaxChi];
    if (threadIdx.x == 0) v0[0] = 1.0;
    __syncthreads();
    double* vin = v0;
    double* vout = v1;
    for (int p = 0; p < n; ++p) {
        vec_slice(site_ptr(sites, f32, b, p, n, cap), 0, dm[p], dm[p + 1], cap, vin, vout);
        __syncthreads();
        double* t = vin;
        vin = vout;
        vout = t;
    }
    const double tr = exp2(0.5 * n) * vin[0];
    __shared__ double s_tr;
    if (threadIdx.x == 0) {
        s_tr = tr;
        trace_out[b] = tr;
        if (!isfinite(tr) || tr == 0.0) atomicOr(status + b, (int)MPDO_ST_NONFINITE);
    }
    __syncthreads();
    if (force && isfinite(s_tr) && s_tr != 0.0) {
        void* S = const_cast<void*>(site_ptr(sites, f32, b, 0, n, cap).p);
        const double inv = 1.0 / s_tr;
        const int cr = dm[1];
        for (int e = threadIdx.x; e < 4 * cr; e += blockDim.x) {
            const size_t i = (size_t)(e / cr) * cap + (e % cr);
            site_st(S, i, site_ld(S, i, f32) * inv, f32);
        }
    }
}

// One step t of both environments, spread over CTAs (a single CTA per
// environment would leave all but two SMs idle and run at one SM's FP64 rate):
//   blockIdx.y == 0: L_{t+1} = L_t B_t[I], EW columns of L_{t+1} per CTA;
//   blockIdx.y == 1: R_p = B_p[I] R_{p+1} with p = n - 1 - t, EW entries per CTA.
// Step 0 uses L_0 = R_n = (1) and also stores them for the readers.
constexpr int EW = 16;
__global__ void __launch_bounds__(256) env_step_kernel(const void* sites, int f32, const int* dims, int n, int cap,
                                                       int t, double* envL, double* envR) {
    const int b = blockIdx.z;
    const int* dm = dims + (size_t)b * (n + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (blockIdx.y == 0) {
        const int p = t, cl = dm[p], cr = dm[p + 1];
        const int r0 = blockIdx.x * EW;
        double* E = envL + (size_t)b * (n + 1) * cap;
        if (p == 0 && blockIdx.x == 0 && threadIdx.x == 0) E[0] = 1.0;
        if (r0 >= cr) return;
        const SiteRef S = site_ptr(sites, f32, b, p, n, cap);
        const double* vin = E + (size_t)p * cap;
        const int c = threadIdx.x % EW, g = threadIdx.x / EW;   // column, row group (16 groups)
        const int r = r0 + c;
        double acc = 0.0;
        if (r < cr)
            for (int l = g; l < cl; l += 256 / EW) acc = fma(p == 0 ? 1.0 : vin[l], S[((size_t)l * 4) * cap + r], acc);
        __shared__ double red[256];
        red[threadIdx.x] = acc;
        __syncthreads();
        if (g == 0 && r < cr) {
            double sum = 0.0;
            for (int k = 0; k < 256 / EW; ++k) sum += red[k * EW + c];
            E[(size_t)(p + 1) * cap + r] = sum;
        }
    } else {
        const int p = n - 1 - t, cl = dm[p], cr = dm[p + 1];
        const int l0 = blockIdx.x * EW;
        double* E = envR + (size_t)b * (n + 1) * cap;
        if (p == n - 1 && blockIdx.x == 0 && threadIdx.x == 0) E[(size_t)n * cap] = 1.0;
        if (l0 >= cl) return;
        const SiteRef S = site_ptr(sites, f32, b, p, n, cap);
        const double* rin = E + (size_t)(p + 1) * cap;
        const int lend = min(l0 + EW, cl);
        for (int l = l0 + warp; l < lend; l += 8) {
            double acc = 0.0;
            for (int r = lane; r < cr; r += 32) acc = fma(S[((size_t)l * 4) * cap + r], p == n - 1 ? 1.0 : rin[r], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) E[(size_t)p * cap + l] = acc;
        }
    }
}

__device__ double block_sum(double v) {
    __shared__ double red[MT / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;   // valid in thread 0
}

// out[b*nq + k] = E(comp at q_k) / E0
__global__ void __launch_bounds__(MT) one_kernel(const void* sites, int f32, const int* dims, int n, int cap,
                                                 const double* envL, const double* envR, const int* qs, int nq,
                                                 int comp, double* out) {
    const int k = blockIdx.x, b = blockIdx.y;
    const int q = qs[k];
    const int* dm = dims + (size_t)b * (n + 1);
    const double* Lq = envL + ((size_t)b * (n + 1) + q) * cap;
    const double* Rq = envR + ((size_t)b * (n + 1) + q + 1) * cap;
    const double E0 = envL[((size_t)b * (n + 1) + n) * cap];
    const SiteRef S = site_ptr(sites, f32, b, q, n, cap);
    const int cl = dm[q], cr = dm[q + 1];
    double part = 0.0;
    for (int r = threadIdx.x; r < cr; r += blockDim.x) {
        double acc = 0.0;
        for (int l = 0; l < cl; ++l) acc = fma(Lq[l], S[((size_t)l * 4 + comp) * cap + r], acc);
        part = fma(acc, Rq[r], part);
    }
    const double tot = block_sum(part);
    if (threadIdx.x == 0) out[(size_t)b * nq + k] = tot / E0;
}

// All-pairs two-point values as one stacked propagation over j (the rows
// w_i for every i < j advance together, so site j's slices are read once per
// j instead of once per (i, j)).  Step j, per instance b and per tile of TW
// columns r of bond j+1:
//   for i < j with need[i]:  x = w_i B_j[cb],  part[b][j][tile][i] = x . R_{j+1}
//                            (over the tile's columns),  w_i <- w_i B_j[I]
//   if need[j] (j < n-1):    w_j = L_j B_j[ca]   (the row starts here)
// w lives in win (read) and wout (written), [b][n][cap] each, swapped per
// step.  The tile's three slices are staged in shared memory ([l][TW] each);
// a warp takes one row i at a time, its lanes split l.  The sum over tiles
// (two_reduce_kernel) keeps the result independent of the launch shape.
constexpr int TW = 4;
__global__ void __launch_bounds__(256) two_stack_kernel(const void* sites, int f32, const int* dims, int n, int cap,
                                                        const double* envL, const double* envR, int ca, int cb,
                                                        const unsigned char* need, int j, const double* win,
                                                        double* wout, double* part, int ntiles) {
    const int b = blockIdx.y, tile = blockIdx.x;
    const int* dm = dims + (size_t)b * (n + 1);
    const int cl = dm[j], cr = dm[j + 1];
    const int r0 = tile * TW;
    if (r0 >= cr) return;
    extern __shared__ double sm[];
    double* sI = sm;                     // [cap][TW]: slice I of site j, the tile's columns
    double* sB = sm + (size_t)cap * TW;  // slice cb
    double* sA = sB + (size_t)cap * TW;  // slice ca
    const SiteRef S = site_ptr(sites, f32, b, j, n, cap);
    for (int e = threadIdx.x; e < cl * TW; e += blockDim.x) {
        const int l = e / TW, c = e % TW, r = r0 + c;
        const bool in = r < cr;
        const size_t base = (size_t)l * 4 * cap + r;
        sI[e] = in ? S[base] : 0.0;
        sB[e] = in ? S[base + (size_t)cb * cap] : 0.0;
        sA[e] = in ? S[base + (size_t)ca * cap] : 0.0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* Lj = envL + ((size_t)b * (n + 1) + j) * cap;
    const double* Rn = envR + ((size_t)b * (n + 1) + j + 1) * cap;
    const double* W = win + (size_t)b * n * cap;
    double* Wn = wout + (size_t)b * n * cap;
    for (int i = warp; i <= j; i += 8) {
        if (!need[i] || (i == j && j >= n - 1)) continue;
        const bool seed = i == j;
        const double* w = seed ? Lj : W + (size_t)i * cap;
        const double* s1 = seed ? sA : sI;
        double a[TW] = {}, v[TW] = {};
        for (int l = lane; l < cl; l += 32) {
            const double wl = w[l];
            const double2 p0 = *reinterpret_cast<const double2*>(s1 + l * TW);
            const double2 p1 = *reinterpret_cast<const double2*>(s1 + l * TW + 2);
            a[0] = fma(wl, p0.x, a[0]);
            a[1] = fma(wl, p0.y, a[1]);
            a[2] = fma(wl, p1.x, a[2]);
            a[3] = fma(wl, p1.y, a[3]);
            if (!seed) {
                const double2 q0 = *reinterpret_cast<const double2*>(sB + l * TW);
                const double2 q1 = *reinterpret_cast<const double2*>(sB + l * TW + 2);
                v[0] = fma(wl, q0.x, v[0]);
                v[1] = fma(wl, q0.y, v[1]);
                v[2] = fma(wl, q1.x, v[2]);
                v[3] = fma(wl, q1.y, v[3]);
            }
        }
#pragma unroll
        for (int c = 0; c < TW; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a[c] += __shfl_xor_sync(0xffffffffu, a[c], o);
                v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
            }
        if (lane == 0) {
            double dot = 0.0;
#pragma unroll
            for (int c = 0; c < TW; ++c)
                if (r0 + c < cr) {
                    Wn[(size_t)i * cap + r0 + c] = a[c];
                    dot = fma(v[c], Rn[r0 + c], dot);
                }
            if (!seed) part[(((size_t)b * n + j) * ntiles + tile) * n + i] = dot;
        }
    }
}

// full[b][i][j] = sum over the tiles of step j of part[b][j][tile][i], / E0
__global__ void two_reduce_kernel(const double* part, const int* dims, const double* envL,
                                  const unsigned char* need, int n, int cap, int B, int ntiles, double* full) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * n * n) return;
    const int b = (int)(t / ((long long)n * n)), i = (int)((t / n) % n), j = (int)(t % n);
    if (j <= i || !need[i]) return;
    const int cr = dims[(size_t)b * (n + 1) + j + 1];
    const int nt = (cr + TW - 1) / TW;
    double sum = 0.0;
    for (int k = 0; k < nt; ++k) sum += part[(((size_t)b * n + j) * ntiles + k) * n + i];
    full[((size_t)b * n + i) * n + j] = sum / envL[((size_t)b * (n + 1) + n) * cap];
}

// trip[t] = (i, j, k): out[b][k] = full[b][i][j] (minus one_a[b][i] one_b[b][j] if connected)
__global__ void gather_kernel(const double* full, const double* one_a, const double* one_b, const int* trip, int m,
                              int np, int n, int B, int connected, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * B) return;
    const int b = t / m, u = t % m;
    const int i = trip[3 * u], j = trip[3 * u + 1], k = trip[3 * u + 2];
    double v = full[((size_t)b * n + i) * n + j];
    if (connected) v -= one_a[(size_t)b * n + i] * one_b[(size_t)b * n + j];
    out[(size_t)b * np + k] = v;
}

}  // namespace

cudaError_t launch_trace_normalize(void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap, int force,
                                   double* trace_out, int* status, cudaStream_t st) {
    trace_kernel<<<B, MT, 0, st>>>(sites, sites_f32, dims, n, chi_cap, force, trace_out, status);
    return cudaGetLastError();
}

cudaError_t launch_environments(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                                double* envL, double* envR, cudaStream_t st) {
    const dim3 grid((chi_cap + EW - 1) / EW, 2, B);
    for (int t = 0; t < n; ++t) {
        env_step_kernel<<<grid, 256, 0, st>>>(sites, sites_f32, dims, n, chi_cap, t, envL, envR);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_measure_1q(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                              const double* envL, const double* envR, const int* d_q, int nq, int comp, double* out,
                              cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    one_kernel<<<dim3(nq, B), MT, 0, st>>>(sites, sites_f32, dims, n, chi_cap, envL, envR, d_q, nq, comp, out);
    return cudaGetLastError();
}

size_t two_stack_doubles(int n, int B, int chi_cap) { return (size_t)2 * B * n * chi_cap; }
size_t two_part_doubles(int n, int B, int chi_cap) { return (size_t)B * n * n * ((chi_cap + TW - 1) / TW); }

cudaError_t launch_measure_2q(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                              const double* envL, const double* envR, int ca, int cb, const unsigned char* d_need_i,
                              double* wstack, double* part, double* full, cudaStream_t st) {
    const int ntiles = (chi_cap + TW - 1) / TW;
    const size_t smem = (size_t)3 * chi_cap * TW * sizeof(double);
    static_assert((size_t)3 * kMaxChi * TW * sizeof(double) <= 48 * 1024, "within the default shared memory");
    double* w[2] = {wstack, wstack + (size_t)B * n * chi_cap};
    for (int j = 0; j < n; ++j) {
        two_stack_kernel<<<dim3(ntiles, B), 256, smem, st>>>(sites, sites_f32, dims, n, chi_cap, envL, envR, ca, cb,
                                                            d_need_i, j, w[j & 1], w[(j + 1) & 1], part, ntiles);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const long long tot = (long long)B * n * n;
    two_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, dims, envL, d_need_i, n, chi_cap, B,
                                                                      ntiles, full);
    return cudaGetLastError();
}

cudaError_t launch_gather_2q(const double* full, const double* one_a, const double* one_b, const int* d_trip,
                             int m, int np, int n, int B, int connected, double* out, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const int tot = m * B;
    gather_kernel<<<(tot + 255) / 256, 256, 0, st>>>(full, one_a, one_b, d_trip, m, np, n, B, connected, out);
    return cudaGetLastError();
}

}  // namespace mpdo
