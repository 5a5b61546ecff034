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

// blockIdx.y == 0: left environments, 1: right environments
__global__ void __launch_bounds__(MT) env_kernel(const void* sites, int f32, const int* dims, int n, int cap,
                                                 double* envL, double* envR) {
    const int b = blockIdx.x;
    const int* dm = dims + (size_t)b * (n + 1);
    if (blockIdx.y == 0) {
        double* E = envL + (size_t)b * (n + 1) * cap;
        if (threadIdx.x == 0) E[0] = 1.0;
        __syncthreads();
        for (int p = 0; p < n; ++p) {
            vec_slice(site_ptr(sites, f32, b, p, n, cap), 0, dm[p], dm[p + 1], cap, E + (size_t)p * cap,
                      E + (size_t)(p + 1) * cap);
            __syncthreads();
        }
    } else {
        double* E = envR + (size_t)b * (n + 1) * cap;
        if (threadIdx.x == 0) E[(size_t)n * cap] = 1.0;
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int p = n - 1; p >= 0; --p) {
            const SiteRef S = site_ptr(sites, f32, b, p, n, cap);
            const double* rin = E + (size_t)(p + 1) * cap;
            double* rout = E + (size_t)p * cap;
            const int cl = dm[p], cr = dm[p + 1];
            for (int l = warp; l < cl; l += nw) {
                double acc = 0.0;
                for (int r = lane; r < cr; r += 32) acc = fma(S[((size_t)l * 4) * cap + r], rin[r], acc);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) rout[l] = acc;
            }
            __syncthreads();
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

// for each (b, i) with need[i]: w = L_i B_i[ca]; for j > i:
// full[b][i][j] = (w B_j[cb]) . R_{j+1} / E0 ;  w <- w B_j[I]
__global__ void __launch_bounds__(MT) two_kernel(const void* sites, int f32, const int* dims, int n, int cap,
                                                 const double* envL, const double* envR, int ca, int cb,
                                                 const unsigned char* need, double* full) {
    const int i = blockIdx.x, b = blockIdx.y;
    if (!need[i] || i >= n - 1) return;
    const int* dm = dims + (size_t)b * (n + 1);
    const double E0 = envL[((size_t)b * (n + 1) + n) * cap];
    __shared__ double w0[kMaxChi], w1[kMaxChi];
    const double* Li = envL + ((size_t)b * (n + 1) + i) * cap;
    vec_slice(site_ptr(sites, f32, b, i, n, cap), ca, dm[i], dm[i + 1], cap, Li, w0);
    __syncthreads();
    double* w = w0;
    double* wn = w1;
    for (int j = i + 1; j < n; ++j) {
        const SiteRef S = site_ptr(sites, f32, b, j, n, cap);
        const double* Rj = envR + ((size_t)b * (n + 1) + j + 1) * cap;
        const int cl = dm[j], cr = dm[j + 1];
        double part = 0.0;
        for (int r = threadIdx.x; r < cr; r += blockDim.x) {
            double acc = 0.0, accI = 0.0;
            for (int l = 0; l < cl; ++l) {
                const double wl = w[l];
                acc = fma(wl, S[((size_t)l * 4 + cb) * cap + r], acc);
                accI = fma(wl, S[((size_t)l * 4) * cap + r], accI);
            }
            part = fma(acc, Rj[r], part);
            wn[r] = accI;
        }
        const double tot = block_sum(part);
        if (threadIdx.x == 0) full[((size_t)b * n + i) * n + j] = tot / E0;
        __syncthreads();
        double* t = w;
        w = wn;
        wn = t;
    }
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
    env_kernel<<<dim3(B, 2), MT, 0, st>>>(sites, sites_f32, dims, n, chi_cap, envL, envR);
    return cudaGetLastError();
}

cudaError_t launch_measure_1q(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                              const double* envL, const double* envR, const int* d_q, int nq, int comp, double* out,
                              cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    one_kernel<<<dim3(nq, B), MT, 0, st>>>(sites, sites_f32, dims, n, chi_cap, envL, envR, d_q, nq, comp, out);
    return cudaGetLastError();
}

cudaError_t launch_measure_2q(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                              const double* envL, const double* envR, int ca, int cb, const unsigned char* d_need_i,
                              double* full, cudaStream_t st) {
    two_kernel<<<dim3(n, B), MT, 0, st>>>(sites, sites_f32, dims, n, chi_cap, envL, envR, ca, cb, d_need_i, full);
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
