// FP64 one-sided (Hestenes) Jacobi SVD of the bond matrices of one layer.
//
// App. B compresses |rho>> bond by bond from its Schmidt spectrum.  Each op
// hands this kernel c rows of length L (the rows of theta~ when m <= n, or
// its columns together with a c x c accumulator Z when m > n).  Plane
// rotations from the left make the rows mutually orthogonal; row j then
// equals s_j * v_j^T (or Z row j = v_j^T), which the truncation step reads.
//
// Parallel order: the round-robin ("circle") tournament pairs all c rows in
// c' - 1 steps of c'/2 disjoint pairs (c' = c rounded up to even), so every
// pair of rows meets once per sweep.  Each pair is handled by one warp: the
// three inner products are reduced with warp shuffles, the rotation is
// applied in a second pass.  The CTAs that share an op meet in a counter
// barrier after every step; every wait is bounded by a wall-clock limit and
// gives up with MPDO_ST_TIMEOUT instead of hanging.  The kernel is launched
// cooperatively, so all CTAs are co-resident.
//
// Rotation (Rutishauser): a = |w_p|^2, b = |w_q|^2, g = w_p.w_q,
// zeta = (b - a) / 2g, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// cs = 1/sqrt(1+t^2), sn = cs t;  w_p <- cs w_p - sn w_q, w_q <- sn w_p + cs w_q.
// A pair is skipped when |g| <= tol sqrt(a b) (tol = sqrt(L) eps unless set).
// A row whose norm is at most eps * ||W||_F is numerically zero: it is set to
// zero and never rotated (its direction is rounding noise).
#include <float.h>
#include <mpdo.h>

#include "internal.h"

namespace mpdo {

namespace {

constexpr int JW = 8;             // warps per CTA
constexpr int JT = JW * 32;
constexpr int kSyncWords = 8 + kMaxSweepsCap;   // per op: [0] arrivals [1] abort [8+s] rotations in sweep s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of the G CTAs working on one op; returns false if it gave up.
__device__ bool op_barrier(unsigned* sw, int G, unsigned& gen, unsigned long long timeout_ns) {
    __shared__ int s_ok;
    __threadfence();
    __syncthreads();
    if (G == 1) return true;
    ++gen;
    if (threadIdx.x == 0) {
        atomicAdd(&sw[0], 1u);
        const unsigned target = gen * (unsigned)G;
        const unsigned long long t0 = globaltimer_ns();
        int ok = 1;
        while (ld_acquire(&sw[0]) < target) {
            if (ld_acquire(&sw[1]) != 0u) {
                ok = 0;
                break;
            }
            if (globaltimer_ns() - t0 > timeout_ns) {
                atomicExch(&sw[1], 1u);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int tour_player(int x, int step, int cp) {
    return x == 0 ? 0 : 1 + ((x - 1 + step) % (cp - 1));
}

// one warp: orthogonalise rows p and q; returns 1 if a rotation was applied
__device__ int pair_rotate(double* wp, double* wq, int L, double* zp, double* zq, int c, double floor2,
                           double tol, int lane) {
    double a = 0.0, b = 0.0, g = 0.0;
    for (int i = lane; i < L; i += 32) {
        const double x = __ldcg(wp + i), y = __ldcg(wq + i);
        a = fma(x, x, a);
        b = fma(y, y, b);
        g = fma(x, y, g);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    g = warp_sum(g);
    if (a <= floor2 || b <= floor2) {
        if (a <= floor2)
            for (int i = lane; i < L; i += 32) __stcg(wp + i, 0.0);
        if (b <= floor2)
            for (int i = lane; i < L; i += 32) __stcg(wq + i, 0.0);
        return 0;
    }
    if (g == 0.0 || fabs(g) <= tol * sqrt(a) * sqrt(b)) return 0;
    const double zeta = (b - a) / (2.0 * g);
    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
    const double cs = 1.0 / sqrt(1.0 + t * t);
    const double sn = cs * t;
    for (int i = lane; i < L; i += 32) {
        const double x = __ldcg(wp + i), y = __ldcg(wq + i);
        __stcg(wp + i, cs * x - sn * y);
        __stcg(wq + i, sn * x + cs * y);
    }
    if (zp) {
        for (int i = lane; i < c; i += 32) {
            const double x = __ldcg(zp + i), y = __ldcg(zq + i);
            __stcg(zp + i, cs * x - sn * y);
            __stcg(zq + i, sn * x + cs * y);
        }
    }
    return 1;
}

__global__ void __launch_bounds__(JT) jacobi_kernel(const OpDesc* descs, const int* cta_op, const int* cta_rank,
                                                    const int* group, unsigned* sync, int max_sweeps, double tol_in,
                                                    unsigned long long timeout_ns, int ld) {
    const int op = cta_op[blockIdx.x];
    const int g = cta_rank[blockIdx.x];
    const int G = group[op];
    const OpDesc& d = descs[op];
    unsigned* sw = sync + (size_t)op * kSyncWords;
    const int c = d.c, L = d.L;
    double* W = d.W;
    double* Z = d.transposed ? d.Z : nullptr;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = g * JW + warp, NW = G * JW;
    unsigned gen = 0;
    __shared__ double s_floor2;

    // Z = I and row norms
    for (int row = gw; row < c; row += NW) {
        const double* w = W + (size_t)row * ld;
        double a = 0.0;
        for (int i = lane; i < L; i += 32) {
            const double x = __ldcg(w + i);
            a = fma(x, x, a);
        }
        a = warp_sum(a);
        if (lane == 0) __stcg(d.snorm + row, a);
        if (Z)
            for (int i = lane; i < c; i += 32) __stcg(Z + (size_t)row * ld + i, i == row ? 1.0 : 0.0);
    }
    if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int j = 0; j < c; ++j) f += __ldcg(d.snorm + j);
        s_floor2 = DBL_EPSILON * DBL_EPSILON * f;
    }
    __syncthreads();
    {
        const double floor2 = s_floor2;
        const double tol = tol_in > 0.0 ? tol_in : sqrt((double)(L > 1 ? L : 1)) * DBL_EPSILON;
        const int cp = c + (c & 1);
        const int npairs = cp / 2;
        int sweeps = max_sweeps < kMaxSweepsCap ? max_sweeps : kMaxSweepsCap;
        bool converged = (c <= 1);
        for (int sweep = 0; sweep < sweeps && !converged; ++sweep) {
            int rot = 0;
            for (int step = 0; step < cp - 1; ++step) {
                for (int i = gw; i < npairs; i += NW) {
                    const int P = tour_player(i, step, cp), Q = tour_player(cp - 1 - i, step, cp);
                    if (P >= c || Q >= c) continue;
                    const int p = P < Q ? P : Q, q = P < Q ? Q : P;
                    rot += pair_rotate(W + (size_t)p * ld, W + (size_t)q * ld, L,
                                       Z ? Z + (size_t)p * ld : nullptr, Z ? Z + (size_t)q * ld : nullptr, c,
                                       floor2, tol, lane);
                }
                if (step == cp - 2 && lane == 0 && rot > 0) atomicAdd(&sw[8 + sweep], (unsigned)rot);
                if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
            }
            converged = (ld_acquire(&sw[8 + sweep]) == 0u);
            // every CTA must read the count before anyone starts the next sweep's counter;
            // counters are per sweep, so no reset is needed.
        }
        if (!converged && g == 0 && threadIdx.x == 0) atomicOr(d.status, (int)MPDO_ST_NOCONV);
    }
    return;
timeout:
    if (threadIdx.x == 0) atomicOr(d.status, (int)MPDO_ST_TIMEOUT);
}

}  // namespace

int jacobi_threads() { return JT; }
size_t jacobi_sync_words_per_op() { return kSyncWords; }

cudaError_t jacobi_max_resident(int* blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, JT, 0);
    if (e != cudaSuccess) return e;
    *blocks = sms * per_sm;
    return cudaSuccess;
}

cudaError_t launch_jacobi(const OpDesc* d_desc, int nops, const int* d_cta_op, const int* d_cta_rank,
                          const int* d_group, unsigned* d_sync, int grid, int max_sweeps, double tol,
                          unsigned long long timeout_ns, int ld, cudaStream_t st) {
    (void)nops;
    if (grid <= 0) return cudaSuccess;
    void* args[] = {(void*)&d_desc, (void*)&d_cta_op, (void*)&d_cta_rank, (void*)&d_group, (void*)&d_sync,
                    (void*)&max_sweeps, (void*)&tol, (void*)&timeout_ns, (void*)&ld};
    return cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid), dim3(JT), args, 0, st);
}

}  // namespace mpdo
