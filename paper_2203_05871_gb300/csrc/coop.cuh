// Device helpers shared by the cooperative per-op kernels (QR, Jacobi SVD):
// a bounded barrier among the CTAs that work on one op, and warp reductions.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace mpdo {

// per-op sync words: [0] barrier arrivals, [1] abort flag, [2, 8) Jacobi pair counters,
// [8 + s] rotations and [8 + kMaxSweepsCap + s] largest off-orthogonality in Jacobi
// sweep s, then one version per Jacobi row block (at most 4 kMaxChi blocks)
constexpr int kSyncWords = 8 + 2 * kMaxSweepsCap + 4 * kMaxChi;

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
__device__ __forceinline__ bool op_barrier(unsigned* sw, int G, unsigned& gen, unsigned long long timeout_ns) {
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

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mpdo
