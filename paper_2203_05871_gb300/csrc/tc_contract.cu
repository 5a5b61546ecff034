// Tensor-core (tcgen05, kind::tf32) contractions of the mixed-precision path:
// the site merge with the gate epilogue (a4-a6) and the reconstruction (a10).
//
// Split precision: every FP64 operand x is cut into two TF32 parts,
// x ~ hi + lo with hi = tf32(x) and lo = tf32(x - hi) (22 significant bits),
// and each product is formed as hi*hi + hi*lo + lo*hi (the lo*lo term is
// below 2^-22 relative).  The tensor core accumulates one K-chunk of 32 in
// FP32 in tensor memory; the chunk sums are then re-accumulated in FP64
// registers, so the FP32 accumulation error stays that of 32 terms.
//
// Tile: M = 128 rows x N = 64 columns, one CTA of 128 threads (4 warps).
// Operands are staged in shared memory in the K-major, no-swizzle layout
// of 8-row x 16-byte core matrices: element (row, k) of a chunk sits at
// (row/8)*SBO + (k/4)*LBO + (row%8)*16 + (k%4)*4 bytes, LBO = 128, SBO = 1024.
// One elected thread issues the MMAs; tcgen05.commit arrives on an mbarrier
// whose wait is bounded (a give-up sets MPDO_ST_TIMEOUT and the CTA returns
// after releasing its tensor memory).
//
// merge : D[(l,s1), (s2,r)] = sum_m A[l,s1,m] B[m,s2,r]; the tile holds 32 l x
//         4 s1 rows and 4 s2 x 16 r columns, so the 16x16 gate is applied in
//         registers (values of the 4 s1 rows of one l come from the 4 lanes of
//         a quad by shuffles); writes Theta' (row-major) and theta~ =
//         lambda_l Theta' (column-major), as the FP64 kernel does.
// recon : B_p'[(l,s1), j] = sum_c Theta'[(l,s1), c] Yk[j, c].
#include <mpdo.h>

#include "internal.h"

namespace mpdo {

namespace {

constexpr int TM = 128, TN = 64, TK = 32;
constexpr int LBO = 128, SBO = 1024;
constexpr int kTileA = TM * TK * 4;   // bytes of one A part (16 KB)
constexpr int kTileB = TN * TK * 4;   // bytes of one B part (8 KB)
constexpr int kSmem = 2 * kTileA + 2 * kTileB + 64;
constexpr long long kWaitLimit = 1ll << 26;   // mbarrier polls before giving up

__host__ __device__ constexpr uint32_t instr_desc_tf32(int M, int N) {
    // D = F32 (bits 4-5 = 1), A = B = TF32 (bits 7-9, 10-12 = 2), both K-major,
    // N >> 3 at bits 17-22, M >> 4 at bits 24-28
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr) {
    // start address >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45),
    // version 1 (bits 46-47), no swizzle (bits 61-63 = 0)
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// byte offset of element (row, k) inside one staged operand part
__device__ __forceinline__ int kmajor_offset(int row, int k) {
    return (row >> 3) * SBO + (k >> 2) * LBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ void split_store(unsigned char* hi, unsigned char* lo, int off, double x) {
    const float xf = (float)x;
    const uint32_t h = tf32_rna(xf);
    const uint32_t l = tf32_rna(xf - __uint_as_float(h));
    *reinterpret_cast<uint32_t*>(hi + off) = h;
    *reinterpret_cast<uint32_t*>(lo + off) = l;
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool kMerge>
__global__ void __launch_bounds__(128, 1) tc_kernel(const OpDesc* descs, int chi_cap) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const OpDesc& d = descs[blockIdx.z];
    const int ld = 4 * chi_cap;
    // tile origin: merge -> rows l0*4.., columns r0..r0+15 of each s2; recon -> rows i0.., columns j0..
    int M, K, ncols;
    const int i0 = blockIdx.y * TM;
    if constexpr (kMerge) {
        M = 4 * d.cl;
        K = d.cm;
        ncols = d.cr;   // r range
        if (i0 >= M || (int)blockIdx.x * 16 >= ncols) return;
    } else {
        M = d.m;
        K = d.n;
        ncols = *d.k_out;
        if (i0 >= M || (int)blockIdx.x * TN >= ncols) return;
    }
    unsigned char* Ahi = smem;
    unsigned char* Alo = smem + kTileA;
    unsigned char* Bhi = smem + 2 * kTileA;
    unsigned char* Blo = smem + 2 * kTileA + kTileB;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * kTileA + 2 * kTileB);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 2 * kTileA + 2 * kTileB + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int s_fail;
    __shared__ double Gs[256];
    if constexpr (kMerge) {
        for (int e = tid; e < 256; e += 128) Gs[e] = d.G[e];
    }

    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = instr_desc_tf32(TM, TN);
    const uint32_t aH = smem_u32(Ahi), aL = smem_u32(Alo), bH = smem_u32(Bhi), bL = smem_u32(Blo);

    double acc[TN];
#pragma unroll
    for (int n = 0; n < TN; ++n) acc[n] = 0.0;
    uint32_t phase = 0;
    const int r0 = blockIdx.x * 16, j0 = blockIdx.x * TN;
    for (int k0 = 0; k0 < K; k0 += TK) {
        // stage A (rows i0.., k0..k0+31) and B (64 columns, k0..)
        for (int e = tid; e < TM * TK; e += 128) {
            const int row = e / TK, k = e % TK;
            const int gi = i0 + row, gk = k0 + k;
            double x = 0.0;
            if (gi < M && gk < K) x = kMerge ? site_ld(d.A, (size_t)gi * chi_cap + gk, d.site_f32) : d.thetap[(size_t)gi * ld + gk];
            split_store(Ahi, Alo, kmajor_offset(row, k), x);
        }
        for (int e = tid; e < TN * TK; e += 128) {
            double x = 0.0;
            int col, k;
            if constexpr (kMerge) {
                // column = s2*16 + rl; element (m = k0+k, s2, r0+rl), r contiguous in memory
                k = e / TN;
                col = e % TN;
                const int s2 = col >> 4, rl = col & 15, gm = k0 + k, gr = r0 + rl;
                if (gm < K && gr < ncols) x = site_ld(d.B, ((size_t)gm * 4 + s2) * chi_cap + gr, d.site_f32);
            } else {
                col = e / TK;
                k = e % TK;
                const int gj = j0 + col, gk = k0 + k;
                if (gj < ncols && gk < K) x = d.Yk[(size_t)gj * ld + gk];
            }
            split_store(Bhi, Blo, kmajor_offset(col, k), x);
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            for (int q = 0; q < TK / 8; ++q) {   // K = 8 per instruction, 2 core matrices
                const uint32_t off = q * 2 * LBO;
                mma_tf32(tmem, smem_desc(aH + off), smem_desc(bH + off), idesc, q > 0 ? 1u : 0u);
                mma_tf32(tmem, smem_desc(aH + off), smem_desc(bL + off), idesc, 1u);
                mma_tf32(tmem, smem_desc(aL + off), smem_desc(bH + off), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(mbar)));
        }
        if (!mbar_wait(smem_u32(mbar), phase)) s_fail = 1;
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // chunk sum of this thread's row -> FP64 accumulators
        {
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            float v[16];
#pragma unroll
            for (int c = 0; c < TN / 16; ++c) {
                tmem_ld16(taddr + c * 16, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[c * 16 + i] += (double)v[i];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (s_fail) break;
    }
    // release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
    if (s_fail) {
        if (tid == 0) atomicOr(d.status, (int)MPDO_ST_TIMEOUT);
        return;
    }

    const int row = i0 + tid;
    if constexpr (kMerge) {
        // gate: out[(s1',s2'), r] = sum G[(s1' s2'), (s1 s2)] Theta[(l,s1),(s2,r)]; the
        // four s1 rows of one l are the four lanes of a quad
        const int s1p = tid & 3, qbase = lane & ~3;
        const int l = row >> 2;
        const double lam = (l < d.cl && d.lam_left) ? d.lam_left[l] : 1.0;
#pragma unroll
        for (int rl = 0; rl < 16; ++rl) {
            double o[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int s1 = 0; s1 < 4; ++s1) {
#pragma unroll
                for (int s2 = 0; s2 < 4; ++s2) {
                    const double v = __shfl_sync(0xffffffffu, acc[s2 * 16 + rl], qbase + s1);
#pragma unroll
                    for (int s2p = 0; s2p < 4; ++s2p) o[s2p] = fma(Gs[(s1p * 4 + s2p) * 16 + s1 * 4 + s2], v, o[s2p]);
                }
            }
            const int r = r0 + rl;
            if (row < M && r < ncols) {
#pragma unroll
                for (int s2p = 0; s2p < 4; ++s2p) {
                    const int col = s2p * d.cr + r;
                    d.thetap[(size_t)row * ld + col] = o[s2p];
                    d.Acm[(size_t)col * ld + row] = lam * o[s2p];
                }
            }
        }
    } else {
        if (row < M)
            for (int n = 0; n < TN; ++n) {
                const int j = j0 + n;
                if (j < ncols) site_st(d.A, (size_t)row * chi_cap + j, acc[n], d.site_f32);
            }
    }
}

}  // namespace

uint32_t tc_instr_desc_tf32(int M, int N) { return instr_desc_tf32(M, N); }
uint64_t tc_smem_desc(uint32_t saddr) { return smem_desc(saddr); }

cudaError_t tc_prepare() {
    cudaError_t e = cudaFuncSetAttribute(tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

cudaError_t launch_tc_merge_gate(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    dim3 grid((chi_cap + 15) / 16, (4 * chi_cap + TM - 1) / TM, nops);
    tc_kernel<true><<<grid, 128, kSmem, st>>>(d_desc, chi_cap);
    return cudaGetLastError();
}

cudaError_t launch_tc_reconstruct(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    dim3 grid((chi_cap + TN - 1) / TN, (4 * chi_cap + TM - 1) / TM, nops);
    tc_kernel<false><<<grid, 128, kSmem, st>>>(d_desc, chi_cap);
    return cudaGetLastError();
}

}  // namespace mpdo
