// FP64-accurate batched GEMM on the tcgen05 tensor cores (the mixed path's
// contractions and its SVD-preconditioner products).
//
//   C = alpha * A B + beta * D  (- I when sub_identity),  A: M x K, B: K x N,
// FP64 (or f32) in and out, computed from exact products of narrow slices of
// the operands (the error-free splitting of Ozaki, Ogita, Oishi & Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012):
//
// 1. Slicing (oz_slice_kernel).  Each row i of A is scaled by 2^-e_i, e_i the
//    binary exponent of its largest |A_ik| (so |a| < 1), rounded to the
//    integer X = round(2^47 a) and cut into S = 6 balanced base-256 digits,
//    a ~ 2^-7 sum_t sigma_t 2^-8t with integers |sigma_t| <= 128; a slice
//    keeps 8 significant bits, so it is exact in bf16 (MPDO_MIXED_BF16X3) and
//    in tf32 (MPDO_MIXED_TF32), and it is stored as sigma_t 2^-8t.  B is cut
//    the same way per column j (exponent f_j).  The rounding error is at most
//    2^-48 of the row's largest entry.
// 2. Products (oz_gemm_kernel).  Every slice pair (t, u) with t + u <= 5 is
//    multiplied on the tensor core: a product sigma_t sigma_u has at most 16
//    bits, so it is exact in FP32, and the sums stay exact while they fit 24
//    bits.  One accumulator per level d = t + u in tensor memory (six), each
//    product already at its own scale 2^-8d through the stored slices.  Every
//    256 values of K the accumulators are drained into FP64 registers: 256
//    products of up to 2^14 fit 2^22, so levels 0 to 3 (at most four pairs,
//    2^24) are summed without any rounding, whatever rounding and alignment
//    the tensor core's FP32 accumulation uses; levels 4 and 5 round at 2^-24
//    of themselves, below 2^-50 of the result.  A drain joins the six levels
//    into one int64 (their exact integer parts) and adds it in FP64.  (Folding levels 3-5 into one
//    accumulator was measured at 2e-12 on the GPU: the accumulator then holds
//    level-3 magnitudes and drops the low bits of every level-5 product at
//    every MMA.)
// 3. Epilogue: C_ij = alpha 2^(e_i + f_j - 14) sum_d L_d + beta D_ij.
// Error: about 2^-46 |A_i|_max |B_j|_max per term of the sum (a numpy model of
// the scheme with per-MMA rounding: 3e-14 of |A_i| |B_j| sqrt(K)), against
// FP64's 2^-53 |A_ik B_kj|: FP64-class accuracy at tensor-core speed.
//
// Data layout.  The slices are written in the tcgen05 canonical K-major,
// no-swizzle layout, pre-tiled: a block of R rows x 64 bytes of K (32 bf16 or
// 16 tf32 values; R = 128 for A, 64 for B) is R x 64 bytes, element (row, k) at
// (row/8)*512 + (k/g)*128 + (row%8)*16 + (k%g)*esize, g = 16/esize (core
// matrices of 8 rows x 16 bytes, LBO = 128 B along K, SBO = 512 B along rows),
// so one cp.async.bulk moves a block into shared memory as it is.  Blocks are
// [slice][row tile][k tile].
//
// Kernel.  One CTA per 128 x 64 tile of C, 320 threads: warp 0 issues the
// bulk copies of the 6 + 6 slice blocks of each k tile into a 3-stage ring
// (72 KB per stage), warp 1 issues the 42 MMAs of a k tile (21 pairs x 2
// instructions of K = 16 bf16 / 8 tf32; M = 128, N = 64) and commits, warps
// 2-9 drain the six accumulators (384 TMEM columns; warp w reads lanes
// 32 (w % 4) .. +31, its half of the 64 columns).  Every wait is bounded by timeout_ns; a wait that
// gives up records MPDO_ST_TIMEOUT in the problem's status word, the other roles
// leave their loops at the next poll, outstanding copies and MMAs are waited
// for (bounded) and the tensor memory is released before the CTA returns.
#include <mpdo.h>

#include <cuda_bf16.h>

#include "internal.h"

namespace mpdo {

namespace {

constexpr int kS = 6;                  // slices per operand
constexpr int kPairs = 21;             // (t, u) with t + u <= 5
constexpr int kLevels = 6;             // one accumulator per level t + u
constexpr int kTileM = 128;            // rows of A (and of C) per tile
constexpr int kTileN = 64;             // columns of B (and of C) per tile
constexpr int kBlockA = kTileM * 64;   // bytes of one slice block of A (8 KB)
constexpr int kBlockB = kTileN * 64;   // of B (4 KB)
constexpr int kStageBytes = kS * (kBlockA + kBlockB);   // A and B slices of one k tile
constexpr int kStages = 3;
constexpr int kRangeK = 256;           // K values between accumulator drains
constexpr int kThreads = 320;
constexpr int kSmem = kStages * kStageBytes + 1024;
static_assert(kLevels * kTileN <= 512, "accumulators exceed tensor memory");
static_assert(kTileM == 128 && kTileN == 64, "oz_set_tiles (internal.h) assumes 128 x 64 tiles");
constexpr int LBO = 128, SBO = 512;

__host__ __device__ constexpr int kt_elems(int esize) { return 64 / esize; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    // start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45), version 1 (46-47), no swizzle
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
           (1ull << 46);
}

// D = F32 (bits 4-5 = 1); A, B = BF16 (1) or TF32 (2) at bits 7-9, 10-12; K-major;
// N >> 3 at bits 17-22; M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc(bool bf16, int M, int N) {
    const uint32_t ab = bf16 ? 1u : 2u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// bounded wait; false when it gave up (timeout) or another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int* abort_flag,
                                          unsigned long long timeout_ns) {
    const unsigned long long t0 = gtimer();
    for (int it = 0;; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if ((it & 63) == 63) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > timeout_ns) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void mma(bool bf16, uint32_t dtmem, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t accumulate) {
    if (bf16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
            "l"(a), "l"(b), "r"(id), "r"(accumulate));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
            "l"(a), "l"(b), "r"(id), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

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

__device__ __forceinline__ int pair_t(int p) {   // pairs in order of level: (0,0) (0,1)(1,0) (0,2)(1,1)(2,0) ...
    constexpr int T[kPairs] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5};
    return T[p];
}
__device__ __forceinline__ int pair_u(int p) {
    constexpr int U[kPairs] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0};
    return U[p];
}

// index of element (r, k) of an operand view
__device__ __forceinline__ size_t oz_index(const OzOperand& X, int r, int k) {
    if (X.mode == 1) return ((size_t)k * 4 + (size_t)(r / X.cr)) * X.cap + (r % X.cr);
    return (size_t)(X.gather ? X.gather[r] : r) * X.rs + (size_t)k * X.ks;
}

// The slicing works on bit patterns with integer arithmetic only: GB300
// issues FP64 instructions at a small fraction of its integer and FP32 rate,
// and the FP64 form of the same cut (scale, round, subtract, repeat) costs
// about 25 of them per element.
//
// Bit pattern of element (r, k), zero-extended (f32 views: 32 bits).
__device__ __forceinline__ unsigned long long oz_bits(const OzOperand& X, int r, int k) {
    const size_t i = oz_index(X, r, k);
    return X.f32 ? (unsigned long long)__float_as_uint(static_cast<const float*>(X.base)[i])
                 : (unsigned long long)__double_as_longlong(static_cast<const double*>(X.base)[i]);
}

// |x| as an unsigned key that orders like |x| within one storage type
__device__ __forceinline__ unsigned long long abs_key(unsigned long long bits, bool f32) {
    return f32 ? (bits & 0x7fffffffull) : (bits & 0x7fffffffffffffffull);
}

__device__ __forceinline__ bool key_nonfinite(unsigned long long key, bool f32) {
    return f32 ? key >= 0x7f800000ull : key >= 0x7ff0000000000000ull;
}

// e with 2^(e-1) <= max |x| < 2^e from the largest key (0 for a zero row)
__device__ __forceinline__ int key_exponent(unsigned long long key, bool f32) {
    if (key == 0) return 0;
    int e = 0;
    if (f32) {
        const int E = (int)(key >> 23);
        if (E > 0) return E - 126;
        frexp((double)__uint_as_float((unsigned)key), &e);      // subnormal float
    } else {
        const int E = (int)(key >> 52);
        if (E > 0) return E - 1022;
        frexp(__longlong_as_double((long long)key), &e);        // subnormal double
    }
    return e;
}

// X = round(x 2^(47 - e)) for a finite x = +-m 2^p of a row with exponent e
// (|x| < 2^e, so |X| <= 2^47), ties away from zero
__device__ __forceinline__ long long fixed_of(unsigned long long bits, bool f32, int e) {
    bool neg;
    unsigned long long m;
    int p;
    if (f32) {
        neg = (bits >> 31) & 1;
        const int E = (int)((bits >> 23) & 0xff);
        m = bits & 0x7fffffull;
        if (E) {
            m |= 1ull << 23;
            p = E - 150;
        } else {
            p = -149;
        }
    } else {
        neg = bits >> 63;
        const int E = (int)((bits >> 52) & 0x7ff);
        m = bits & 0xfffffffffffffull;
        if (E) {
            m |= 1ull << 52;
            p = E - 1075;
        } else {
            p = -1074;
        }
    }
    const int sh = p + 47 - e;
    long long X;
    if (m == 0)
        X = 0;
    else if (sh >= 0)
        X = (long long)(m << (sh < 63 ? sh : 63));   // m 2^sh < 2^47: no bits leave
    else if (sh <= -62)
        X = 0;
    else
        X = (long long)((m + (1ull << (-sh - 1))) >> -sh);
    return neg ? -X : X;
}

// The slices of G consecutive fixed-point values X[0..G) (|X| <= 2^47):
// balanced base-256 digits X = sum_t sigma_t 2^(8(5 - t)), |sigma_t| <= 128,
// from the lowest digit up; stored as sigma_t 2^-8t, 16 bytes per slice.
// nan: the row has a non-finite entry, every slice is NaN.
template <int G, bool kBf16>
__device__ __forceinline__ void slice_group(const long long* X, bool nan, uint4* out /* [kS] */) {
    int sig[kS][G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        long long d = X[g];
#pragma unroll
        for (int t = kS - 1; t > 0; --t) {
            const int lo = (int)(((unsigned)d + 128u) & 255u) - 128;
            sig[t][g] = lo;
            d = (d - lo) >> 8;                                      // exact: d - lo = 0 mod 256
        }
        sig[0][g] = (int)d;
    }
#pragma unroll
    for (int t = 0; t < kS; ++t) {
        const float scale = __int_as_float((127 - 8 * t) << 23);   // 2^-8t
        float sl[G];
#pragma unroll
        for (int g = 0; g < G; ++g) sl[g] = nan ? __int_as_float(0x7fc00000) : (float)sig[t][g] * scale;
        if constexpr (kBf16) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const __nv_bfloat162 p = __floats2bfloat162_rn(sl[2 * h], sl[2 * h + 1]);
                w[h] = *reinterpret_cast<const uint32_t*>(&p);
            }
            out[t] = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            out[t] = make_uint4(__float_as_uint(sl[0]), __float_as_uint(sl[1]), __float_as_uint(sl[2]),
                                __float_as_uint(sl[3]));
        }
    }
}

// Strided views (a transposed operand, the right site of a merge): a block
// takes 32 consecutive rows, lane = row and warp = a slice of the K range, so
// that the 32 lanes of a load read 32 neighbouring rows at one k (coalesced).
template <bool kBf16>
__device__ void slice_rows_tiled(const OzOperand& X, int r0, int R, int K, int Kt, unsigned char* out, int* ex,
                                 int tile, int Rt) {
    constexpr int esize = kBf16 ? 2 : 4;
    constexpr int G = 16 / esize;
    constexpr int KT = kt_elems(esize);
    __shared__ unsigned long long s_mx[8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool f32 = X.f32 != 0;
    const int r = r0 + lane;
    const bool live = r < R;
    unsigned long long mx = 0;
    if (live)
        for (int k = warp; k < K; k += 8) {
            const unsigned long long key = abs_key(oz_bits(X, r, k), f32);
            mx = key > mx ? key : mx;
        }
    s_mx[warp][lane] = mx;
    __syncthreads();
    for (int w = 0; w < 8; ++w) mx = s_mx[w][lane] > mx ? s_mx[w][lane] : mx;
    const bool bad = key_nonfinite(mx, f32);   // the largest key of a row with a NaN or an inf is one
    const int e = bad ? 0 : key_exponent(mx, f32);
    if (warp == 0) ex[r] = e;
    const int rt = r / tile, rr = r % tile;
    const size_t block = (size_t)tile * 64;
    const size_t within = (size_t)(rr >> 3) * SBO + (size_t)(rr & 7) * 16;
    for (int g0 = warp * G; g0 < Kt * KT; g0 += 8 * G) {
        long long x[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int k = g0 + g;
            x[g] = (live && !bad && k < K) ? fixed_of(oz_bits(X, r, k), f32, e) : 0;
        }
        uint4 sl[kS];
        slice_group<G, kBf16>(x, bad && live, sl);
        const int kt = g0 / KT, kk = g0 % KT;
#pragma unroll
        for (int t = 0; t < kS; ++t) {
            unsigned char* blk = out + (((size_t)t * Rt + rt) * Kt + kt) * block;
            *reinterpret_cast<uint4*>(blk + within + (size_t)(kk / G) * LBO) = sl[t];
        }
    }
}

// grid (row groups of 8, 2 = A | B, problems).  Views whose rows are
// contiguous (ks == 1) take one warp per row, lanes along k; the others 32 rows
// per block (slice_rows_tiled), the blocks past rows / 32 returning at once.
template <bool kBf16>
__global__ void __launch_bounds__(256) oz_slice_kernel(const OzProblem* probs) {
    constexpr int esize = kBf16 ? 2 : 4;
    constexpr int G = 16 / esize;          // values per 16-byte store
    constexpr int KT = kt_elems(esize);
    const OzProblem& P = probs[blockIdx.z];
    const bool isB = blockIdx.y == 1;
    const OzOperand& X = isB ? P.B : P.A;
    const int N = P.Ndyn ? *P.Ndyn : P.N;
    const int R = isB ? N : P.M;
    const int tile = isB ? kTileN : kTileM;         // rows per block
    const int Rt = isB ? P.Nt : P.Mt;
    const int K = P.K, Kt = P.Kt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* out = static_cast<unsigned char*>(isB ? P.bs : P.as);
    int* ex = isB ? P.eb : P.ea;
    if (!(X.mode == 0 && X.ks == 1)) {
        const int r0 = blockIdx.x * 32;
        if (r0 >= Rt * tile) return;   // uniform over the block (Rt * tile is a multiple of 32)
        slice_rows_tiled<kBf16>(X, r0, R, K, Kt, out, ex, tile, Rt);
        return;
    }
    const int r = blockIdx.x * 8 + warp;
    if (r >= Rt * tile) return;
    const bool live = r < R;
    const bool f32 = X.f32 != 0;
    unsigned long long mx = 0;
    if (live)
        for (int k = lane; k < K; k += 32) {
            const unsigned long long key = abs_key(oz_bits(X, r, k), f32);
            mx = key > mx ? key : mx;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    const bool bad = key_nonfinite(mx, f32);
    const int e = bad ? 0 : key_exponent(mx, f32);
    if (lane == 0) ex[r] = e;
    const int rt = r / tile, rr = r % tile;
    const size_t block = (size_t)tile * 64;
    const size_t within = (size_t)(rr >> 3) * SBO + (size_t)(rr & 7) * 16;
    for (int g0 = lane * G; g0 < Kt * KT; g0 += 32 * G) {
        long long x[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int k = g0 + g;
            x[g] = (live && !bad && k < K) ? fixed_of(oz_bits(X, r, k), f32, e) : 0;
        }
        uint4 sl[kS];
        slice_group<G, kBf16>(x, bad && live, sl);
        const int kt = g0 / KT, kk = g0 % KT;
#pragma unroll
        for (int t = 0; t < kS; ++t) {
            unsigned char* blk = out + (((size_t)t * Rt + rt) * Kt + kt) * block;
            *reinterpret_cast<uint4*>(blk + within + (size_t)(kk / G) * LBO) = sl[t];
        }
    }
}

// barriers: full[kStages], empty[kStages], accumulators full, accumulators drained, final
constexpr int kBarFull = 0, kBarEmpty = kStages, kBarAccFull = 2 * kStages, kBarAccEmpty = 2 * kStages + 1,
              kBarFinal = 2 * kStages + 2;

template <bool kBf16>
__global__ void __launch_bounds__(kThreads, 1) oz_gemm_kernel(const OzProblem* probs,
                                                               unsigned long long timeout_ns) {
    constexpr int esize = kBf16 ? 2 : 4;
    constexpr int KT = kt_elems(esize);
    constexpr int kRangeTiles = kRangeK / KT;
    extern __shared__ __align__(1024) unsigned char smem[];
    const OzProblem& P = probs[blockIdx.z];
    const int N = P.Ndyn ? *P.Ndyn : P.N;
    const int mt = blockIdx.y, nt = blockIdx.x;
    if (mt * kTileM >= P.M || nt * kTileN >= N) return;
    const int Kt = P.Kt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kStages * kStageBytes + 128);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + kStages * kStageBytes + 144);
    if (threadIdx.x == 0) {
        *abort_flag = 0;
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + kBarFull + s)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + kBarEmpty + s)));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + kBarAccFull)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(bar + kBarAccEmpty)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + kBarFinal)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const int nrange = (Kt + kRangeTiles - 1) / kRangeTiles;

    if (warp == 0) {
        // producer: bulk copies of the slice blocks of k tile kt into stage kt % kStages
        if (lane == 0) {
            const unsigned char* as = static_cast<const unsigned char*>(P.as);
            const unsigned char* bs = static_cast<const unsigned char*>(P.bs);
            int issued = 0;
            for (int kt = 0; kt < Kt; ++kt) {
                const int s = kt % kStages;
                if (kt >= kStages &&
                    !mbar_wait(smem_u32(bar + kBarEmpty + s), ((kt / kStages) - 1) & 1, abort_flag, timeout_ns))
                    break;
                const uint32_t full = smem_u32(bar + kBarFull + s);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full), "r"(kStageBytes)
                             : "memory");
                unsigned char* st = smem + (size_t)s * kStageBytes;
                for (int t = 0; t < kS; ++t) {
                    const unsigned char* srcA = as + (((size_t)t * P.Mt + mt) * Kt + kt) * kBlockA;
                    const unsigned char* srcB = bs + (((size_t)t * P.Nt + nt) * Kt + kt) * kBlockB;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(st + t * kBlockA)),
                        "l"(srcA), "r"(kBlockA), "r"(full)
                        : "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_u32(st + kS * kBlockA + t * kBlockB)),
                        "l"(srcB), "r"(kBlockB), "r"(full)
                        : "memory");
                }
                issued = kt + 1;
            }
            // copies still in flight complete on their full barrier before the CTA leaves
            for (int kt = (issued > kStages ? issued - kStages : 0); kt < issued; ++kt)
                mbar_wait(smem_u32(bar + kBarFull + kt % kStages), (kt / kStages) & 1, abort_flag, timeout_ns);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t id = idesc(kBf16, kTileM, kTileN);
            int r = 0;
            bool first[kLevels];
#pragma unroll
            for (int l = 0; l < kLevels; ++l) first[l] = true;
            for (int kt = 0; kt < Kt; ++kt) {
                const int s = kt % kStages;
                if (kt % kRangeTiles == 0 && kt > 0) {
                    // accumulators of the previous range must be drained first
                    if (!mbar_wait(smem_u32(bar + kBarAccEmpty), (r - 1) & 1, abort_flag, timeout_ns)) break;
#pragma unroll
                    for (int l = 0; l < kLevels; ++l) first[l] = true;
                }
                if (!mbar_wait(smem_u32(bar + kBarFull + s), (kt / kStages) & 1, abort_flag, timeout_ns)) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t st = smem_u32(smem + (size_t)s * kStageBytes);
#pragma unroll
                for (int p = 0; p < kPairs; ++p) {
                    const int t = pair_t(p), u = pair_u(p);
                    const int lvl = t + u;
                    const uint32_t d = tmem + (uint32_t)(lvl * kTileN);
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const uint32_t off = q * 2 * LBO;
                        mma(kBf16, d, smem_desc(st + t * kBlockA + off), smem_desc(st + kS * kBlockA + u * kBlockB + off),
                            id, first[lvl] ? 0u : 1u);
                        first[lvl] = false;
                    }
                }
                commit(smem_u32(bar + kBarEmpty + s));   // frees the stage once these MMAs have read it
                if (kt % kRangeTiles == kRangeTiles - 1 || kt == Kt - 1) {
                    commit(smem_u32(bar + kBarAccFull));   // accumulators of range r complete
                    ++r;
                }
            }
            commit(smem_u32(bar + kBarFinal));
            mbar_wait(smem_u32(bar + kBarFinal), 0, abort_flag, timeout_ns);   // every MMA issued has completed
        }
    } else {
        // epilogue warps 2..9: rows 32 (warp % 4) + lane, columns half * 32 .. + 31
        const int ew = warp - 2;
        const int lane_base = 32 * (warp & 3);
        const int half = ew >> 2;
        const uint32_t taddr = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(half * 32);
        double acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.0;
        bool ok = true;
        for (int r = 0; r < nrange; ++r) {
            if (!mbar_wait(smem_u32(bar + kBarAccFull), r & 1, abort_flag, timeout_ns)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // level d holds n_d 2^-8d with n_d an integer (exact for d <= 3;
            // levels 4 and 5 are rounded to the nearest 2^-32 and 2^-40):
            // the range's sum is S 2^-40 with the integer
            // S = sum_d n_d 2^(8 (5 - d)), |S| < 2^63, formed in int64 and
            // converted once (integer arithmetic instead of twelve FP64
            // operations per element).  A NaN slice reaches level 0.
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                long long S[16];
                unsigned nan = 0;
#pragma unroll
                for (int lvl = 0; lvl < kLevels; ++lvl) {
                    float v[16];
                    tmem_ld16(taddr + (uint32_t)(lvl * kTileN + c * 16), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const float scale = __int_as_float((127 + 8 * lvl) << 23);   // 2^8d
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const long long n = __float2int_rn(v[i] * scale);
                        if (lvl == 0) {
                            S[i] = n;
                            nan |= (v[i] != v[i]) ? 1u << i : 0u;
                        } else {
                            S[i] = S[i] * 256 + n;
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    acc[c * 16 + i] += ((nan >> i) & 1u) ? __longlong_as_double(0x7ff8000000000000ll) : (double)S[i];
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar + kBarAccEmpty)) : "memory");
        }
        if (ok && !*abort_flag) {
            const int i = mt * kTileM + lane_base + lane;
            if (i < P.M) {
                const int ei = P.ea[i];
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = nt * kTileN + half * 32 + jj;
                    if (j >= N) continue;
                    double v = P.alpha * ldexp(acc[jj], ei + P.eb[j] - 54);   // acc in units of 2^-40
                    const size_t row = P.c_gather ? (size_t)P.c_gather[i] : (size_t)i;
                    if (P.D) {
                        const size_t di = row * P.ldd + j;
                        v += P.beta * (P.d_f32 ? (double)static_cast<const float*>(P.D)[di]
                                               : static_cast<const double*>(P.D)[di]);
                    }
                    if (P.sub_identity && i == j) v -= 1.0;
                    const size_t ci = row * P.ldc + j;
                    if (P.c_f32)
                        static_cast<float*>(P.C)[ci] = (float)v;
                    else
                        static_cast<double*>(P.C)[ci] = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    if (threadIdx.x == 0 && *abort_flag && P.status) atomicOr(P.status, (int)MPDO_ST_TIMEOUT);
}

// The problems of one kind for every op of a chunk, from the op descriptors.
__global__ void oz_prep_kernel(const OpDesc* descs, int nops, int kind, OzProblem* out, int cap, int bf16) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nops) return;
    const OpDesc& d = descs[s];
    const int ld = 4 * cap;
    OzProblem P{};
    auto rowmajor = [](const void* base, int f32, long long ld_) {   // (r, k) at r * ld + k
        return OzOperand{base, f32, ld_, 1, 0, 1, 1, nullptr};
    };
    auto colmajor = [](const void* base, int f32, long long ld_) {   // (r, k) at k * ld + r
        return OzOperand{base, f32, 1, ld_, 0, 1, 1, nullptr};
    };
    switch (kind) {
        case OZ_MERGE:   // Theta[(l, s1), (s2, r)] = sum_m A[(l, s1), m] B[m, (s2, r)]
            P.M = 4 * d.cl;
            P.K = d.cm;
            P.N = 4 * d.cr;
            P.A = rowmajor(d.A, d.site_f32, cap);
            P.B = OzOperand{d.B, d.site_f32, 0, 0, 1, d.cr, cap, nullptr};
            P.C = d.thetap;
            P.ldc = ld;
            break;
        case OZ_RECON:   // B_p'[(l, s1), j] = sum_c Theta'[(l, s1), c] Yk[j, c], j < k (device)
            P.M = d.m;
            P.K = d.n;
            P.N = min(d.chi_max, d.c);
            P.Ndyn = d.k_out;
            P.A = rowmajor(d.thetap, 0, ld);
            P.B = rowmajor(d.Yk, 0, ld);
            P.C = d.A;
            P.ldc = cap;
            P.c_f32 = d.site_f32;
            break;
        case OZ_E:       // E = U U^T - I
            P.M = P.N = P.K = d.c;
            P.A = rowmajor(d.U32, 1, ld);
            P.B = rowmajor(d.U32, 1, ld);
            P.C = d.E;
            P.ldc = ld;
            P.sub_identity = 1;
            break;
        case OZ_Q:       // Q = U - E U / 2
            P.M = P.N = P.K = d.c;
            P.A = rowmajor(d.E, 0, ld);
            P.B = colmajor(d.U32, 1, ld);
            P.C = d.Q;
            P.ldc = ld;
            P.alpha = -0.5;
            P.beta = 1.0;
            P.D = d.U32;
            P.ldd = ld;
            P.d_f32 = 1;
            break;
        default:         // OZ_W: W = Q W0
            P.M = d.c;
            P.N = d.L;
            P.K = d.c;
            P.A = rowmajor(d.Q, 0, ld);
            P.B = colmajor(d.W0, 0, ld);
            P.C = d.W;
            P.ldc = ld;
            break;
    }
    if (kind != OZ_Q) {
        P.alpha = 1.0;
        P.beta = 0.0;
    }
    P.as = d.oz_as;
    P.bs = d.oz_bs;
    P.ea = d.oz_ea;
    P.eb = d.oz_eb;
    P.status = d.status;
    oz_set_tiles(P, bf16 != 0);
    out[s] = P;
}

// Theta' = G Theta in place (rows (l, s1), columns s2 cr + r) and theta~ =
// lambda_{p-1}[l] Theta' column-major in Acm; one thread per (l, r).
__global__ void __launch_bounds__(256) gate_weight_kernel(const OpDesc* descs, int chi_cap) {
    const OpDesc& d = descs[blockIdx.y];
    __shared__ double Gs[256];
    Gs[threadIdx.x] = d.G[threadIdx.x];
    __syncthreads();
    const int ld = 4 * chi_cap;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.cl * d.cr) return;
    const int l = e / d.cr, r = e % d.cr;
    double th[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) th[i] = d.thetap[(size_t)(l * 4 + (i >> 2)) * ld + (i & 3) * d.cr + r];
    const double lam = d.lam_left ? d.lam_left[l] : 1.0;
#pragma unroll 4
    for (int o = 0; o < 16; ++o) {
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < 16; ++i) v = fma(Gs[o * 16 + i], th[i], v);
        const int row = l * 4 + (o >> 2), col = (o & 3) * d.cr + r;
        d.thetap[(size_t)row * ld + col] = v;
        d.Acm[(size_t)col * ld + row] = lam * v;
    }
}

}  // namespace

cudaError_t launch_oz_ops(const OpDesc* d_desc, int nops, int kind, OzProblem* probs, int chi_cap, bool bf16,
                          unsigned long long timeout_ns, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    oz_prep_kernel<<<(nops + 127) / 128, 128, 0, st>>>(d_desc, nops, kind, probs, chi_cap, bf16 ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int big = 4 * chi_cap;
    return launch_oz_gemm(probs, nops, big, big, big, bf16, timeout_ns, st);
}

cudaError_t launch_gate_weight(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st) {
    if (nops <= 0) return cudaSuccess;
    dim3 g((chi_cap * chi_cap + 255) / 256, nops);
    gate_weight_kernel<<<g, 256, 0, st>>>(d_desc, chi_cap);
    return cudaGetLastError();
}

size_t oz_slice_bytes(int rows, int K, bool bf16) {
    // room for either operand: ceil(rows / 128) tiles of 8 KB cover ceil(rows / 64) of 4 KB
    const int KT = kt_elems(bf16 ? 2 : 4);
    const size_t Rt = (rows + kTileM - 1) / kTileM, Kt = (K + KT - 1) / KT;
    return (size_t)kS * Rt * Kt * kBlockA;
}

size_t oz_exp_ints(int rows) { return (size_t)((rows + kTileM - 1) / kTileM) * kTileM; }

void oz_tiles(OzProblem& p, bool bf16) { oz_set_tiles(p, bf16); }

cudaError_t oz_prepare() {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

cudaError_t launch_oz_gemm(const OzProblem* d_probs, int count, int max_m, int max_n, int max_rows_sliced,
                           bool bf16, unsigned long long timeout_ns, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int mt = (max_m + kTileM - 1) / kTileM, nt = (max_n + kTileN - 1) / kTileN;
    const int rows = ((max_rows_sliced + kTileM - 1) / kTileM) * kTileM;
    dim3 sg((rows + 7) / 8, 2, count);
    if (bf16)
        oz_slice_kernel<true><<<sg, 256, 0, st>>>(d_probs);
    else
        oz_slice_kernel<false><<<sg, 256, 0, st>>>(d_probs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g(nt, mt, count);
    if (bf16)
        oz_gemm_kernel<true><<<g, kThreads, kSmem, st>>>(d_probs, timeout_ns);
    else
        oz_gemm_kernel<false><<<g, kThreads, kSmem, st>>>(d_probs, timeout_ns);
    return cudaGetLastError();
}

namespace {

// problem s of a GemmDesc batch as an OzProblem (one thread per problem)
__global__ void gemm_desc_oz_kernel(const GemmDesc* descs, int count, OzScratch scr, int bf16) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    const GemmDesc& d = descs[s];
    OzProblem P{};
    P.M = d.M;
    P.N = d.N;
    P.K = d.K;
    // A (M x K): stored M x K, or K x M when a_trans
    P.A = d.a_trans ? OzOperand{d.A, d.a_f32, 1, d.lda, 0, 1, 1, nullptr}
                    : OzOperand{d.A, d.a_f32, d.lda, 1, 0, 1, 1, nullptr};
    // column j of B (K x N) as a row of K values: stored K x N, or N x K when b_trans
    P.B = d.b_trans ? OzOperand{d.B, d.b_f32, d.ldb, 1, 0, 1, 1, nullptr}
                    : OzOperand{d.B, d.b_f32, 1, d.ldb, 0, 1, 1, nullptr};
    P.C = d.C;
    P.ldc = d.ldc;
    P.alpha = d.alpha;
    P.beta = d.beta;
    P.D = d.D;
    P.ldd = d.ldd;
    P.d_f32 = d.d_f32;
    P.sub_identity = d.sub_identity;
    P.as = scr.as + (size_t)s * scr.slot_bytes;
    P.bs = scr.bs + (size_t)s * scr.slot_bytes;
    P.ea = scr.ea + (size_t)s * scr.exp_ints;
    P.eb = scr.eb + (size_t)s * scr.exp_ints;
    P.status = d.status;
    oz_set_tiles(P, bf16 != 0);
    scr.probs[s] = P;
}

}  // namespace

cudaError_t launch_gemm_tc(const GemmDesc* d_desc, int count, int max_m, int max_n, int max_k, const OzScratch& scr,
                           bool bf16, unsigned long long timeout_ns, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    // every operand must fit its slot
    const int big = max_m > max_n ? max_m : max_n;
    if (oz_slice_bytes(big, max_k, bf16) > scr.slot_bytes || oz_exp_ints(big) > scr.exp_ints)
        return cudaErrorInvalidValue;
    gemm_desc_oz_kernel<<<(count + 127) / 128, 128, 0, st>>>(d_desc, count, scr, bf16 ? 1 : 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_oz_gemm(scr.probs, count, max_m, max_n, big, bf16, timeout_ns, st);
}

}  // namespace mpdo

// ---------------------------------------------------------------------------
// mpdo_gemm_tc: the same product on caller matrices (include/mpdo.h)
// ---------------------------------------------------------------------------
#include <string>

extern "C" int mpdo_gemm_tc(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                            int ldc, int kind, void* cuda_stream) {
    using namespace mpdo;
    if (M < 1 || N < 1 || K < 1 || lda < K || ldb < N || ldc < N || !A || !B || !C) {
        set_last_error("mpdo_gemm_tc: need M, N, K >= 1, lda >= K, ldb >= N, ldc >= N and non-NULL matrices");
        return MPDO_EINVAL;
    }
    if (kind != MPDO_MIXED_TF32 && kind != MPDO_MIXED_BF16X3) {
        set_last_error("mpdo_gemm_tc: kind must be MPDO_MIXED_TF32 or MPDO_MIXED_BF16X3");
        return MPDO_EINVAL;
    }
    const bool bf16 = kind == MPDO_MIXED_BF16X3;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    OzProblem P{};
    P.M = M;
    P.N = N;
    P.K = K;
    P.A = OzOperand{A, 0, lda, 1, 0, 1, 1, nullptr};
    P.B = OzOperand{B, 0, 1, ldb, 0, 1, 1, nullptr};
    P.C = C;
    P.ldc = ldc;
    P.alpha = 1.0;
    oz_tiles(P, bf16);
    const size_t sa = oz_slice_bytes(M, K, bf16), sb = oz_slice_bytes(N, K, bf16);
    unsigned char* buf = nullptr;
    const size_t ia = oz_exp_ints(M), ib = oz_exp_ints(N);
    const size_t bytes = sa + sb + sizeof(int) * (ia + ib) + sizeof(OzProblem) + 256;
    cudaError_t e = cudaMalloc((void**)&buf, bytes);
    if (e != cudaSuccess) {
        set_last_error(std::string("mpdo_gemm_tc: ") + cudaGetErrorString(e));
        return MPDO_ENOMEM;
    }
    P.as = buf;
    P.bs = buf + sa;
    P.ea = reinterpret_cast<int*>(buf + sa + sb);
    P.eb = P.ea + ia;
    OzProblem* d_p = reinterpret_cast<OzProblem*>(
        (reinterpret_cast<uintptr_t>(P.eb + ib) + 255) & ~static_cast<uintptr_t>(255));
    e = oz_prepare();
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_p, &P, sizeof(P), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_oz_gemm(d_p, 1, M, N, M > N ? M : N, bf16, 4000000000ull, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) {
        set_last_error(std::string("mpdo_gemm_tc: ") + cudaGetErrorString(e));
        return MPDO_ECUDA;
    }
    return MPDO_OK;
}
