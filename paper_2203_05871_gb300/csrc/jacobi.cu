// FP64 one-sided (Hestenes) Jacobi SVD of the bond matrices of one layer.
//
// App. B compresses |rho>> bond by bond from its Schmidt spectrum.  Each op
// hands this kernel c rows of length L (the rows of theta~ when m <= n, or
// its columns when m > n, then with a c x c accumulator Z whose rows turn
// alongside).  Plane rotations from the left make the rows mutually
// orthogonal; row j then equals s_j v_j^T (or Z row j = v_j^T), which the
// truncation step reads.
//
// Block-pair ordering.  The rows are cut into blocks of b rows (b chosen so
// that two blocks, with their Z parts, fit in 128 KB of shared memory).  A
// round-robin ("circle") tournament over the blocks meets every pair of
// blocks once per sweep; in a round each CTA loads one or more block pairs
// into shared memory, rotates every cross pair of rows (and, in the first
// round of a sweep, every pair inside each block), and stores the blocks back
// to their home rows.  The op's CTAs take the block pairs of a sweep from a
// shared counter in round order, and a pair waits only for its two blocks to
// leave the previous round (a version per block); one barrier per sweep.
// Every wait is bounded by a wall-clock limit after which the kernel records
// MPDO_ST_TIMEOUT and returns.  The launch is cooperative (all CTAs resident).
// Within a block pair one warp owns one pair of rows: the inner product is
// reduced with warp shuffles, the rotation is applied in shared memory.
//
// Rotation (Rutishauser): a = |w_p|^2, b = |w_q|^2, g = w_p.w_q,
// zeta = (b - a) / 2g, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// cs = 1/sqrt(1+t^2), sn = cs t;  w_p <- cs w_p - sn w_q, w_q <- sn w_p + cs w_q,
// and then |w_p|^2 = a - t g, |w_q|^2 = b + t g (recomputed from the row when
// the update loses more than 90% of the old value, and at every sweep start).
// A pair is skipped when |g| <= tol sqrt(a b) (tol = sqrt(L) eps unless set):
// kept rows are normalised into singular vectors, so they must be orthogonal
// relative to their own norms.
//
// The same kernel, instantiated for float, is the preconditioning pass of the
// mixed-precision SVD: it orthogonalises an FP32 copy of the rows (scaled to
// unit mean square norm) and accumulates its rotations in U32; the FP64 pass
// then starts from Q W with Q the FP64-orthogonalised U32 (see api.cu).
// A row whose norm is at most eps * ||W||_F (FP64 eps, in both passes) is
// numerically zero: it is set to zero and never rotated (its direction is
// rounding noise).
//
// Further pieces, each described where it is implemented:
//  - FP32 pass on rows of at most 1024 elements: the register path (16 warps,
//    one block of each pair in registers, U32 turned by the block pair's
//    accumulated rotation);
//  - FP64 pass: scaled (fast) rotations, one FMA per element (scaled_rotate);
//  - FP64 pass: pairs of two rows the truncation discards are skipped once the
//    ranking is settled (kth_largest and the sweep-start gate);
//  - convergence: the FP32 pass stops at <= c/4 rotations or a largest rotated
//    off-orthogonality of 1e-3, the FP64 pass at no rotation or a largest
//    rotated rho with rho^2 <= 1e-6 tol.
#include <float.h>
#include <mpdo.h>

#include "coop.cuh"
#include "internal.h"

namespace mpdo {

namespace {

// warps per CTA: the FP32 pass is latency-bound and runs 16 warps (at most 128
// registers each; measured on the chi = 256 chain: 129 ms per step with 8 warps,
// 117 with 12, 104 with 16); the FP64 pass keeps 8 (its blocks of 8 rows feed 8 warps)
template <typename T>
constexpr int kWarps = sizeof(T) == 4 ? 16 : 8;
template <typename T>
constexpr int kThreads = kWarps<T> * 32;
constexpr int kRowBytes = kJacobiRowBytes;             // two blocks of rows in shared memory
constexpr int kMaxB = kJacobiMaxB;
constexpr int kSmemBytes = kRowBytes + 6 * kMaxB * 8;  // rows + norms (2b) + scales (2b) + row ids
constexpr int kSwQueue = 2;   // per-op sync words 2, 3: the block-pair counters of alternate sweeps
constexpr int kSwVer = 8 + 2 * kMaxSweepsCap;   // per-op sync words: one version per row block
static_assert(kSwVer + 4 * kMaxChi <= kSyncWords, "a version for every row block");

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait (thread 0) until row blocks P and Q (those < nb) have left round R - 1,
// i.e. their versions reached R; bounded by timeout_ns, after which the op's
// abort flag is raised.  Returns 0 if it gave up.
__device__ int wait_blocks(const unsigned* ver, int P, int Q, int nb, unsigned R, unsigned* abort_flag,
                           unsigned long long timeout_ns) {
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        const bool okP = P >= nb || ld_acquire(ver + P) >= R;
        const bool okQ = Q >= nb || ld_acquire(ver + Q) >= R;
        if (okP && okQ) return 1;
        if (ld_acquire(abort_flag) != 0u) return 0;
        if (globaltimer_ns() - t0 > timeout_ns) {
            atomicExch(abort_flag, 1u);
            return 0;
        }
        __nanosleep(32);
    }
}
constexpr double kScaleFloor = 0x1p-32;   // FP64 row scales below this are multiplied into the row

__device__ __forceinline__ int tour_player(int x, int step, int cp) {
    return x == 0 ? 0 : 1 + ((x - 1 + step) % (cp - 1));
}

// <x, y> over L elements: lane-strided with four independent accumulators
// (shared-memory latency is hidden by ILP: one CTA of 8 warps per SM)
template <typename T>
__device__ __forceinline__ T row_dot(const T* x, const T* y, int L, int lane) {
    T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int i = lane;
    for (; i + 96 < L; i += 128) {
        const T x0 = x[i], x1 = x[i + 32], x2 = x[i + 64], x3 = x[i + 96];
        const T y0 = y[i], y1 = y[i + 32], y2 = y[i + 64], y3 = y[i + 96];
        s0 = fma(x0, y0, s0);
        s1 = fma(x1, y1, s1);
        s2 = fma(x2, y2, s2);
        s3 = fma(x3, y3, s3);
    }
    for (; i < L; i += 32) s0 = fma(x[i], y[i], s0);
    return warp_sum((s0 + s1) + (s2 + s3));
}

constexpr int kMS = 2 * kMaxB;   // side of a block pair's accumulated rotation (FP32 pass)

template <typename T>
struct Ctx {
    float* M;         // FP32 shared-memory path: the block pair's accumulated rotation [kMS][kMS], else nullptr
    T* rows;          // [2b][rowlen] in shared memory
    T* nrm;           // [2b]
    double* dsc;      // [2b] FP64 pass: the row is dsc times the stored row (scaled rotations)
    int* rid;         // [2b] global row index or -1
    unsigned* rho2;   // largest g^2 / (a b) rotated in this CTA and sweep (float bits)
    int rowlen, L;    // row length in smem (W part + Z part), W part length
    T floor2, tol;
    double thr;       // FP64 pass: pairs of rows whose squared norms are both below thr are skipped
};

// Rotation parameters (cs, sn, t) zeroing <w_p, w_q> = g for |w_p|^2 = a,
// |w_q|^2 = b.  FP64: t is found in FP32 (an inexact angle only slows the
// last digits of convergence), cs = 1/sqrt(1+t^2) is then refined by two
// Newton steps in FP64 so that cs^2 + sn^2 = 1 to FP64 rounding: the rotation
// applied to the rows is orthogonal in FP64.  FP32: computed directly.
__device__ __forceinline__ void rot_params(double a, double b, double g, double& cs, double& sn, double& t) {
    const double r = b - a;
    // scale (r, g) by a power of two so that both fit FP32's range
    const double m = fmax(fabs(r), fabs(g));
    int e = (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1023;
    e = e < -1022 ? -1022 : (e > 1022 ? 1022 : e);
    const double sc = __longlong_as_double((long long)(1023 - e) << 52);
    const float rf = (float)(r * sc), gf = (float)(g * sc);
    const float zeta = rf / (2.0f * gf);
    float tf;
    if (fabsf(zeta) > 1e18f)
        tf = 0.5f / zeta;
    else
        tf = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
    t = (double)tf;
    const double q = fma(t, t, 1.0);
    double c = (double)rsqrtf((float)q);
    c = c * fma(-0.5 * q, c * c, 1.5);
    c = c * fma(-0.5 * q, c * c, 1.5);
    cs = c;
    sn = c * t;
}

__device__ __forceinline__ void rot_params(float a, float b, float g, float& cs, float& sn, float& t) {
    const float zeta = (b - a) / (2.0f * g);
    t = fabsf(zeta) > 1e18f ? 0.5f / zeta : copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
    cs = rsqrtf(fmaf(t, t, 1.0f));
    sn = cs * t;
}

// FP64 rotation on scaled rows (fast plane rotation with dynamic scaling,
// Anda & Park 1994): the rows are w_p = d_p x_p, w_q = d_q x_q, and
//   w_p' = cs w_p - sn w_q = (cs d_p) (x_p - t (d_q / d_p) x_q),
//   w_q' = sn w_p + cs w_q = (cs d_q) (x_q + t (d_p / d_q) x_p),
// so the stored rows take one FMA per element and the factor cs goes to the
// scales.  |t| <= 1, so a scale shrinks by at most 1/sqrt(2) per rotation; a
// scale below 2^-32 is multiplied into its row.  The kernel multiplies every
// row by its scale after the last sweep.
template <typename T>
__device__ int scaled_rotate(const Ctx<T>& C, int p, int q, T* rp, T* rq, double a, double b, double g, double cs,
                             double t, double dp, double dq, int lane) {
    const double al = t * (dq / dp), be = t * (dp / dq);
    int i = lane;
    for (; i + 96 < C.rowlen; i += 128) {
        double x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = rp[i + 32 * u];
            y[u] = rq[i + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            rp[i + 32 * u] = fma(-al, y[u], x[u]);
            rq[i + 32 * u] = fma(be, x[u], y[u]);
        }
    }
    for (; i < C.rowlen; i += 32) {
        const double x = rp[i], y = rq[i];
        rp[i] = fma(-al, y, x);
        rq[i] = fma(be, x, y);
    }
    __syncwarp();
    dp *= cs;
    dq *= cs;
    double na = fma(-t, g, a), nb = fma(t, g, b);
    if (na < 0.1 * a) na = dp * dp * row_dot(rp, rp, C.L, lane);
    if (nb < 0.1 * b) nb = dq * dq * row_dot(rq, rq, C.L, lane);
    if (dp < kScaleFloor) {
        for (int k = lane; k < C.rowlen; k += 32) rp[k] *= dp;
        dp = 1.0;
    }
    if (dq < kScaleFloor) {
        for (int k = lane; k < C.rowlen; k += 32) rq[k] *= dq;
        dq = 1.0;
    }
    __syncwarp();
    if (lane == 0) {
        C.nrm[p] = na;
        C.nrm[q] = nb;
        C.dsc[p] = dp;
        C.dsc[q] = dq;
    }
    __syncwarp();
    return 1;
}

// One warp: rows p, q (shared-memory slots).  Returns 1 if it rotated.
template <typename T>
__device__ int pair_rotate(const Ctx<T>& C, int p, int q, int lane) {
    if (C.rid[p] < 0 || C.rid[q] < 0) return 0;
    if constexpr (sizeof(T) == 8) {
        if (C.nrm[p] < C.thr && C.nrm[q] < C.thr) return 0;   // two rows the truncation discards
    }
    T* rp = C.rows + (size_t)p * C.rowlen;
    T* rq = C.rows + (size_t)q * C.rowlen;
    const T a = C.nrm[p], b = C.nrm[q];
    if (a <= C.floor2 || b <= C.floor2) {
        if (a <= C.floor2 && a != T(0)) {
            for (int i = lane; i < C.L; i += 32) rp[i] = T(0);
            __syncwarp();
            if (lane == 0) C.nrm[p] = T(0);
        }
        if (b <= C.floor2 && b != T(0)) {
            for (int i = lane; i < C.L; i += 32) rq[i] = T(0);
            __syncwarp();
            if (lane == 0) C.nrm[q] = T(0);
        }
        __syncwarp();
        return 0;
    }
    T g = row_dot(rp, rq, C.L, lane);
    if constexpr (sizeof(T) == 8) g *= C.dsc[p] * C.dsc[q];
    // |g| <= tol sqrt(a b), written without squares of squares: in FP32, g^2
    // and a b underflow for rows below ~1e-10 of the largest, and those pairs
    // would pass as converged without ever being rotated
    if constexpr (sizeof(T) == 4) {
        if (g == T(0) || fabsf(g) <= C.tol * sqrtf(a) * sqrtf(b)) return 0;
    } else {
        if (g == T(0) || g * g <= C.tol * C.tol * a * b) return 0;   // no underflow in FP64's range
    }
    T cs, sn, t;
    rot_params(a, b, g, cs, sn, t);
    if (t == T(0)) return 0;
    if (lane == 0) atomicMax(C.rho2, __float_as_uint((float)(g / a * (g / b))));
    if constexpr (sizeof(T) == 8) return scaled_rotate(C, p, q, rp, rq, a, b, g, cs, t, C.dsc[p], C.dsc[q], lane);
    int i = lane;
    for (; i + 96 < C.rowlen; i += 128) {
        T x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[u] = rp[i + 32 * u];
            y[u] = rq[i + 32 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            rp[i + 32 * u] = fma(cs, x[u], -sn * y[u]);
            rq[i + 32 * u] = fma(sn, x[u], cs * y[u]);
        }
    }
    for (; i < C.rowlen; i += 32) {
        const T x = rp[i], y = rq[i];
        rp[i] = fma(cs, x, -sn * y);
        rq[i] = fma(sn, x, cs * y);
    }
    if constexpr (sizeof(T) == 4) {
        if (C.M) {   // the same rotation of rows p, q of the accumulator
            float* mp = C.M + p * kMS;
            float* mq = C.M + q * kMS;
            for (int j = lane; j < kMS; j += 32) {
                const float x = mp[j], y = mq[j];
                mp[j] = fmaf(cs, x, -sn * y);
                mq[j] = fmaf(sn, x, cs * y);
            }
        }
    }
    __syncwarp();
    T na = fma(-t, g, a), nb = fma(t, g, b);
    if (na < T(0.1) * a) na = row_dot(rp, rp, C.L, lane);
    if (nb < T(0.1) * b) nb = row_dot(rq, rq, C.L, lane);
    if (lane == 0) {
        C.nrm[p] = na;
        C.nrm[q] = nb;
    }
    __syncwarp();
    return 1;
}

// All pairs inside each of the two blocks (circle method, first round of a
// sweep only), then all cross pairs between the two blocks.
template <typename T>
__device__ int process_block_pair(const Ctx<T>& C, int b, bool intra, int warp, int lane) {
    int rot = 0;
    if (intra && b > 1) {
        const int bp = b + (b & 1);
        for (int t = 0; t < bp - 1; ++t) {
            for (int x = warp; x < bp; x += kWarps<T>) {   // x < bp/2: block 0, else block 1
                const int blk = x < bp / 2 ? 0 : 1;
                const int y = x % (bp / 2);
                const int P = tour_player(y, t, bp), Q = tour_player(bp - 1 - y, t, bp);
                if (P >= b || Q >= b) continue;
                rot += pair_rotate(C, blk * b + min(P, Q), blk * b + max(P, Q), lane);
            }
            __syncthreads();
        }
    }
    for (int t = 0; t < b; ++t) {
        for (int i = warp; i < b; i += kWarps<T>) rot += pair_rotate(C, i, b + (i + t) % b, lane);
        __syncthreads();
    }
    return rot;
}

// ---------------------------------------------------------------------------
// FP32 pass, register path (W rows of at most kJacobiRegL elements).
//
// A block pair holds 2b <= 64 rows.  Block 0's W rows live in registers (warp w
// of RW = 16 holds slots w and w + RW), block 1's in shared memory.  In cross
// step t warp w meets partner q = (t + w) mod b: it loads that row once,
// rotates it against its own rows in registers and stores it once.  The U32
// rows take no part in the inner products: every rotation of rows (p, q) is
// applied to rows (p, q) of a 64 x 64 accumulator M (identity at the start of
// the block pair), and at the end the 2b U32 rows are replaced by M times
// themselves, one column per thread.  The pass is latency-bound (one CTA per
// SM), hence as many warps as the registers of the rows allow.
//
// Cross rotations act on scaled rows (fast plane rotations with dynamic
// scaling, Anda & Park 1994): row p is d_p x_p, and
//   x_p <- x_p - t (d_q / d_p) x_q,  x_q <- x_q + t (d_p / d_q) x_p,  d <- cs d,
// one FMA per element instead of two multiplies and two FMAs.  The scales
// start at 1 when a block pair is loaded and are multiplied in when it is
// stored; a row meets at most b = 32 partners in between, and cs >= 1/sqrt(2),
// so a scale stays above 2^-16.
constexpr int RW = kWarps<float>;
constexpr int RT = kThreads<float>;
constexpr int kRegL = kJacobiRegL / 32;   // W elements per lane per row
constexpr int kRegRows = (kMaxB + RW - 1) / RW;   // block-0 rows per warp at most
constexpr int kM = 2 * kMaxB;             // accumulator dimension
constexpr int kZT = 128;                  // U32 columns per tile of the accumulator product
constexpr int kSmemReg = kJacobiRegL * kMaxB * 4 + kM * kM * 4 + kM * 12;
constexpr int kSmemSmemF32 = kSmemBytes + kM * kM * 4;   // shared-memory path: rows, norms, ids, M
constexpr int kSmemF32 = kSmemReg > kSmemSmemF32 ? kSmemReg : kSmemSmemF32;
static_assert(kRegRows * RW >= kMaxB, "block 0 must fit the warps' registers");
static_assert(RT == (kM / 4) * (kZT / 4), "one 4 x 4 output tile per thread");
static_assert(kM * kZT + kM * kM <= kJacobiRegL * kMaxB, "U32 tile and M^T fit the rows' space");

struct RegCtx {
    float* rows;      // [b][kJacobiRegL]: the W rows of the block in shared memory, zero past L
    float* M;         // [kM][kM]: accumulated rotation of the block pair's rows (row-major)
    float* nrm;       // [2b]: squared norms (slot s of block k at k b + s)
    float* dsc;       // [b]: scales of block 1's rows during the cross pairs
    int* rid;         // [2b]: global row index or -1
    unsigned* rho2;   // largest g^2 / (a b) rotated in this CTA and sweep (float bits)
    int b, L;
    float floor2, tol;
};

// FP32 rotation parameters with the fast division (the angle only needs FP32
// accuracy; 2g is never above 2^126 since the rows are scaled to unit mean
// square norm)
__device__ __forceinline__ void rot_params_fast(float a, float b, float g, float& cs, float& sn, float& t) {
    const float zeta = __fdividef(b - a, 2.0f * g);
    t = fabsf(zeta) > 1e18f ? __fdividef(0.5f, zeta)
                            : __fdividef(copysignf(1.0f, zeta), fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
    cs = rsqrtf(fmaf(t, t, 1.0f));
    sn = cs * t;
}

__device__ __forceinline__ void rotate_m(const RegCtx& C, int ip, int iq, float cs, float sn, int lane) {
    float* mp = C.M + ip * kM;
    float* mq = C.M + iq * kM;
#pragma unroll
    for (int j = lane; j < kM; j += 32) {
        const float x = mp[j], y = mq[j];
        mp[j] = fmaf(cs, x, -sn * y);
        mq[j] = fmaf(sn, x, cs * y);
    }
}

// U32 rows <- M U32 rows for the 2b rows of a block pair (rid: their global
// rows, -1 for none), in column tiles of kZT staged in shared memory at stage
// (>= kM kZT + kM kM floats, free: the W rows are stored by then): thread
// (rg, cg) of 16 x 32 computes rows 4 rg .. 4 rg + 3 and columns 4 cg ..
// 4 cg + 3 of the tile, reading M^T and the tile as float4.  Called by all
// threads of the CTA.
__device__ void apply_m_u32(const float* M, const int* rid, int n2, float* Z, int ld, int c, float* stage) {
    float* Zt = stage;              // [kM][kZT]
    float* Mt = stage + kM * kZT;   // [kM][kM]: M transposed
    for (int i = threadIdx.x; i < kM * kM; i += RT) Mt[(i % kM) * kM + i / kM] = M[i];
    const int rg = threadIdx.x >> 5, cg = threadIdx.x & 31;
    for (int k0 = 0; k0 < c; k0 += kZT) {
        __syncthreads();
        for (int e = threadIdx.x; e < kM * (kZT / 4); e += RT) {
            const int j = e / (kZT / 4), kk = 4 * (e % (kZT / 4));
            const int row = j < n2 ? rid[j] : -1;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (row >= 0 && k0 + kk < c) v = __ldcg(reinterpret_cast<const float4*>(Z + (size_t)row * ld + k0 + kk));
            *reinterpret_cast<float4*>(Zt + j * kZT + kk) = v;
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) acc[ii][kk] = 0.0f;
#pragma unroll 4
        for (int j = 0; j < n2; ++j) {
            const float4 m = *reinterpret_cast<const float4*>(Mt + j * kM + 4 * rg);
            const float4 z = *reinterpret_cast<const float4*>(Zt + j * kZT + 4 * cg);
            const float mv[4] = {m.x, m.y, m.z, m.w}, zv[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) acc[ii][kk] = fmaf(mv[ii], zv[kk], acc[ii][kk]);
        }
        const int k = k0 + 4 * cg;
#pragma unroll
        for (int ii = 0; ii < 4; ++ii) {
            const int i = 4 * rg + ii;
            const int row = i < n2 ? rid[i] : -1;
            if (row >= 0 && k < c)
                __stcg(reinterpret_cast<float4*>(Z + (size_t)row * ld + k),
                       make_float4(acc[ii][0], acc[ii][1], acc[ii][2], acc[ii][3]));
        }
    }
}

// One warp: shared-memory slots p < q of the block whose rows sit at
// accumulator offset mo (plain rotations).  Returns 1 if it rotated.
__device__ int intra_pair_reg(const RegCtx& C, int p, int q, int mo, int lane) {
    const int ip = mo + p, iq = mo + q;
    if (C.rid[ip] < 0 || C.rid[iq] < 0) return 0;
    float* rp = C.rows + (size_t)p * kJacobiRegL;
    float* rq = C.rows + (size_t)q * kJacobiRegL;
    const float a = C.nrm[ip], b = C.nrm[iq];
    if (a <= C.floor2 || b <= C.floor2) {
        if (a <= C.floor2 && a != 0.0f) {
            for (int i = lane; i < C.L; i += 32) rp[i] = 0.0f;
            __syncwarp();
            if (lane == 0) C.nrm[ip] = 0.0f;
        }
        if (b <= C.floor2 && b != 0.0f) {
            for (int i = lane; i < C.L; i += 32) rq[i] = 0.0f;
            __syncwarp();
            if (lane == 0) C.nrm[iq] = 0.0f;
        }
        __syncwarp();
        return 0;
    }
    const float g = row_dot(rp, rq, C.L, lane);
    if (g == 0.0f || fabsf(g) <= C.tol * sqrtf(a) * sqrtf(b)) return 0;
    float cs, sn, t;
    rot_params_fast(a, b, g, cs, sn, t);
    if (t == 0.0f) return 0;
    if (lane == 0) atomicMax(C.rho2, __float_as_uint(g / a * (g / b)));
    for (int i = lane; i < C.L; i += 32) {
        const float x = rp[i], y = rq[i];
        rp[i] = fmaf(cs, x, -sn * y);
        rq[i] = fmaf(sn, x, cs * y);
    }
    rotate_m(C, ip, iq, cs, sn, lane);
    __syncwarp();
    float na = fmaf(-t, g, a), nb = fmaf(t, g, b);
    if (na < 0.1f * a) na = row_dot(rp, rp, C.L, lane);
    if (nb < 0.1f * b) nb = row_dot(rq, rq, C.L, lane);
    if (lane == 0) {
        C.nrm[ip] = na;
        C.nrm[iq] = nb;
    }
    __syncwarp();
    return 1;
}

// All pairs inside the block held in shared memory (circle method).
__device__ int intra_block_reg(const RegCtx& C, int mo, int warp, int lane) {
    const int b = C.b;
    if (b < 2) return 0;
    int rot = 0;
    const int bp = b + (b & 1);
    for (int t = 0; t < bp - 1; ++t) {
        for (int x = warp; x < bp / 2; x += RW) {
            const int P = tour_player(x, t, bp), Q = tour_player(bp - 1 - x, t, bp);
            if (P >= b || Q >= b) continue;
            rot += intra_pair_reg(C, min(P, Q), max(P, Q), mo, lane);
        }
        __syncthreads();
    }
    return rot;
}

// W rows of accumulator slots s0 .. s0 + b - 1 into the shared-memory rows,
// zero-padded to kJacobiRegL (the padding stays zero under every rotation, so
// the register loops need no bound on the row length)
__device__ __forceinline__ void load_block_reg(const RegCtx& C, const float* W, int ld, int s0, int warp, int lane) {
    for (int s = warp; s < C.b; s += RW) {
        const int row = C.rid[s0 + s];
        float* dst = C.rows + (size_t)s * kJacobiRegL;
        if (row < 0) {
            for (int k = lane; k < kJacobiRegL; k += 32) dst[k] = 0.0f;
            continue;
        }
        const float* w = W + (size_t)row * ld;
        for (int k = lane; k < kJacobiRegL; k += 32) dst[k] = k < C.L ? __ldcg(w + k) : 0.0f;
    }
}

// One block pair of the register path: load, intra pairs (first round of a
// sweep), cross pairs, store, U32 update.  Returns this warp's rotations.
__device__ int block_pair_reg(const RegCtx& C, float* W, float* Z, int ld, int c, int nb, const int bl[2],
                              bool intra, double* snorm, int warp, int lane) {
    __shared__ int s_any;
    const int b = C.b, L = C.L;
    int rot = 0;
    for (int i = threadIdx.x; i < kM * kM; i += RT) C.M[i] = (i / kM == i % kM) ? 1.0f : 0.0f;
    if (threadIdx.x == 0) s_any = 0;
    if (threadIdx.x < 2 * b) {
        const int s = threadIdx.x;
        const int blk = bl[s / b];
        const int row = blk * b + (s % b);
        const bool ok = blk < nb && row < c;
        C.rid[s] = ok ? row : -1;
        C.nrm[s] = ok ? (float)__ldcg(snorm + row) : 0.0f;
        if (s < b) C.dsc[s] = 1.0f;
    }
    __syncthreads();
    // block 0 through shared memory into registers
    load_block_reg(C, W, ld, 0, warp, lane);
    __syncthreads();
    if (intra) rot += intra_block_reg(C, 0, warp, lane);
    float x[kRegRows][kRegL];
    float ar[kRegRows], dx[kRegRows];
#pragma unroll
    for (int r = 0; r < kRegRows; ++r) {
        const int s = r * RW + warp;
        const bool own = s < b && C.rid[s] >= 0;
        ar[r] = own ? C.nrm[s] : 0.0f;
        dx[r] = 1.0f;
#pragma unroll
        for (int u = 0; u < kRegL; ++u) x[r][u] = own ? C.rows[(size_t)s * kJacobiRegL + u * 32 + lane] : 0.0f;
    }
    __syncthreads();
    // block 1 into shared memory
    load_block_reg(C, W, ld, b, warp, lane);
    __syncthreads();
    if (intra) rot += intra_block_reg(C, b, warp, lane);
    // cross pairs: at step t the warps meet distinct partners q = (t + warp) mod b
    for (int t = 0; t < b; ++t) {
        const int q = (t + warp) % b;
        if (warp < b && C.rid[b + q] >= 0) {
            float* rq = C.rows + (size_t)q * kJacobiRegL;
            float y[kRegL];
#pragma unroll
            for (int u = 0; u < kRegL; ++u) y[u] = rq[u * 32 + lane];
            float bq = C.nrm[b + q], dy = C.dsc[q];
            bool ymod = false;
#pragma unroll
            for (int r = 0; r < kRegRows; ++r) {
                const int s = r * RW + warp;
                if (s >= b || C.rid[s] < 0) continue;
                const float a = ar[r];
                if (a <= C.floor2 || bq <= C.floor2) {
                    if (a <= C.floor2 && a != 0.0f) {
#pragma unroll
                        for (int u = 0; u < kRegL; ++u) x[r][u] = 0.0f;
                        ar[r] = 0.0f;
                        dx[r] = 1.0f;
                    }
                    if (bq <= C.floor2 && bq != 0.0f) {
#pragma unroll
                        for (int u = 0; u < kRegL; ++u) y[u] = 0.0f;
                        bq = 0.0f;
                        dy = 1.0f;
                        ymod = true;
                    }
                    continue;
                }
                float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, g3 = 0.0f;
#pragma unroll
                for (int u = 0; u < kRegL; u += 4) {
                    g0 = fmaf(x[r][u], y[u], g0);
                    g1 = fmaf(x[r][u + 1], y[u + 1], g1);
                    g2 = fmaf(x[r][u + 2], y[u + 2], g2);
                    g3 = fmaf(x[r][u + 3], y[u + 3], g3);
                }
                const float g = warp_sum((g0 + g1) + (g2 + g3)) * (dx[r] * dy);
                if (g == 0.0f || fabsf(g) <= C.tol * sqrtf(a) * sqrtf(bq)) continue;
                float cs, sn, tt;
                rot_params_fast(a, bq, g, cs, sn, tt);
                if (tt == 0.0f) continue;
                if (lane == 0) atomicMax(C.rho2, __float_as_uint(g / a * (g / bq)));
                const float ratio = __fdividef(dy, dx[r]);
                const float al = tt * ratio, be = __fdividef(tt, ratio);
#pragma unroll
                for (int u = 0; u < kRegL; ++u) {
                    const float xv = x[r][u], yv = y[u];
                    x[r][u] = fmaf(-al, yv, xv);
                    y[u] = fmaf(be, xv, yv);
                }
                rotate_m(C, s, b + q, cs, sn, lane);
                dx[r] *= cs;
                dy *= cs;
                float na = fmaf(-tt, g, a), nq = fmaf(tt, g, bq);
                if (na < 0.1f * a) {
                    float s0 = 0.0f;
#pragma unroll
                    for (int u = 0; u < kRegL; ++u) s0 = fmaf(x[r][u], x[r][u], s0);
                    na = warp_sum(s0) * (dx[r] * dx[r]);
                }
                if (nq < 0.1f * bq) {
                    float s0 = 0.0f;
#pragma unroll
                    for (int u = 0; u < kRegL; ++u) s0 = fmaf(y[u], y[u], s0);
                    nq = warp_sum(s0) * (dy * dy);
                }
                ar[r] = na;
                bq = nq;
                ymod = true;
                ++rot;
            }
            if (ymod) {
#pragma unroll
                for (int u = 0; u < kRegL; ++u) rq[u * 32 + lane] = y[u];
                __syncwarp();
                if (lane == 0) {
                    C.nrm[b + q] = bq;
                    C.dsc[q] = dy;
                }
            }
        }
        __syncthreads();
    }
    // store: block 0 from registers, block 1 from shared memory, scales multiplied in
#pragma unroll
    for (int r = 0; r < kRegRows; ++r) {
        const int s = r * RW + warp;
        if (s >= b || C.rid[s] < 0) continue;
        float* w = W + (size_t)C.rid[s] * ld;
#pragma unroll
        for (int u = 0; u < kRegL; ++u) {
            const int e = u * 32 + lane;
            if (e < L) __stcg(w + e, x[r][u] * dx[r]);
        }
        if (lane == 0) __stcg(snorm + C.rid[s], (double)ar[r]);
    }
    for (int s = warp; s < b; s += RW) {
        const int row = C.rid[b + s];
        if (row < 0) continue;
        const float* src = C.rows + (size_t)s * kJacobiRegL;
        const float dv = C.dsc[s];
        float* w = W + (size_t)row * ld;
        for (int k = lane; k < L; k += 32) __stcg(w + k, src[k] * dv);
        if (lane == 0) __stcg(snorm + row, (double)C.nrm[b + s]);
    }
    if (lane == 0 && rot > 0) atomicOr(&s_any, 1);
    __syncthreads();
    if (s_any) apply_m_u32(C.M, C.rid, 2 * b, Z, ld, c, C.rows);
    __syncthreads();
    return rot;
}

// The kk-th largest of v[0..c) (non-negative), by bisection on the bit
// pattern (non-negative doubles order like their bits).  Called by every
// thread of a CTA of kThreads<double>; every thread returns the same value.
constexpr int kSelPer = (4 * kMaxChi + kThreads<double> - 1) / kThreads<double>;
__device__ double kth_largest(const double* v, int c, int kk) {
    __shared__ int s_cnt[kWarps<double>];
    unsigned long long key[kSelPer];
#pragma unroll
    for (int i = 0; i < kSelPer; ++i) {
        const int j = threadIdx.x + i * kThreads<double>;
        key[i] = j < c ? (unsigned long long)__double_as_longlong(fmax(__ldcg(v + j), 0.0)) : 0ull;
    }
    unsigned long long x = 0ull;
    for (int bit = 62; bit >= 0; --bit) {
        const unsigned long long cand = x | (1ull << bit);
        int n = 0;
#pragma unroll
        for (int i = 0; i < kSelPer; ++i) n += key[i] >= cand;
        n = __reduce_add_sync(0xffffffffu, n);
        if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = n;
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps<double>; ++w) tot += s_cnt[w];
        __syncthreads();
        if (tot >= kk) x = cand;
    }
    return __longlong_as_double((long long)x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads<T>, 1) jacobi_kernel(const OpDesc* descs, const int* cta_op, const int* cta_rank,
                                                       const int* group, unsigned* sync, int max_sweeps,
                                                       double tol_in, unsigned long long timeout_ns, int ld,
                                                       float pre_rho2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kF32 = sizeof(T) == 4;
    const int op = cta_op[blockIdx.x];
    if (op < 0) return;   // a CTA the plan left unused (graph step)
    const int g = cta_rank[blockIdx.x];
    const int G = group[op];
    const OpDesc& d = descs[op];
    unsigned* sw = sync + (size_t)op * kSyncWords;
    const int c = d.c, L = d.L;
    int b = kF32 ? d.jb32 : d.jb;
    T* W;
    T* Z;
    if constexpr (kF32) {
        W = d.W32;
        Z = d.U32;
    } else {
        W = d.W;
        Z = d.transposed ? d.Z : nullptr;
    }
    const int zl = (!kF32 && Z) ? c : 0;   // FP32: U32 is turned per block pair, not staged
    // a block size that does not fit shared memory (or the registers) is a
    // planning error: every CTA of the op sees it and returns at once
    if (b < 1 || b > kMaxB ||
        ((!kF32 || !jacobi_f32_reg(L)) && (size_t)2 * b * (L + zl) * sizeof(T) > (size_t)kRowBytes)) {
        if (threadIdx.x == 0) atomicOr(d.status, (int)MPDO_ST_CAPACITY);
        return;
    }
    // the same value, read again so that the range the check proves does not
    // reach the register allocation of the FP32 paths (it made them spill)
    b = *(volatile const int*)(kF32 ? &d.jb32 : &d.jb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned gen = 0;
    __shared__ double s_floor2, s_scale;
    __shared__ int s_conv;
    __shared__ unsigned s_rho2;
    __shared__ int s_pair;

    Ctx<T> C;
    C.rowlen = L + zl;
    C.L = L;
    C.rows = reinterpret_cast<T*>(smem_raw);
    // the per-row data at a fixed offset past the rows' budget: the FP32
    // path's U32 update stages its tiles over the rows (48 KB)
    C.nrm = reinterpret_cast<T*>(smem_raw + kRowBytes);
    C.M = (kF32 && !jacobi_f32_reg(L)) ? reinterpret_cast<float*>(smem_raw + kSmemBytes) : nullptr;
    C.dsc = reinterpret_cast<double*>(C.nrm + 2 * b);
    C.rid = reinterpret_cast<int*>(C.dsc + 2 * b);
    double* dscale = d.snorm + ld;   // FP64 pass: per-row scales (the QR's column norms are dead here)
    C.rho2 = &s_rho2;
    C.thr = 0.0;
    float rho2_stop;
    {
        const double eps = kF32 ? (double)FLT_EPSILON : DBL_EPSILON;
        const double tol = tol_in > 0.0 ? tol_in : sqrt((double)(L > 1 ? L : 1)) * eps;
        C.tol = (T)tol;
        rho2_stop = (float)(1e-6 * tol);
    }

    if (kF32 && g == 0 && threadIdx.x == 0 && d.pre_ok) *d.pre_ok = 0;   // set again only on success
    // squared row norms of the FP64 input (for the zero floor and the FP32 scale)
    const double* W64 = kF32 ? d.W0 : d.W;
    for (int row = g * kWarps<T> + warp; row < c; row += G * kWarps<T>) {
        const double* w = W64 + (size_t)row * ld;
        double a = 0.0;
        for (int i = lane; i < L; i += 32) {
            const double x = __ldcg(w + i);
            a = fma(x, x, a);
        }
        a = warp_sum(a);
        if (lane == 0) {
            __stcg(d.snorm + row, a);
            if constexpr (!kF32) __stcg(dscale + row, 1.0);
        }
    }
    if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int j = 0; j < c; ++j) f += __ldcg(d.snorm + j);
        // numerical zero of the FP64 data in both passes: the FP32 copy of a row
        // far below eps32 ||W|| is still accurate relative to its own norm (the
        // rows of R are graded), so the preconditioning pass must rotate it too
        s_floor2 = DBL_EPSILON * DBL_EPSILON * f;
        s_scale = f > 0.0 ? sqrt((double)c / f) : 1.0;   // FP32 pass: rows of unit mean square norm
    }
    __syncthreads();
    // initial Z (identity, or Zinit) and, for the FP32 pass, the scaled copy of the rows
    for (int row = g * kWarps<T> + warp; row < c; row += G * kWarps<T>) {
        if (Z) {
            bool copied = false;
            if constexpr (!kF32) {
                if (d.Zinit) {
                    for (int i = lane; i < c; i += 32) __stcg(Z + (size_t)row * ld + i, __ldcg(d.Zinit + (size_t)row * ld + i));
                    copied = true;
                }
            }
            if (!copied)
                for (int i = lane; i < c; i += 32) Z[(size_t)row * ld + i] = (i == row) ? T(1) : T(0);
        }
        if constexpr (kF32) {
            const double sc = s_scale;
            for (int i = lane; i < L; i += 32) W[(size_t)row * ld + i] = (float)(__ldcg(d.W0 + (size_t)row * ld + i) * sc);
        }
    }
    C.floor2 = (T)(kF32 ? s_floor2 * s_scale * s_scale : s_floor2);
    if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
    {
        const bool reg = kF32 && jacobi_f32_reg(L);
        RegCtx RC;
        RC.rows = reinterpret_cast<float*>(smem_raw);
        RC.M = reinterpret_cast<float*>(smem_raw + (size_t)kJacobiRegL * kMaxB * 4);
        RC.nrm = RC.M + kM * kM;
        RC.dsc = RC.nrm + kM;
        RC.rid = reinterpret_cast<int*>(RC.dsc + kM / 2);
        RC.rho2 = &s_rho2;
        RC.b = b;
        RC.L = L;
        RC.floor2 = (float)C.floor2;
        RC.tol = (float)C.tol;
        const int nb = (c + b - 1) / b;
        const int nbp = nb + (nb & 1);
        const int npair = nbp / 2;
        const int sweeps = max_sweeps < kMaxSweepsCap ? max_sweeps : kMaxSweepsCap;
        int conv = (c <= 1);
        int used = 0;
        for (int sweep = 0; sweep < sweeps && !conv; ++sweep) {
            int rot = 0;
            if (threadIdx.x == 0) s_rho2 = 0u;
            // fresh squared row norms, then the tail threshold (same in every CTA)
            for (int row = g * kWarps<T> + warp; row < c; row += G * kWarps<T>) {
                const T* w = W + (size_t)row * ld;
                T a = 0;
                for (int i = lane; i < L; i += 32) {
                    const T x = __ldcg(w + i);
                    a = fma(x, x, a);
                }
                a = warp_sum(a);
                if constexpr (!kF32) {
                    const double dv = __ldcg(dscale + row);
                    a = a * dv * dv;
                }
                if (lane == 0) __stcg(d.snorm + row, (double)a);
            }
            if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
            if constexpr (!kF32) {
                // Rows the truncation discards (below the chi_max + max(16, chi_max / 8)
                // largest) must end orthogonal to the kept rows, not to one another:
                // the kept rows are then exact singular vectors, the discarded weight
                // is the sum of the discarded rows' squared norms (a trace), and
                // rows already orthogonal to ~1e-4 have norms equal to their singular
                // values to ~1e-8, far finer than the margin.  So once the previous
                // sweep rotated by at most 1e-4, pairs of two discarded rows are skipped.
                // The first sweep after the FP32 preconditioner qualifies too when that
                // pass ended by its off-orthogonality rule (every pair at ~1e-6 then).
                if (threadIdx.x == 0) {
                    const int kk = d.chi_max + max(16, d.chi_max / 8);
                    const bool settled = sweep > 0
                                             ? __uint_as_float(ld_acquire(&sw[8 + kMaxSweepsCap + sweep - 1])) <= 1e-8f
                                             : (d.pre_ok && __ldcg(d.pre_ok) == 1);
                    s_conv = settled && !d.full_svd && kk < c;
                }
                __syncthreads();
                // the threshold is fixed when the gate first opens, so that a row
                // near it keeps its side (a row changing side later would bring its
                // unprocessed pairs back and cost another sweep)
                if (s_conv && C.thr == 0.0) C.thr = kth_largest(d.snorm, c, d.chi_max + max(16, d.chi_max / 8));
                __syncthreads();
            }
            // The block pairs of a sweep go to the op's CTAs through a shared
            // counter (position q: round q / npair, pair q % npair), and a round
            // has no barrier: a pair waits only until its two blocks have left
            // the previous round (a version per block).  A CTA whose pairs are
            // cheap (both blocks discarded, or already orthogonal) takes more of
            // them, and a round starts where its blocks are ready.  Positions are
            // taken in order, so the pairs a CTA waits for are held by CTAs that
            // can progress.  Two counters alternate by sweep; the next one is
            // cleared during this sweep (every CTA is past its last use).
            if (g == 0 && threadIdx.x == 0) atomicExch(&sw[kSwQueue + ((sweep + 1) & 1)], 0u);
            for (;;) {
                if (threadIdx.x == 0) s_pair = (int)atomicAdd(&sw[kSwQueue + (sweep & 1)], 1u);
                __syncthreads();
                const int qpos = s_pair;
                __syncthreads();   // read by all before thread 0 takes the next one
                if (qpos >= (nbp - 1) * npair) break;
                const int r = qpos / npair, i = qpos % npair;
                const int P = tour_player(i, r, nbp), Q = tour_player(nbp - 1 - i, r, nbp);
                const unsigned R = (unsigned)(sweep * (nbp - 1) + r);   // rounds of this launch before
                if (threadIdx.x == 0) s_conv = wait_blocks(sw + kSwVer, P, Q, nb, R, &sw[1], timeout_ns);
                __syncthreads();
                if (!s_conv) goto timeout;
                const int bl[2] = {P < Q ? P : Q, P < Q ? Q : P};
                do {
                    if constexpr (kF32) {
                        if (reg) {
                            rot += block_pair_reg(RC, W, Z, ld, c, nb, bl, r == 0, d.snorm, warp, lane);
                            break;
                        }
                    }
                    if constexpr (!kF32) {   // both blocks discarded: nothing to do
                        int pred = 1;
                        if (threadIdx.x < 2 * b) {
                            const int blk = bl[threadIdx.x / b];
                            const int row = blk * b + (threadIdx.x % b);
                            if (blk < nb && row < c) pred = __ldcg(d.snorm + row) < C.thr;
                        }
                        if (__syncthreads_and(pred)) break;
                    }
                    // load the two blocks (slot s < b: block bl[0]; s >= b: block bl[1])
                    for (int s = warp; s < 2 * b; s += kWarps<T>) {
                        const int blk = bl[s / b];
                        const int row = blk * b + (s % b);
                        const bool ok = blk < nb && row < c;
                        T* dst = C.rows + (size_t)s * C.rowlen;
                        if (ok) {
                            const T* w = W + (size_t)row * ld;
                            for (int k = lane; k < L; k += 32) dst[k] = __ldcg(w + k);
                            if (zl)
                                for (int k = lane; k < c; k += 32) dst[L + k] = __ldcg(Z + (size_t)row * ld + k);
                            __syncwarp();
                            const T nv = (T)__ldcg(d.snorm + row);
                            if (lane == 0) {
                                C.nrm[s] = nv;
                                if constexpr (!kF32) C.dsc[s] = __ldcg(dscale + row);
                                C.rid[s] = row;
                            }
                        } else if (lane == 0) {
                            C.nrm[s] = T(0);
                            if constexpr (!kF32) C.dsc[s] = 1.0;
                            C.rid[s] = -1;
                        }
                    }
                    if (C.M)   // FP32 shared-memory path: the block pair's rotation starts at I
                        for (int e = threadIdx.x; e < kMS * kMS; e += blockDim.x)
                            C.M[e] = (e / kMS == e % kMS) ? 1.0f : 0.0f;
                    __syncthreads();
                    const int rot_bp = process_block_pair(C, b, r == 0, warp, lane);
                    rot += rot_bp;
                    // store back
                    for (int s = warp; s < 2 * b; s += kWarps<T>) {
                        const int row = C.rid[s];
                        if (row < 0) continue;
                        const T* src = C.rows + (size_t)s * C.rowlen;
                        T* w = W + (size_t)row * ld;
                        for (int k = lane; k < L; k += 32) __stcg(w + k, src[k]);
                        if (zl)
                            for (int k = lane; k < c; k += 32) __stcg(Z + (size_t)row * ld + k, src[L + k]);
                        if (lane == 0) {
                            __stcg(d.snorm + row, (double)C.nrm[s]);
                            if constexpr (!kF32) __stcg(dscale + row, C.dsc[s]);
                        }
                    }
                    if constexpr (kF32) {   // U32 rows of the pair turned by the accumulated rotation
                        if (C.M && __syncthreads_or(rot_bp > 0))
                            apply_m_u32(C.M, C.rid, 2 * b, Z, ld, c, reinterpret_cast<float*>(C.rows));
                    }
                    __syncthreads();
                } while (false);
                // the pair's rows (and U32 rows) are stored: its blocks leave round r
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) {
                    if (P < nb) st_release(&sw[kSwVer + P], R + 1);
                    if (Q < nb) st_release(&sw[kSwVer + Q], R + 1);
                }
            }
            if (lane == 0 && rot > 0) atomicAdd(&sw[8 + sweep], (unsigned)rot);
            __syncthreads();
            if (threadIdx.x == 0 && s_rho2) atomicMax(&sw[8 + kMaxSweepsCap + sweep], s_rho2);
            if (!op_barrier(sw, G, gen, timeout_ns)) goto timeout;
            // FP32 pass: done when fewer than c/4 pairs still rotate (a few pairs
            // sit at FP32's resolution forever; the FP64 pass finishes them), or
            // when the largest relative off-orthogonality rotated away was at most
            // pre_rho (default 1e-3): the rows are then orthogonal to ~pre_rho^2,
            // near FP32's rounding level for these inner products, and further
            // sweeps only chase rounding.
            // FP64: no rotation, or the largest rotated rho had rho^2 <= 1e-6 tol: by
            // quadratic convergence the next sweep would meet pairs at ~rho^2, far
            // under tol, and rotate nothing (1e-20 for tol = sqrt(L) eps at L = 1024)
            if (threadIdx.x == 0)
                s_conv = (ld_acquire(&sw[8 + sweep]) <= (kF32 ? (unsigned)(c / 4) : 0u)) ||
                         (__uint_as_float(ld_acquire(&sw[8 + kMaxSweepsCap + sweep])) <= (kF32 ? pre_rho2 : rho2_stop));
            __syncthreads();
            conv = s_conv;
            used = sweep + 1;
        }
        if constexpr (!kF32) {   // rows out of their scales (the last round ended with a barrier)
            for (int row = g * kWarps<T> + warp; row < c; row += G * kWarps<T>) {
                const double dv = __ldcg(dscale + row);
                if (dv == 1.0) continue;
                T* w = W + (size_t)row * ld;
                for (int i = lane; i < L; i += 32) __stcg(w + i, __ldcg(w + i) * dv);
                if (Z)
                    for (int i = lane; i < c; i += 32) __stcg(Z + (size_t)row * ld + i, __ldcg(Z + (size_t)row * ld + i) * dv);
            }
        }
        if (g == 0 && threadIdx.x == 0) {
            if (!kF32) {
                if (d.sweeps_out) *d.sweeps_out += used;
                if (!conv) atomicOr(d.status, (int)MPDO_ST_NOCONV);
            } else {
                if (d.sweeps_out) *d.sweeps_out += used << 16;   // FP32 sweeps in the high half
                if (d.pre_ok)
                    *d.pre_ok = used > 0 && __uint_as_float(ld_acquire(&sw[8 + kMaxSweepsCap + used - 1])) <= pre_rho2;
            }
        }
    }
    return;
timeout:
    if (threadIdx.x == 0) atomicOr(d.status, (int)MPDO_ST_TIMEOUT);
}

}  // namespace

size_t jacobi_sync_words_per_op() { return kSyncWords; }
size_t jacobi_sync_words(int nops) { return (size_t)nops * kSyncWords; }


cudaError_t jacobi_max_resident(int* blocks) {
    int dev = 0, sms = 0, per64 = 0, per32 = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(jacobi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(jacobi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemF32)) !=
        cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per64, jacobi_kernel<double>, kThreads<double>, kSmemBytes)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per32, jacobi_kernel<float>, kThreads<float>, kSmemF32)) != cudaSuccess)
        return e;
    *blocks = sms * (per64 < per32 ? per64 : per32);
    return cudaSuccess;
}

cudaError_t launch_jacobi(const OpDesc* d_desc, int nops, const int* d_cta_op, const int* d_cta_rank,
                          const int* d_group, unsigned* d_sync, int grid, int max_sweeps, double tol,
                          unsigned long long timeout_ns, int ld, bool fp32, cudaStream_t st, double pre_rho) {
    (void)nops;
    if (grid <= 0) return cudaSuccess;
    float pre_rho2 = (float)(pre_rho * pre_rho);
    void* args[] = {(void*)&d_desc, (void*)&d_cta_op, (void*)&d_cta_rank, (void*)&d_group, (void*)&d_sync,
                    (void*)&max_sweeps, (void*)&tol, (void*)&timeout_ns, (void*)&ld, (void*)&pre_rho2};
    const void* fn = fp32 ? (const void*)jacobi_kernel<float> : (const void*)jacobi_kernel<double>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(fp32 ? kThreads<float> : kThreads<double>), args,
                                       fp32 ? kSmemF32 : kSmemBytes, st);
}

}  // namespace mpdo
