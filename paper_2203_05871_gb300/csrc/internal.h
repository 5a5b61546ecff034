// Internal declarations shared by the libmpdo translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace mpdo {

constexpr int kMaxChi = 512;          // chi_cap upper bound (config: N=40 grid at chi=512)
constexpr int kMaxSweepsCap = 128;    // size of the per-op rotation-counter array

// ---------------------------------------------------------------------------
// Trotter schedule (host).  One op acts on path positions (p, p+1).
// ---------------------------------------------------------------------------
struct Op {
    int kind;      // 0 = gate, 1 = swap
    int p;         // left path position
    int qa, qb;    // qubits at p and p+1 before the op
    int bond;      // bond index (gates), -1 for swaps
    double frac;   // fraction of dt (gates), 0 for swaps
};
using Layer = std::vector<Op>;

// Sets the message returned by mpdo_last_error() on this thread.
void set_last_error(const std::string& msg);

// Builds the layers of one second-order step; returns "" or an error message.
std::string build_schedule(int n, const std::vector<int>& bi, const std::vector<int>& bj,
                           std::vector<Layer>& layers, std::vector<double>& weights);

// ---------------------------------------------------------------------------
// Per-op descriptor of one two-site update, filled by the host per layer.
// All pointers are device pointers.  Matrices in the workspace are row-major
// with leading dimension ld = 4 * chi_cap.
// ---------------------------------------------------------------------------
struct OpDesc {
    int b;             // instance
    int op;            // op index within the step (for the rank log)
    int p;             // left path position
    int cl, cm, cr;    // bond dims chi_{p-1}, chi_p, chi_{p+1}
    int m, n;          // 4*cl, 4*cr
    int transposed;    // 1: Jacobi rows carry a c x c accumulator Z (unused since the QR step)
    int c, L;          // Jacobi problem: c rows of length L
    int jb;            // Jacobi block size (rows per shared-memory block), FP64 pass
    int jb32;          // same for the FP32 preconditioning pass
    int chi_max;
    double cutoff;
    const double* G;   // 16x16 gate, row-major G[(s1' s2'), (s1 s2)]
    void* A;           // site p    [cl][4][chi_cap] (double, or float when site_f32)
    void* B;           // site p+1  [cm][4][chi_cap]
    int site_f32;      // site tensors stored as float (MPDO_STORE_F32)
    const double* lam_left;  // lambda_{p-1} (nullptr => 1)
    double* lam_out;   // lambda_p
    double* thetap;    // Theta'  m x n (ld)
    double* Acm;       // theta~ column-major (column k at Acm + k*ld), input of the QR
    double* W0;        // rows of R from the QR (== W in the FP64 path)
    double* W;         // Jacobi rows: theta~ (m x n) or theta~^T (n x m)
    double* Z;         // c x c rotation accumulator when transposed
    const double* Zinit;  // initial Z (nullptr => identity)
    float* W32;        // mixed path: FP32 rows of the preconditioning Jacobi (c x L)
    float* U32;        // mixed path: FP32 accumulated rotations (c x c)
    double* E;         // mixed path: U32 U32^T - I (c x c)
    double* Q;         // mixed path: orthogonalised U32 (c x c)
    double* Yk;        // k x n right singular vectors (rows), ld
    double* snorm;     // 2*ld doubles of scratch: row norms (Jacobi), R diagonal and column norms (QR)
    int* k_out;        // new chi_p
    int* status;       // per-instance status word
    double* max_disc;  // per-instance max discarded weight
    int* rank_log;     // &log[b][step*n_ops + op] or nullptr
    int* sweeps_out;   // Jacobi sweeps used (or nullptr)
    int* pre_ok;       // mixed path: 1 when the FP32 pass ended with every pair orthogonal to ~1e-6
                       // (its last sweep rotated by at most 1e-3); written by that pass, read by
                       // the FP64 pass (or nullptr)
    int forced_k;      // > 0: truncation rank imposed (replay of a recorded run)
    int full_svd;      // 1: orthogonalise every pair of rows (the adjoint needs all singular vectors)
    double* tape_V;    // adjoint recompute: all c sorted right singular vectors (c x n), or nullptr
    double* tape_s;    // adjoint recompute: all c sorted singular values
    void *oz_as, *oz_bs;   // mixed path: slice blocks of the tensor-core products (oz_gemm.cu)
    int *oz_ea, *oz_eb;    // and their row / column exponents
};

// Site tensor element i as double (storage f64 or f32), and the store back.
__device__ __forceinline__ double site_ld(const void* p, size_t i, int f32) {
    return f32 ? (double)static_cast<const float*>(p)[i] : static_cast<const double*>(p)[i];
}
__device__ __forceinline__ void site_st(void* p, size_t i, double v, int f32) {
    if (f32)
        static_cast<float*>(p)[i] = (float)v;
    else
        static_cast<double*>(p)[i] = v;
}

// ---------------------------------------------------------------------------
// kernel launchers (each returns the cudaError_t of the launch)
// ---------------------------------------------------------------------------
struct GateSpec {        // one gate to build
    int b;               // instance
    int kind;            // 0 gate, 1 swap
    int qa, qb, bond;
    double tau;          // frac * dt
    double wa, wb;       // on-site weights 1/deg
};
cudaError_t launch_build_gates(const GateSpec* d_specs, int count, int n, int nb,
                               const double* d_params, double* d_gates, cudaStream_t st);

cudaError_t launch_merge_gate(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st);
cudaError_t launch_reconstruct(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st);

struct JacobiPlan {
    int grid;            // total CTAs (cooperative)
    int max_resident;    // co-resident capacity
};
constexpr int kJacobiRowBytes = 128 * 1024;   // shared memory for the two row blocks of a pair
constexpr int kJacobiMaxB = 32;               // rows per block at most
constexpr int kQrWarps = 8;                   // warps per QR CTA
// rows per block for rows of length rowlen (elem_bytes each): two blocks fit the
// shared-memory budget, and there are at least two blocks when c > 1
__host__ __device__ inline int jacobi_block_rows(int rowlen, int c, int elem_bytes) {
    int b = kJacobiMaxB;
    while (b > 1 && (size_t)2 * b * rowlen * elem_bytes > (size_t)kJacobiRowBytes) b >>= 1;
    while (b > 1 && b >= c) b >>= 1;
    return b;
}
// FP32 preconditioning pass: rows of at most kJacobiRegL elements take the
// register path (one block of b <= kJacobiMaxB rows in shared memory, the
// other in registers), longer rows the shared-memory path above; in both the
// U32 rows are turned once per block pair by its accumulated rotation, so only
// the L-long W rows are staged.
constexpr int kJacobiRegL = 1024;
__host__ __device__ inline bool jacobi_f32_reg(int L) { return L <= kJacobiRegL; }
__host__ __device__ inline int jacobi_block_rows_f32(int L, int c) {
    if (!jacobi_f32_reg(L)) return jacobi_block_rows(L, c, 4);
    int b = kJacobiMaxB;
    while (b > 1 && b >= c) b >>= 1;
    return b;
}
// whether b rows per block fit the FP32 pass for rows of length L
__host__ __device__ inline bool jacobi_f32_fits(int b, int L, int c) {
    (void)c;
    return jacobi_f32_reg(L) ? b <= kJacobiMaxB : (size_t)2 * b * L * 4 <= (size_t)kJacobiRowBytes;
}
// block pairs per tournament round
__host__ __device__ inline int jacobi_pairs_per_round(int c, int b) {
    const int nb = (c + b - 1) / b;
    return (nb + (nb & 1)) / 2;
}
cudaError_t jacobi_max_resident(int* blocks);
// d_cta_op[grid]: op index of each CTA; d_cta_rank[grid]: rank within its op;
// d_group[nops]: CTAs per op.  d_sync: per-op counters (zeroed by the caller,
// layout documented in jacobi.cu).
// fp32 = true: the FP32 preconditioning pass on (W32 | U32) (U32 starts as I,
// W32 is filled from W0, scaled); false: the FP64 pass on (W | Z).
cudaError_t launch_jacobi(const OpDesc* d_desc, int nops, const int* d_cta_op, const int* d_cta_rank,
                          const int* d_group, unsigned* d_sync, int grid, int max_sweeps, double tol,
                          unsigned long long timeout_ns, int ld, bool fp32, cudaStream_t st,
                          double pre_rho = 1e-3);   // FP32 pass: stop once no rotation exceeds pre_rho
size_t jacobi_sync_words_per_op();
// sync words of a Jacobi launch over nops ops (theirs and the grid barrier's)
size_t jacobi_sync_words(int nops);

cudaError_t launch_truncate(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st);

// ---------------------------------------------------------------------------
// FP64-accurate GEMM on the tensor cores from exact slice products (oz_gemm.cu)
// ---------------------------------------------------------------------------
// One operand as a view over (row, k): A's rows are the rows i of A, B's rows
// the columns j of B.  mode 0: element (r, k) at base[g(r) * rs + k * ks], g(r) =
// gather[r] (or r when gather is null); mode 1 (right site of a merge): element
// (n, k) at base[(k * 4 + n / cr) * cap + n % cr].
struct OzOperand {
    const void* base;
    int f32;             // elements are float (else double)
    long long rs, ks;
    int mode, cr, cap;
    const int* gather;   // row gather (mode 0), or nullptr
};
// C = alpha A B + beta D (- I), C and D row-major (f64 or f32); row i of C and D
// is row c_gather[i] of their storage when c_gather is set
struct OzProblem {
    int M, N, K;
    const int* Ndyn;     // non-null: N is read on the device (<= N, which sizes the tiles)
    OzOperand A, B;
    void* C;
    int ldc, c_f32;
    const int* c_gather;
    double alpha, beta;
    const void* D;
    int ldd, d_f32, sub_identity;
    void *as, *bs;       // slice blocks of A and B
    int *ea, *eb;        // row / column exponents
    int Mt, Nt, Kt;      // tiles (128 rows, 64 columns, 64 bytes of K)
    int* status;         // MPDO_ST_TIMEOUT when a wait gives up (or nullptr)
};
// tiles of a problem: 128 rows of A, 64 columns of B, 64 bytes of K (32 bf16 or 16 tf32 values)
__host__ __device__ inline void oz_set_tiles(OzProblem& p, bool bf16) {
    const int KT = bf16 ? 32 : 16;
    p.Mt = (p.M + 127) / 128;
    p.Nt = (p.N + 63) / 64;
    p.Kt = (p.K + KT - 1) / KT;
}
size_t oz_slice_bytes(int rows, int K, bool bf16);   // slice blocks of an operand of rows x K
size_t oz_exp_ints(int rows);                          // its exponent array (rows rounded up to a tile)
void oz_tiles(OzProblem& p, bool bf16);
cudaError_t oz_prepare();
// slices both operands of count problems, then multiplies; max_m / max_n /
// max_rows_sliced bound the grids (CTAs outside a problem's tiles return)
cudaError_t launch_oz_gemm(const OzProblem* d_probs, int count, int max_m, int max_n, int max_rows_sliced, bool bf16,
                           unsigned long long timeout_ns, cudaStream_t st);

// The mixed path's tensor-core products of a chunk of ops, built on the
// device from the op descriptors (so the host-planned and the graph step
// share them): kind OZ_MERGE Theta = A B (then launch_gate_weight applies the
// gate and the left weights), OZ_RECON B_p' = Theta' Yk^T, OZ_E E = U U^T - I,
// OZ_Q Q = U - E U / 2, OZ_W W = Q W0.  probs: scratch for nops problems.
enum { OZ_MERGE = 0, OZ_RECON = 1, OZ_E = 2, OZ_Q = 3, OZ_W = 4 };
cudaError_t launch_oz_ops(const OpDesc* d_desc, int nops, int kind, OzProblem* probs, int chi_cap, bool bf16,
                          unsigned long long timeout_ns, cudaStream_t st);
// Theta' = G Theta in place in thetap and theta~ = lambda_l Theta' (column-major, Acm)
cudaError_t launch_gate_weight(const OpDesc* d_desc, int nops, int chi_cap, cudaStream_t st);

// Blocked Householder QR of the mixed path (qr_blocked.cu): panels of nb columns
// chosen by largest norm and factored with pivoting inside the panel in one CTA,
// compact-WY trailing updates as tensor-core products with FP64-class accuracy.
// Same output as launch_qr: the rows of R P^T in d.W0.  Scratch: d.W (panel
// reflectors and products), d.snorm (column norms, permutation), the op's slice
// buffers.  One panel loop over the chunk (ops with fewer columns idle through it).
int qrb_panel_width(int chi_cap);
// kernels one launch_qr_blocked issues for ranks up to r_max
int qrb_kernels(int chi_cap, int r_max);
// the blocked QR needs d.W to hold its scratch (48 ld + 256 doubles of ld^2)
inline bool qrb_fits(int chi_cap) { return 4 * chi_cap >= 128; }
cudaError_t qrb_prepare();
// r_max: the largest min(m, n) of the chunk's ops (<= 0: the capacity 4 chi_cap)
cudaError_t launch_qr_blocked(const OpDesc* d_desc, int nops, int chi_cap, OzProblem* probs, bool bf16,
                              unsigned long long timeout_ns, cudaStream_t st, int r_max);

int qr_threads();
cudaError_t qr_max_resident(int* blocks);
cudaError_t launch_qr(const OpDesc* d_desc, const int* d_cta_op, const int* d_cta_rank, const int* d_group,
                      unsigned* d_sync, int grid, unsigned long long timeout_ns, int ld, cudaStream_t st);

// C = alpha * A op(B) + beta * D (- I): see gemm.cu
struct GemmDesc {
    int M, N, K;
    const void* A;
    int lda, a_f32;
    const void* B;
    int ldb, b_f32, b_trans;
    double* C;
    int ldc;
    double alpha, beta;
    const void* D;
    int ldd, d_f32;
    int sub_identity;
    int a_trans;      // A stored K x M (default 0)
    int sym;          // 1: C is symmetric (A B with B = A^T, D = nullptr): only the tiles on and
                      // above the diagonal are computed, each written to both triangles
    int* status;      // tensor-core route: MPDO_ST_TIMEOUT lands here (or nullptr)
};
cudaError_t launch_gemm(const GemmDesc* d_desc, int count, int max_m, int max_n, bool fp32_compute,
                        cudaStream_t st);
// The batched GemmDesc products (f64 operands, sym computed in full) on the
// tensor cores: problem s takes slot s of the scratch (slices of slot_bytes per
// operand, exponents of exp_ints per operand, oz_slice_bytes / oz_exp_ints of
// the largest dimension) and probs[s]; max_m, max_n, max_k bound every product.
struct OzScratch {
    unsigned char *as, *bs;
    int *ea, *eb;
    OzProblem* probs;
    size_t slot_bytes, exp_ints;
};
cudaError_t launch_gemm_tc(const GemmDesc* d_desc, int count, int max_m, int max_n, int max_k, const OzScratch& scr,
                           bool bf16, unsigned long long timeout_ns, cudaStream_t st);

cudaError_t launch_trace_normalize(void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                                   int force, double* trace_out, int* status, cudaStream_t st);
cudaError_t launch_environments(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                                double* envL, double* envR, cudaStream_t st);
// E(comp at q) for the listed qubits: out[b][k] = <sigma^c_q> (divided by E0)
cudaError_t launch_measure_1q(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                              const double* envL, const double* envR, const int* d_q, int nq,
                              int comp, double* out, cudaStream_t st);
// all-pairs propagation: E(ca at i, cb at j) / E0 for every i with need[i] and
// every j > i into full[b][i][j]; unused entries untouched.  Scratch: wstack
// (two_stack_doubles) and part (two_part_doubles), device.
size_t two_stack_doubles(int n, int B, int chi_cap);
size_t two_part_doubles(int n, int B, int chi_cap);
cudaError_t launch_measure_2q(const void* sites, int sites_f32, const int* dims, int n, int B, int chi_cap,
                              const double* envL, const double* envR, int ca, int cb,
                              const unsigned char* d_need_i, double* wstack, double* part, double* full,
                              cudaStream_t st);
// d_trip[m][3] = (i, j, k): out[b][k] = full[b][i][j] (- one_a[b][i] one_b[b][j] if connected)
cudaError_t launch_gather_2q(const double* full, const double* one_a, const double* one_b,
                             const int* d_trip, int m, int np, int n, int B, int connected,
                             double* out, cudaStream_t st);

// ---------------------------------------------------------------------------
// adjoint (reverse mode through the Trotter sweep; adjoint.cu)
// ---------------------------------------------------------------------------
// Batched strided copy: dst[i][j] = scale * src[i][j] (src == nullptr: 0),
// i < rows, j < cols.  One launch serves count copies (grid.y = copy).
struct Copy2D {
    const double* src;
    double* dst;
    int rows, cols, src_ld, dst_ld;
    double scale;
};
cudaError_t launch_copy2d(const Copy2D* d_desc, int count, int max_rows, cudaStream_t st);

// One op of the backward sweep.  Matrices are compact row-major (leading
// dimension = row length); m = 4 cl, n = 4 cr, c = min(m, n), k = new chi_p.
struct BwdDesc {
    int cl, cm, cr, m, n, c, k;
    int is_gate;            // 0 for swaps (no parameter gradient)
    const double* G;        // the op's 16 x 16 gate
    const double* thetap;   // Theta' (m x n)
    const double* V;        // c x n sorted right singular vectors (rows)
    const double* s;        // c sorted singular values
    const double* lam;      // lambda_{p-1} (cl) or nullptr (p == 0)
    const double* sbar;     // cotangent of lambda_p (k)
    double* lbar_left;      // cotangent of lambda_{p-1} (cl), accumulated; nullptr when p == 0
    double* Vbar;           // k x n: cotangent of V_k^T, then scaled by 1/s_j^2
    double* K;              // c x k: V V-bar^T
    double* Om;             // c x k: Lorentzian-broadened F o K, zero diagonal
    double* Mk;             // k x c: Om^T - S_k^-2 K^T + diag(s-bar / s)
    double* S2;             // 2k x n: [V_k ; Om^T V]
    double* S3;             // 2k x n: [H_k ; V_k]
    double* X1;             // m x n: Theta' H, then Theta = A B
    double* X2;             // m x n: Theta'-bar, then Theta-bar
    double* gpart;          // [parts][256] partial G-bar sums of this launch
    double* gacc;           // [256] G-bar of the op, accumulated over steps
};
cudaError_t launch_svd_bwd_coeffs(const BwdDesc* d_desc, int nops, double rel_broadening, double rel_degenerate,
                                  cudaStream_t st);
cudaError_t launch_lambda_bwd(const BwdDesc* d_desc, int nops, int max_cl, cudaStream_t st);
cudaError_t launch_gate_bwd(const BwdDesc* d_desc, int nops, int parts, cudaStream_t st);
constexpr int kGateBwdParts = 32;

// Loss cotangent at the final state: for L = sum_i a_i <z_i> + sum_{i<j}
// W_ij (<z_i z_j> - <z_i><z_j>), writes dL/dB_k into sbar (site layout) for
// every instance and site, and coef[b] = (b_0..b_{N-1}, c, E(I), L).
// a [B][N], W [B][N][N] symmetric with zero diagonal.
struct LossScratch {
    double *L0, *L1, *L2, *R0, *R1, *R2, *T, *coef;
};
cudaError_t launch_loss_cotangent(const double* sites, const int* dims, int n, int B, int chi_cap, const double* a,
                                  const double* W, const LossScratch& s, double* sbar, cudaStream_t st);

// Parameter gradient from the accumulated G-bar of every (instance, op):
// X-bar = Frechet derivative of exp at (tau L_op)^T applied to G-bar (top
// right block of exp([[X^T, G-bar], [0, X^T]])), L-bar = tau X-bar, then
// dL/dtheta = <L-bar, dL_op/dtheta>.  grad [B][6n + 2nb] in the packing of
// the parameters (h_x, h_y, h_z, g0, g1, g2 per qubit, J, Jz per bond).
cudaError_t launch_param_grad(const GateSpec* d_specs, int count, int n, int nb, const double* d_params,
                              const double* gacc, double* contrib, int B, int n_ops, double* grad, cudaStream_t st);

}  // namespace mpdo
