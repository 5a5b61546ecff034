/*
 * libmpdo -- MPO Lindblad-equation solver for one GB300 (sm_103a).
 *
 * Evolves the density matrix of N qubits, stored as a matrix product operator
 * in the normalised Pauli basis P_a/sqrt(2), a in (I, X, Y, Z) (App. A,
 * Eq. (mpo_def): the vectorised |rho>> is an MPS with local dimension 4),
 * under the Lindblad equation of Sec. 2.1 (Eq. (dtrho), Eq. (H0),
 * Eq. (K_def), Eqs. (D0)-(D2)), by second-order Trotter steps of two-site
 * propagator gates exp(L_ij dt) with SVD truncation after every gate (App. B:
 * the more severe of a relative discarded-weight cutoff and a maximum bond
 * dimension).  Observables are the Pauli expectation values of Sec. 2.3,
 * Eq. (mu) and Eq. (2Qdef), and the connected correlator of Eq. (etadef).
 *
 * Conventions
 *  - Every function returns MPDO_OK (0) or a negative MPDO_E* code and never
 *    aborts; mpdo_last_error() gives a message for the calling thread.
 *  - Host arrays passed in are caller-owned and copied during the call.
 *  - The context owns all device memory; it is allocated in mpdo_init (state
 *    and measurement buffers, sized by chi_cap) and mpdo_build_gates (gates
 *    and per-op workspaces, sized by the bond graph), never during a step.
 *  - Work is ordered on the CUDA stream given to mpdo_init.  Calls that return
 *    results in host memory synchronise that stream.
 *  - Bond dimensions are dynamic (chosen by truncation on the device) and
 *    bounded by each instance's chi_max <= chi_cap.
 *  - The state is real: in the Pauli basis the Lindbladian of Sec. 2.1 maps
 *    Hermitian operators to Hermitian operators, so the gate matrices and the
 *    MPO coefficients are real (MPDO_STORE_F64 plays the role of complex128
 *    storage, MPDO_STORE_F32 of complex64).
 */
#ifndef MPDO_H
#define MPDO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpdo_ctx mpdo_ctx;

/* return codes */
enum {
    MPDO_OK = 0,
    MPDO_EINVAL = -1,      /* invalid argument (message says which) */
    MPDO_ENOMEM = -2,      /* device or host allocation failed */
    MPDO_ECUDA = -3,       /* a CUDA runtime call failed */
    MPDO_ENOCONV = -4,     /* Jacobi SVD hit its sweep limit (some instance) */
    MPDO_ETIMEOUT = -5,    /* a device-side wait gave up (kernel returned early) */
    MPDO_ENONFINITE = -6,  /* NaN/Inf detected in some instance */
    MPDO_ECAPACITY = -7,   /* requested size exceeds a capacity fixed at init */
    MPDO_ESTATE = -8       /* call out of order (e.g. step before build_gates) */
};

/* per-instance status bits reported by mpdo_status */
enum {
    MPDO_ST_NOCONV = 1,
    MPDO_ST_NONFINITE = 2,
    MPDO_ST_TIMEOUT = 4,
    MPDO_ST_CAPACITY = 8
};

/* contraction precision (merge, gate and reconstruct contractions) */
enum { MPDO_FP64 = 0, MPDO_MIXED_TF32 = 1, MPDO_MIXED_BF16X3 = 2 };
/* storage of the site tensors */
enum { MPDO_STORE_F64 = 0, MPDO_STORE_F32 = 1 };

typedef struct {
    int n_qubits;            /* N >= 3 (Sec. 2.1 model; the paper's solver wants N > 2) */
    int batch;               /* B >= 1 independent instances sharing one bond graph */
    int chi_cap;             /* capacity bond dimension, >= every chi_max, <= 512 */
    int precision;           /* MPDO_FP64 | MPDO_MIXED_TF32 | MPDO_MIXED_BF16X3 */
    int storage;             /* MPDO_STORE_F64 | MPDO_STORE_F32: element type of the stored site
                                tensors (f32: half the memory; every contraction, the SVD
                                and the measurements still compute in FP64 or the chosen
                                mixed precision, and round the new sites to float).  The
                                gradient needs MPDO_STORE_F64. */
    int trotter_order;       /* 2: symmetric second-order product; 4: Suzuki's triple jump
                                S2(w1 dt) S2(w0 dt) S2(w1 dt), w1 = 1/(2 - 2^(1/3)), w0 = 1 - 2 w1
                                (App. B uses order 4; odd orders are not built) */
    int force_trace;         /* 1: rho /= tr rho after every step (App. B b_force_rho_trace) */
    int jacobi_max_sweeps;   /* sweep limit of the Jacobi SVD (default 100, at most 128) */
    double jacobi_tol;       /* <= 0: sqrt(L) * DBL_EPSILON for rows of length L */
    unsigned barrier_timeout_ms;  /* limit of every device-side wait (default 4000) */
    int max_slots;           /* <= 0: automatic; else max two-site ops in flight */
    int device;              /* CUDA device ordinal; < 0: the calling thread's current device */
    int qr_blocked;          /* mixed path only: 1 = blocked Householder QR (window-pivoted panels of
                                16 columns, trailing updates on the tensor cores); 0 (default) =
                                the column-by-column QR, measured faster on this GPU */
    double precond_rho;      /* mixed path only: the FP32 preconditioning sweeps stop after a sweep
                                whose largest rotation (relative off-orthogonality |g|/sqrt(a b) of
                                a rotated pair) was at most this (<= 0: 1e-3); a smaller value
                                trades FP32 sweeps for fewer FP64 finishing sweeps.  Accuracy is
                                unchanged: the FP64 sweeps finish to the FP64 tolerance. */
} mpdo_config;

typedef struct {
    /* per-instance model parameters, row-major [B][N] (h_y, g1 may be NULL = 0) */
    const double *h_x, *h_y, *h_z;     /* on-site fields of Eq. (H0) */
    const double *g0, *g1, *g2;        /* rates of Eqs. (D0), (D1), (D2), >= 0 */
    int n_bonds;                       /* >= 1; every qubit must be on some bond */
    const int *bond_i, *bond_j;        /* [n_bonds] qubits = positions on the MPO path */
    const double *J, *Jz;              /* [B][n_bonds] couplings of Eq. (K_def); Jz may be NULL */
    const int *chi_max;                /* [B] max bond dimension (App. B max_dim_rho) */
    const double *cutoff;              /* [B] max relative discarded weight (App. B cut_off_rho) */
    const char *init_pauli;            /* 2N chars, e.g. "+z+z-x" (Sec. 2.2); NULL = all "+z" */
} mpdo_model;

/* Fill *cfg with defaults (n_qubits, batch and chi_cap still to be set). */
int mpdo_config_default(mpdo_config *cfg);

/* Create a context: validates cfg, allocates every device buffer for
 * chi_cap and the bond graph size given later (up to n_qubits).  cuda_stream
 * is a cudaStream_t (NULL = legacy default stream) that all work is ordered on. */
int mpdo_init(mpdo_ctx **out, const mpdo_config *cfg, void *cuda_stream);

/* Build the op list of one Trotter step from the bond graph (even
 * nearest-neighbour bonds, odd ones, then each long-range bond through swap
 * gates; Sec. 2.5 maps any connectivity onto the 1D path), then build every
 * two-site gate exp(L_op * f * dt) on the device (16x16, real, Pauli basis)
 * and reset the state to the Pauli product state rho(t0) of Sec. 2.2.
 * model arrays are host memory.  Errors: EINVAL (bad graph, negative rates,
 * chi_max > chi_cap, malformed init string), ECUDA. */
int mpdo_build_gates(mpdo_ctx *ctx, const mpdo_model *model, double dt);

/* Replace every instance's state by the graph state of Sec. 2.2, Eq.
 * (graph_state): all qubits +x, then a controlled-Z on every pair (i, j) of
 * pairs[n_pairs][2] (host memory; path positions, i != j; the CZs commute, so
 * the order is immaterial).  Each CZ runs as a two-site gate (its Pauli-basis
 * superoperator, a signed permutation) through the same merge / QR / SVD /
 * truncation path as a Trotter step, with swap gates bringing j next to i; the
 * state is exact while each instance's chi_max holds the graph state's bond
 * dimensions (at most 4^k across a cut crossed by k pairs).  Call after
 * mpdo_build_gates (which sets the Pauli product state instead).  EINVAL,
 * ESTATE, and the status errors of mpdo_trotter_step. */
int mpdo_init_graph_state(mpdo_ctx *ctx, const int *pairs, int n_pairs);

/* Advance every instance by n_steps Trotter steps (cfg.trotter_order).  Per op:
 * merge the two sites, apply the gate, weight by the left Schmidt values,
 * Householder QR (only R is kept), SVD of R (FP64 one-sided Jacobi on its
 * rows), truncate, write the two new sites.  After each
 * step the trace is forced to 1 when cfg.force_trace.  Returns ENOCONV /
 * ENONFINITE / ETIMEOUT when some instance reported that status (the other
 * instances are still advanced), ESTATE before mpdo_build_gates. */
int mpdo_trotter_step(mpdo_ctx *ctx, int n_steps);

/* mpdo_trotter_step with the step captured into a CUDA graph: the first call
 * after mpdo_build_gates captures one step (planner kernels read the bond
 * dimensions on the device and size every launch there, so nothing returns
 * to the host inside a step) and every call replays it n_steps times, then
 * synchronises once.  Same results, rank log and status errors as
 * mpdo_trotter_step; kernel profiling is not collected; EINVAL while forced
 * ranks are set; ECAPACITY if a chunk holds more ops than co-resident CTAs. */
int mpdo_trotter_step_graph(mpdo_ctx *ctx, int n_steps);
/* <sigma^comp_q> / tr rho for each q in qubits[nq] and each instance
 * (Eq. (mu)); comp in 'X','Y','Z','I'.  out is [B][nq] doubles, a host
 * pointer (out_on_device = 0; the call synchronises) or a device pointer. */
int mpdo_measure_1q(mpdo_ctx *ctx, const int *qubits, int nq, char comp, double *out,
                    int out_on_device);

/* <sigma^comp[0]_i sigma^comp[1]_j> / tr rho for each pair (i, j) in
 * pairs[np][2] (i != j, Eq. (2Qdef)); connected != 0 subtracts
 * <sigma_i><sigma_j> (Eq. (etadef)).  out is [B][np] (host or device). */
int mpdo_measure_2q(mpdo_ctx *ctx, const int *pairs, int np, const char comp[2], int connected,
                    double *out, int out_on_device);

/* Second Renyi entropy of every instance, Sec. 2.3 Eq. (S_2):
 * S2 = -ln tr(rho^2) of the normalised rho.  In the orthonormal basis
 * P_a/sqrt2 tr(rho^2) = <<rho|rho>> / (tr rho)^2, the squared norm of the
 * coefficient MPS over the squared trace, computed by a left-to-right sweep of
 * Gram matrices (batched FP64 GEMMs).  out is [B] doubles, host (out_on_device
 * = 0; the call synchronises) or device.  Uses the per-op workspaces (the state
 * is untouched).  ESTATE before mpdo_build_gates. */
int mpdo_renyi2(mpdo_ctx *ctx, double *out, int out_on_device);

/* Operator space entanglement entropy of every instance, Sec. 2.3 Eq. (OSEE):
 * the von Neumann entropy -sum_k p_k ln p_k, p_k = s_k^2 / sum s^2, of the
 * normalised vectorised state |rho>> for the cut between path positions bond
 * and bond + 1 (bond in [0, N-2]; the paper's central bond is N/2 - 1), from
 * its exact Schmidt values s_k: Gram matrices X, Y of the two halves (batched
 * FP64 GEMM sweeps), X = F_X^T F_X and Y = F_Y^T F_Y from FP64 Jacobi SVDs, s_k
 * the singular values of F_X F_Y^T (a third Jacobi SVD).  Independent of the
 * gauge of the stored tensors.  out as for mpdo_renyi2.  A Jacobi SVD that hits
 * cfg.jacobi_max_sweeps sets MPDO_ST_NOCONV for its instance (mpdo_status).
 * EINVAL (bond), ESTATE, ECUDA. */
int mpdo_osee(mpdo_ctx *ctx, int bond, double *out, int out_on_device);

/* Per-instance status bits (MPDO_ST_*), largest relative discarded weight of
 * any op since the last build_gates, current bond dimensions chi[B][N-1] and
 * the trace before the last normalisation trace_before[B].  Any pointer may
 * be NULL.  Host memory; synchronises the stream. */
int mpdo_status(mpdo_ctx *ctx, int *status, double *max_discarded, int *chi, double *trace_before);

/* Replace instance b's state: dims[N+1] bond dimensions (dims[0] = dims[N] = 1,
 * each <= chi_max of b), tensors = the N site tensors (dims[p], 4, dims[p+1])
 * packed one after another, row-major, host memory.  Schmidt weights are set
 * to 1.  Used to start from a prepared (e.g. saturated) state. */
int mpdo_set_state(mpdo_ctx *ctx, int b, const int *dims, const double *tensors);

/* Copy instance b's state out: dims[N+1] and the packed site tensors (at most
 * cap doubles; returns ECAPACITY if they do not fit).  Host memory. */
int mpdo_get_state(mpdo_ctx *ctx, int b, int *dims, double *tensors, long long cap);

/* Number of ops (gates + swaps) of one Trotter step, and of swaps. */
int mpdo_op_counts(mpdo_ctx *ctx, int *n_ops, int *n_swaps, int *n_layers);

/* Rank log: the truncation rank k of every op of the last mpdo_trotter_step
 * call, [B][n_steps * n_ops] in step order.  cap = capacity of k in ints. */
int mpdo_rank_log(mpdo_ctx *ctx, int *k, long long cap);

/* Impose the truncation ranks of the next mpdo_trotter_step calls (frozen-rank
 * mode, App. B's rule replaced by a recorded sequence): k is host memory,
 * [B][n_steps][n_ops] in the layout of mpdo_rank_log; step s of every later
 * mpdo_trotter_step call (counted from that call's first step) uses row s, steps
 * beyond n_steps use the rule.  Each k must be in [1, chi_max of its instance];
 * an op never keeps more values than its bond matrix has.  k = NULL or
 * n_steps <= 0 clears.  mpdo_build_gates clears as well.  Used for finite-
 * difference gradients, which need the ranks held fixed.  EINVAL, ESTATE. */
int mpdo_force_ranks(mpdo_ctx *ctx, const int *k, int n_steps);
/* Autotune the Jacobi SVD's rows per block for each bond-dimension class
 * (chi_l, chi_r) in classes[n_classes][2] (each in [1, chi_cap]): for every
 * candidate block size that fits shared memory, the Jacobi launch is timed on
 * seeded graded matrices of the class's shape, one per op in flight (the
 * largest layer), and the fastest is kept (FP64 pass, and the FP32 pass of the
 * mixed path).  Later steps (plain and graph) use the table; classes not tuned
 * keep the default rule (largest block that fits).  chosen (host, may be NULL)
 * receives [n_classes][2] = (FP64 block, FP32 block or 0).  Uses the per-op
 * workspaces only (the state is untouched); synchronises.  EINVAL, ESTATE, ECUDA. */
int mpdo_autotune(mpdo_ctx *ctx, const int *classes, int n_classes, int *chosen);
/* Copy instance b's gate matrices out: [n_ops][16][16] row-major doubles in
 * step order (swaps included), host memory, cap = capacity in doubles. */
int mpdo_gates(mpdo_ctx *ctx, int b, double *out, long long cap);

/* Host-only (no GPU needed): the op list of one Trotter step for an n-qubit
 * path with the given bonds.  ops[k*7 + (0..6)] = (layer, kind 0 gate /
 * 1 swap, left position p, qubit at p, qubit at p+1, bond index or -1,
 * fraction of dt times 2).  cap = capacity of ops in ints; *n_ops receives
 * the number of ops (also when ops is NULL).  EINVAL for a bad graph. */
int mpdo_schedule(int n, int n_bonds, const int *bond_i, const int *bond_j, int *ops, long long cap,
                  int *n_ops);

/* Host-side fault injection, for testing the failure handling (Sec. 2.5's
 * solver has none; every device-side wait here is bounded).  kind =
 * MPDO_FAULT_DROP_CTA: the next Householder QR launch of mpdo_trotter_step
 * leaves out one CTA of the first op that was planned two or more, while that
 * op's group still counts it; the op's other CTAs then wait at their first
 * barrier for a CTA that never arrives, give up after cfg.barrier_timeout_ms,
 * record MPDO_ST_TIMEOUT for the op's instance and return, and the step
 * returns MPDO_ETIMEOUT.  The GPU context stays usable.  One-shot (cleared once
 * applied); kind = 0 cancels.  EINVAL for an unknown kind. */
enum { MPDO_FAULT_DROP_CTA = 1 };
int mpdo_inject_fault(mpdo_ctx *ctx, int kind);

/* Kernel timing.  mpdo_profile_enable(ctx, 1) brackets every kernel launch
 * of the step with CUDA events on the context stream and accumulates, per
 * kernel kind k (0 merge+gate, 1 Jacobi SVD (FP64), 2 truncate, 3 reconstruct,
 * 4 trace, 5 environments/measure, 6 gate build, 7 FP32 preconditioning
 * Jacobi, 8 preconditioner GEMMs, 9 Householder QR), the device time in ms,
 * the number of kernels launched and the algorithmic flops of the work launched
 * (merge 32 cl cm cr, gate 512 cl cr, SVD 21 n^3 with n = 4 max(cl, cr),
 * reconstruct 32 cl cr k; 0 for the other kinds).  mpdo_profile_read copies
 * up to kmax kinds (any pointer may be NULL) and, if reset != 0, zeroes them. */
int mpdo_profile_enable(mpdo_ctx *ctx, int on);
int mpdo_profile_read(mpdo_ctx *ctx, double *ms, long long *launches, double *flops, int kmax, int reset);
/* FP64 Jacobi sweeps summed over the SVDs profiled since the last reset, the
 * number of those SVDs, and the FP32 preconditioning sweeps (mixed precision
 * only).  Profiling must be enabled. */
int mpdo_profile_sweeps(mpdo_ctx *ctx, long long *sweeps, long long *svds, long long *sweeps_fp32);

/* The critical path of the same SVDs: every chunk of ops shares one Jacobi
 * launch per pass, which lasts as long as its slowest op.  crit and crit_fp32
 * are the sums over chunks of the largest FP64 and FP32 sweep counts of any op
 * in the chunk; chunks is the number of chunks.  Any pointer may be NULL.
 * Profiling must be enabled; mpdo_profile_read(reset = 1) zeroes them. */
int mpdo_profile_sweeps_critical(mpdo_ctx *ctx, long long *crit, long long *crit_fp32, long long *chunks);

/* mpdo_measure_1q without any device allocation, on a state held in the
 * caller's device memory.  For callers that cannot call cudaMalloc: frameworks
 * that give all device memory to their own allocator up front (a hidden
 * allocation would fail or break their accounting), and code whose rules
 * forbid the runtime's allocator.  The paper has no counterpart; it is the
 * same computation as mpdo_measure_1q.
 *   sites   device, [batch][n_qubits][chi_cap][4][chi_cap] doubles, the site
 *           tensors (l, a, r) of each instance (f64 elements only, the layout
 *           of an MPDO_STORE_F64 context)
 *   dims    device, [batch][n_qubits+1] ints, bond dimensions, dims[0] =
 *           dims[n_qubits] = 1, each in [1, chi_cap]
 *   qubits  device, [nq] ints in [0, n_qubits)
 *   out     device, [batch][nq] doubles: <sigma^comp_q> / tr rho
 *   cuda_stream  cudaStream_t the work is ordered on (NULL = default stream)
 * dims and qubits are read on the device, so the host cannot check them: the
 * call clamps them into range before any kernel uses them, and writes NaN to
 * out[b][k] when a bond dimension of instance b or qubits[k] was out of range.
 * Scratch: a static device array of 2^18 doubles (2 MiB) that every device
 * loading the library keeps until the process exits; a call needs
 * 2 * batch * (n_qubits + 1) * chi_cap doubles plus batch * (n_qubits + 2) +
 * 2 * nq ints (two per double), and larger sizes are rejected with ECAPACITY.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  All calls share the array and it keeps
 * the last call's contents; calls that overlap on the GPU race on it.
 * Asynchronous: returns after queuing the kernels; EINVAL / ECAPACITY / ECUDA
 * with mpdo_last_error(). */
int mpdo_measure_1q_noalloc(const double *sites, const int *dims, int n_qubits, int batch, int chi_cap,
                            const int *qubits, int nq, char comp, double *out, void *cuda_stream);

/* C = A B with FP64 semantics on the tensor cores: the product the mixed path
 * uses for its contractions and SVD-preconditioner GEMMs, on caller matrices
 * (the paper has none; its contractions are FP64 ITensor/LAPACK calls).  Each
 * row of A and column of B is scaled by a power of two and cut into six 8-bit
 * slices, exact in tf32 (kind = MPDO_MIXED_TF32) or bf16 (MPDO_MIXED_BF16X3);
 * the 21 slice products of the leading levels are formed by tcgen05 MMAs with
 * error-free FP32 accumulation per 256 values of K and summed in FP64, so the
 * error is about 2^-46 |A_i|max |B_j|max per term of the sum.
 *   A  device, M x K row-major (lda >= K);  B  device, K x N (ldb >= N);
 *   C  device, M x N (ldc >= N), overwritten.
 * Allocates its slice scratch (cudaMalloc) per call and synchronises the
 * stream.  A non-finite entry makes its row of C (A) or column (B) NaN.
 * EINVAL (sizes, kind), ENOMEM, ECUDA. */
int mpdo_gemm_tc(int M, int N, int K, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
                 int kind, void *cuda_stream);

/* Reverse-mode gradient of the observables with respect to the model
 * parameters (the paper has no gradient; this differentiates the update of
 * App. B as implemented here, with the ranks of the forward run held fixed).
 *
 * mpdo_grad_forward advances every instance by n_steps Trotter steps exactly
 * as mpdo_trotter_step does, and keeps what the backward pass needs: a device
 * checkpoint of the state at the start of every step (compact site tensors,
 * Schmidt weights, bond dimensions: about sum_p 4 chi_p chi_{p+1} doubles per
 * instance and step), the trace divided out after each step and the rank of
 * every truncation.  The checkpoints are allocated by this call and kept until
 * the next mpdo_grad_forward or mpdo_destroy.  The observables at the final
 * time are then read with mpdo_measure_1q / mpdo_measure_2q as usual.
 *
 * mpdo_grad_backward returns, per instance b, the gradient of
 *   L_b = sum_i zbar[b][i] <sigma^z_i>
 *       + sum_{i<j} wbar[b][i][j] (<sigma^z_i sigma^z_j> - <sigma^z_i><sigma^z_j>)
 * at the final time of the last mpdo_grad_forward (Eq. (mu), Eq. (etadef)):
 * zbar is [B][N] and wbar [B][N][N] host arrays (only the entries i < j of wbar
 * are read; either may be NULL = 0), i.e. the cotangents of the observables,
 * as in a vector-Jacobian product.  grad is [B][6N + 2 n_bonds] host memory,
 * packed like the model: d/dh_x[N], d/dh_y[N], d/dh_z[N], d/dg0[N], d/dg1[N],
 * d/dg2[N], d/dJ[n_bonds], d/dJz[n_bonds].  loss (host [B], may be NULL)
 * receives L_b.  The pass recomputes every step from its checkpoint with the
 * recorded ranks, differentiates each op (gate contraction, weighting, the
 * truncated SVD with Lorentzian-broadened 1/(s_j^2 - s_i^2), width 1e-12 s_0^2,
 * pairs equal to 1e-10 relative treated as one degenerate subspace)
 * and maps the gate cotangents to the parameters through the Frechet
 * derivative of exp.  Afterwards the context again holds the final state.
 * Accuracy: FP64; the truncated-SVD backward divides by gaps s_j^2 - s_i^2 and
 * by kept s_j^2, so kept singular values far below the largest (a cutoff much
 * under 1e-10) amplify the rounding of the forward SVD.
 * Errors: ESTATE without a preceding mpdo_grad_forward or after the state
 * changed (step, set_state, build_gates); EINVAL for non-finite weights;
 * ENOMEM; the status errors of mpdo_trotter_step.
 *
 * mpdo_grad = mpdo_grad_forward then mpdo_grad_backward. */
int mpdo_grad_forward(mpdo_ctx *ctx, int n_steps);
int mpdo_grad_backward(mpdo_ctx *ctx, const double *zbar, const double *wbar, double *grad, double *loss);
int mpdo_grad(mpdo_ctx *ctx, int n_steps, const double *zbar, const double *wbar, double *grad, double *loss);
/* Message of the last error on this thread ("" if none). */
const char *mpdo_last_error(void);

/* Free every device buffer of the context (NULL is a no-op). */
void mpdo_destroy(mpdo_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MPDO_H */
