// The libmpdo context and the host helpers shared by the C-ABI translation
// units (api.cu: init, build, step, measure; grad.cu: the adjoint).
#pragma once

#include <mpdo.h>

#include <string>
#include <vector>

#include "internal.h"

namespace mpdo {

constexpr int kProfKinds = 10;
enum { K_MERGE = 0, K_JACOBI = 1, K_TRUNC = 2, K_RECON = 3, K_TRACE = 4, K_MEASURE = 5, K_GATES = 6, K_JACOBI32 = 7,
       K_GEMM = 8, K_QR = 9 };

// Records msg for mpdo_last_error() and returns code.
int fail(int code, const std::string& msg);

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return ::mpdo::fail(MPDO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

// One (instance, op) work item of a layer.
struct Item {
    int b, layer, idx;
};

// Where the recompute of a step for the adjoint records one op (device
// pointers into the tape arena; rows are compact, leading dimension = the
// row length).
struct TapeSlot {
    double* A;        // site p before the op, (4 cl) x cm
    double* B;        // site p+1 before the op, (4 cm) x cr  (= cm x 4 cr)
    double* lam;      // lambda_{p-1}, cl values (unused when p == 0)
    double* thetap;   // Theta' = G (A B), (4 cl) x (4 cr)
    double* V;        // all c right singular vectors, sorted, c x (4 cr)
    double* s;        // all c singular values, sorted descending
};

struct GradState;   // adjoint buffers (grad.cu)
void grad_free(GradState* g);
struct GraphState;  // captured step (graph.cu)
void graph_free(GraphState* g);

}  // namespace mpdo

struct mpdo_ctx {
    mpdo_config cfg{};
    cudaStream_t st = nullptr;
    int dev = 0;
    int N = 0, B = 0, cap = 0, ld = 0;
    bool built = false;
    bool full_svd = false;   // set while the gradient runs: every SVD keeps all its singular vectors
    // schedule
    std::vector<mpdo::Layer> layers;
    std::vector<double> weights;
    std::vector<int> layer_op0;   // op index of each layer's first op
    int n_ops = 0, n_swaps = 0, max_layer = 0;
    int nb = 0;
    std::vector<int> chi_max;
    std::vector<double> cutoff;
    // state (device)
    double* d_sites = nullptr;    // [B][N][cap][4][cap], float elements when cfg.storage == MPDO_STORE_F32
    double* d_lam = nullptr;      // [B][N][cap]   lambda_p for p = 0..N-2
    int* d_dims = nullptr;        // [B][N+1]
    int* d_status = nullptr;      // [B]
    double* d_maxdisc = nullptr;  // [B]
    double* d_trace = nullptr;    // [B]
    double* d_params = nullptr;   // [B][6N + 2nb]
    double* d_gates = nullptr;    // [B][n_ops][256]
    mpdo::GateSpec* d_specs = nullptr;   // [B][n_ops]
    // per-slot workspaces
    int slots = 0;
    double *d_thetap = nullptr, *d_W = nullptr, *d_Z = nullptr, *d_Yk = nullptr, *d_snorm = nullptr;
    int* d_sweeps = nullptr;      // [slots] Jacobi sweeps of the last chunk
    int* d_pre_ok = nullptr;      // [slots] mixed path: the FP32 pass ended by its off-orthogonality rule
    bool mixed = false;           // mixed-precision SVD (FP32 preconditioning + FP64 finish)
    bool oz_bf16 = false;         // mixed path: tensor-core slices in bf16 (MPDO_MIXED_BF16X3), else tf32
    unsigned char *d_oz_as = nullptr, *d_oz_bs = nullptr;   // [slots] slice blocks of the tensor-core products
    int *d_oz_ea = nullptr, *d_oz_eb = nullptr;             // [slots][4 chi_cap] their exponents
    mpdo::OzProblem* d_oz = nullptr;                        // [slots] problems of one launch
    size_t oz_slot_bytes = 0;
    double *d_W0 = nullptr, *d_E = nullptr, *d_Q = nullptr;
    float *d_W32 = nullptr, *d_U32 = nullptr;
    mpdo::GemmDesc* d_gemm = nullptr;
    mpdo::GemmDesc* h_gemm = nullptr;   // pinned, [3][slots]
    mpdo::Copy2D* d_copy = nullptr;     // [4][slots] tape copies of a chunk
    mpdo::Copy2D* h_copy = nullptr;     // pinned
    std::vector<int> h_sweeps;
    long long prof_sweeps = 0, prof_svds = 0, prof_sweeps32 = 0;
    long long prof_crit = 0, prof_crit32 = 0, prof_chunks = 0;   // per chunk: largest sweeps of any op
    mpdo::OpDesc* d_desc = nullptr;
    mpdo::OpDesc* h_desc = nullptr;     // pinned
    int *d_cta = nullptr, *h_cta = nullptr;   // [3][grid cap]: op, rank, then group [slots]
    unsigned* d_sync = nullptr;
    int jacobi_resident = 0;
    int qr_resident = 0;
    // measurement
    double *d_wstack = nullptr, *d_part = nullptr;   // all-pairs propagation scratch
    double *d_envL = nullptr, *d_envR = nullptr, *d_full = nullptr, *d_one_a = nullptr, *d_one_b = nullptr,
           *d_out = nullptr;
    int *d_q = nullptr, *d_pairs = nullptr;
    unsigned char* d_need = nullptr;
    // host mirrors
    std::vector<int> h_dims;
    std::vector<int> rank_log;    // [B][steps*n_ops] of the last trotter_step call
    int rank_steps = 0;
    // imposed truncation ranks (mpdo_force_ranks): [B][forced_steps][n_ops]
    std::vector<int> forced;
    int forced_steps = 0;
    // adjoint
    mpdo::GradState* grad = nullptr;
    long long gen = 0;            // bumped whenever the state changes (step, set_state, build_gates)
    long long layout = 0;         // bumped whenever the op list or the workspaces change (build_gates)
    mpdo::GraphState* graph = nullptr;
    // autotuned Jacobi rows per block: [(chi_l * (cap+1) + chi_r) * 2 + fp32], 0 = the default rule
    std::vector<int> jb_table;
    int* d_jb_table = nullptr;
    // descriptors of the Gram-matrix GEMM sweeps (global.cu), grown on demand
    mpdo::GemmDesc* d_gq = nullptr;
    size_t gq_cap = 0;
    // host-side fault injection (mpdo_inject_fault): MPDO_FAULT_* of the next QR launch, 0 = none
    int inject = 0;
    // profiling
    bool prof = false;
    cudaEvent_t ev[2 * mpdo::kProfKinds] = {};
    double prof_ms[mpdo::kProfKinds] = {};
    long long prof_launch[mpdo::kProfKinds] = {};
    double prof_flops[mpdo::kProfKinds] = {};
};

namespace mpdo {

void free_all(mpdo_ctx* c);
int release_slots(mpdo_ctx* c);
inline size_t site_elems(const mpdo_ctx* c) { return (size_t)c->cap * 4 * c->cap; }
inline int sites_f32(const mpdo_ctx* c) { return c->cfg.storage == MPDO_STORE_F32 ? 1 : 0; }
inline size_t site_esize(const mpdo_ctx* c) { return sites_f32(c) ? sizeof(float) : sizeof(double); }
// site tensor (b, p), as stored (double or float)
inline void* site_v(mpdo_ctx* c, int b, int p) {
    return reinterpret_cast<char*>(c->d_sites) + ((size_t)b * c->N + p) * site_elems(c) * site_esize(c);
}
// site tensor (b, p) of an FP64-stored state (the adjoint requires MPDO_STORE_F64)
inline double* site(mpdo_ctx* c, int b, int p) { return c->d_sites + ((size_t)b * c->N + p) * site_elems(c); }
int check_status_code(mpdo_ctx* c);

// Bracket a launch with events when profiling; prof_collect reads the time
// after a stream synchronisation (so only call it where the host waits anyway).
struct ProfScope {
    mpdo_ctx* c;
    int k;
    ProfScope(mpdo_ctx* c_, int k_) : c(c_), k(k_) {
        if (c->prof) cudaEventRecord(c->ev[2 * k], c->st);
    }
    void stop() {
        if (c->prof) cudaEventRecord(c->ev[2 * k + 1], c->st);
    }
};
// adds the time between the events of kind k, the kernels launched between
// them and their algorithmic flops to the profile
void prof_collect(mpdo_ctx* c, int k, double flops, int kernels);

// Jacobi rows per block of a (chi_l, chi_r) class: the autotuned value, else dflt.
inline int tuned_block_rows(const mpdo_ctx* c, int cl, int cr, bool fp32, int dflt) {
    if (c->jb_table.empty() || cl > c->cap || cr > c->cap) return dflt;
    const int v = c->jb_table[((size_t)cl * (c->cap + 1) + cr) * 2 + (fp32 ? 1 : 0)];
    return v > 0 ? v : dflt;
}

// Co-resident CTA plan of the Jacobi launch over h[0..nops): hbase receives
// [op of each CTA | rank | CTAs per op], total the number of CTAs.
int plan_jacobi(mpdo_ctx* c, const OpDesc* h, int nops, bool fp32, int* hbase, int& total);

// The (instance, op) items of layer li, instances with the larger chi_max first
// (stable), and the number of ops per chunk: `slots`, or at most a quarter of
// the co-resident Jacobi CTAs (>= 16) when the instances' chi_max differ, so
// that the large ops of a chunk get their share of CTAs instead of one each.
std::vector<Item> layer_items(mpdo_ctx* c, int li);
int chunk_ops(mpdo_ctx* c);

// Descriptor of item `it` in workspace slot s, with the bond dimensions of
// c->h_dims (forced rank and tape cleared).
void fill_desc(mpdo_ctx* c, const Item& it, int s, OpDesc& d);

// One chunk of (instance, op) items of a layer: merge + gate, QR, Jacobi SVD,
// truncate, reconstruct.  forced (per item, or nullptr) imposes ranks; tape
// (per item, or nullptr) records what the adjoint needs; log_ranks writes the
// ranks into c->rank_log at row `step`.
// Orthogonality tolerance of the FP64 Jacobi pass.  The mixed path's
// contractions carry ~1e-7 relative error (TF32 split), so its FP64 finish
// stops at 1e-10 (singular values stay exact to ~1e-20, vectors to ~1e-10,
// five orders inside the mixed path's 1e-5 bound) instead of sqrt(L) eps;
// the FP64 path, an explicit jacobi_tol and the gradient keep the strict one.
constexpr double kMixedFinishTol = 1e-10;
// largest rotation (relative off-orthogonality) of the FP32 preconditioning
// sweep after which that pass stops
inline double precond_rho(const mpdo_ctx* c) { return c->cfg.precond_rho > 0.0 ? c->cfg.precond_rho : 1e-3; }
inline double fp64_jacobi_tol(const mpdo_ctx* c) {
    return (c->cfg.jacobi_tol <= 0.0 && c->mixed && !c->full_svd) ? kMixedFinishTol : c->cfg.jacobi_tol;
}

int run_chunk(mpdo_ctx* c, const std::vector<Item>& items, int step, const int* forced, const TapeSlot* tape,
              bool log_ranks);

// The trace normalisation that ends every step (when cfg.force_trace).
int normalize_trace(mpdo_ctx* c);

}  // namespace mpdo
