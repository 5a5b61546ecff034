// C ABI of the adjoint: mpdo_grad_forward, mpdo_grad_backward, mpdo_grad.
//
// Forward: the Trotter steps of mpdo_trotter_step, with a checkpoint of the
// state (compact site tensors, Schmidt weights, bond dimensions) at the start
// of every step, the traces divided out at the end of every step and the
// rank of every truncation.
// Backward: the loss cotangent at the final state (adjoint.cu), then for
// each step from the last: undo the trace normalisation (B-bar_0 /= t; the
// loss is a ratio of traces, so the term of dt/dB drops out exactly), restore
// the step's checkpoint, recompute the step with the recorded ranks while
// taping every op (inputs, Theta', all singular values and vectors), and run
// the ops' backward passes in reverse layer order.  The gate cotangents of
// every (instance, op) accumulate over the steps (the gate is the same in
// every step) and become parameter gradients through the Frechet derivative
// of exp at the end.
#include <mpdo.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "ctx.h"
#include "internal.h"

using namespace mpdo;

namespace mpdo {

namespace {

constexpr double kBroadening = 1e-12;   // delta = kBroadening * s_0^2 in the Lorentzian 1/(s_j^2 - s_i^2)
constexpr double kDegenerate = 1e-10;   // singular values equal to this (relative) form a degenerate pair
constexpr int kBwdGemms = 10;

// bump allocator over device chunks (checkpoints of one forward run)
struct Arena {
    std::vector<double*> chunks;
    size_t cap_last = 0, used_last = 0;
    cudaError_t get(size_t n, double** out) {
        n = (n + 31) & ~(size_t)31;   // 256-byte granules
        if (chunks.empty() || used_last + n > cap_last) {
            const size_t want = std::max(n, (size_t)32 << 20);   // 256 MiB of doubles at least
            double* p = nullptr;
            cudaError_t e = dalloc(&p, want);
            if (e != cudaSuccess) return e;
            chunks.push_back(p);
            cap_last = want;
            used_last = 0;
        }
        *out = chunks.back() + used_last;
        used_last += n;
        return cudaSuccess;
    }
    void reset() {
        for (double* p : chunks) cudaFree(p);
        chunks.clear();
        cap_last = used_last = 0;
    }
};

struct StepRecord {
    std::vector<int> dims;   // [B][N+1] at the start of the step
    double* sites = nullptr; // compact site tensors, (b, p) in order
    double* lam = nullptr;   // copy of d_lam
};

struct TapeRec {   // one (instance, op) of a recomputed step
    int b, layer, idx, op, p, cl, cm, cr, k;
    TapeSlot slot;
};

}  // namespace

struct GradState {
    bool recorded = false;
    long long gen = -1;
    int n_steps = 0;
    Arena ck;
    std::vector<StepRecord> steps;   // n_steps + 1 records (the last one: the final state)
    std::vector<int> ranks;          // [B][n_steps * n_ops]
    double* d_traces = nullptr;      // [n_steps][B]
    Copy2D *h_cp = nullptr, *d_cp = nullptr;
    int cp_cap = 0;
    double* d_tape = nullptr;
    size_t tape_cap = 0;
    // backward slots
    int bslots = 0;
    size_t ws_slot = 0;
    double* d_ws = nullptr;
    BwdDesc *h_bd = nullptr, *d_bd = nullptr;
    GemmDesc *h_bg = nullptr, *d_bg = nullptr;   // [kBwdGemms][bslots]
    Copy2D *h_bc = nullptr, *d_bc = nullptr;     // [5][bslots]
    // mixed path: the backward products on the tensor cores (one slot per op in flight)
    unsigned char* d_oz = nullptr;
    OzScratch oz{};
    // adjoint state and loss
    double *d_sbar = nullptr, *d_lbar = nullptr, *d_gacc = nullptr, *d_contrib = nullptr, *d_grad = nullptr;
    double *d_a = nullptr, *d_W = nullptr, *d_ls = nullptr;
    LossScratch ls{};
    int alloc_B = 0, alloc_N = 0, alloc_cap = 0, alloc_ops = 0, alloc_P = 0;
};

void grad_free(GradState* g) {
    if (!g) return;
    g->ck.reset();
    void* ptrs[] = {g->d_traces, g->d_cp, g->d_tape, g->d_ws,   g->d_bd, g->d_bg, g->d_bc,  g->d_sbar,
                    g->d_lbar,   g->d_gacc, g->d_contrib, g->d_grad, g->d_a, g->d_W, g->d_ls, g->d_oz};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    void* hptrs[] = {g->h_cp, g->h_bd, g->h_bg, g->h_bc};
    for (void* p : hptrs)
        if (p) cudaFreeHost(p);
    delete g;
}

namespace {

int ensure_copy_descs(mpdo_ctx* c, GradState* g, int need) {
    if (g->cp_cap >= need) return MPDO_OK;
    if (g->d_cp) cudaFree(g->d_cp);
    if (g->h_cp) cudaFreeHost(g->h_cp);
    g->d_cp = nullptr;
    g->h_cp = nullptr;
    g->cp_cap = 0;
    CU(dalloc(&g->d_cp, (size_t)need));
    CU(cudaMallocHost((void**)&g->h_cp, sizeof(Copy2D) * need));
    g->cp_cap = need;
    (void)c;
    return MPDO_OK;
}

// checkpoint the current state into r
int save_state(mpdo_ctx* c, GradState* g, StepRecord& r) {
    const int B = c->B, N = c->N, cap = c->cap;
    r.dims = c->h_dims;
    size_t total = 0;
    for (int b = 0; b < B; ++b)
        for (int p = 0; p < N; ++p) total += (size_t)4 * r.dims[b * (N + 1) + p] * r.dims[b * (N + 1) + p + 1];
    CU(g->ck.get(total, &r.sites));
    CU(g->ck.get((size_t)B * N * cap, &r.lam));
    int rc = ensure_copy_descs(c, g, B * N);
    if (rc) return rc;
    CU(cudaStreamSynchronize(c->st));   // the descriptor buffer is reused
    size_t off = 0;
    int nc = 0, max_rows = 1;
    for (int b = 0; b < B; ++b)
        for (int p = 0; p < N; ++p) {
            const int cl = r.dims[b * (N + 1) + p], cr = r.dims[b * (N + 1) + p + 1];
            g->h_cp[nc++] = Copy2D{site(c, b, p), r.sites + off, 4 * cl, cr, cap, cr, 1.0};
            off += (size_t)4 * cl * cr;
            max_rows = std::max(max_rows, 4 * cl);
        }
    CU(cudaMemcpyAsync(g->d_cp, g->h_cp, sizeof(Copy2D) * nc, cudaMemcpyHostToDevice, c->st));
    CU(launch_copy2d(g->d_cp, nc, max_rows, c->st));
    CU(cudaMemcpyAsync(r.lam, c->d_lam, sizeof(double) * B * N * cap, cudaMemcpyDeviceToDevice, c->st));
    return MPDO_OK;
}

int restore_state(mpdo_ctx* c, GradState* g, const StepRecord& r) {
    const int B = c->B, N = c->N, cap = c->cap;
    int rc = ensure_copy_descs(c, g, B * N);
    if (rc) return rc;
    CU(cudaStreamSynchronize(c->st));
    size_t off = 0;
    int nc = 0, max_rows = 1;
    for (int b = 0; b < B; ++b)
        for (int p = 0; p < N; ++p) {
            const int cl = r.dims[b * (N + 1) + p], cr = r.dims[b * (N + 1) + p + 1];
            g->h_cp[nc++] = Copy2D{r.sites + off, site(c, b, p), 4 * cl, cr, cr, cap, 1.0};
            off += (size_t)4 * cl * cr;
            max_rows = std::max(max_rows, 4 * cl);
        }
    CU(cudaMemcpyAsync(g->d_cp, g->h_cp, sizeof(Copy2D) * nc, cudaMemcpyHostToDevice, c->st));
    CU(launch_copy2d(g->d_cp, nc, max_rows, c->st));
    CU(cudaMemcpyAsync(c->d_lam, r.lam, sizeof(double) * B * N * cap, cudaMemcpyDeviceToDevice, c->st));
    c->h_dims = r.dims;
    CU(cudaMemcpyAsync(c->d_dims, c->h_dims.data(), sizeof(int) * c->h_dims.size(), cudaMemcpyHostToDevice,
                       c->st));
    CU(cudaStreamSynchronize(c->st));
    return MPDO_OK;
}

int alloc_backward(mpdo_ctx* c, GradState* g) {
    const int B = c->B, N = c->N, cap = c->cap, ld = c->ld;
    const int P = 6 * N + 2 * c->nb;
    if (g->d_sbar && g->alloc_B == B && g->alloc_N == N && g->alloc_cap == cap && g->alloc_ops == c->n_ops &&
        g->alloc_P == P)
        return MPDO_OK;
    void* ptrs[] = {g->d_ws, g->d_bd, g->d_bg, g->d_bc, g->d_sbar, g->d_lbar, g->d_gacc, g->d_contrib,
                    g->d_grad, g->d_a, g->d_W, g->d_ls, g->d_oz};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    void* hptrs[] = {g->h_bd, g->h_bg, g->h_bc};
    for (void* p : hptrs)
        if (p) cudaFreeHost(p);
    g->d_ws = g->d_sbar = g->d_lbar = g->d_gacc = g->d_contrib = g->d_grad = g->d_a = g->d_W = g->d_ls = nullptr;
    g->d_oz = nullptr;
    g->oz = OzScratch{};
    g->d_bd = g->h_bd = nullptr;
    g->d_bg = g->h_bg = nullptr;
    g->d_bc = g->h_bc = nullptr;
    g->d_sbar = nullptr;
    CU(dalloc(&g->d_sbar, (size_t)B * N * site_elems(c)));
    CU(dalloc(&g->d_lbar, (size_t)B * N * cap));
    CU(dalloc(&g->d_gacc, (size_t)B * c->n_ops * 256));
    CU(dalloc(&g->d_contrib, (size_t)B * c->n_ops * 14));
    CU(dalloc(&g->d_grad, (size_t)B * P));
    CU(dalloc(&g->d_a, (size_t)B * N));
    CU(dalloc(&g->d_W, (size_t)B * N * N));
    // loss scratch: L0, L2, R0, R2 [B][N+1][cap]; L1, R1 [B][N+1][N][cap]; T [B][N][N][cap]; coef [B][N+3]
    const size_t v = (size_t)B * (N + 1) * cap, w = v * N, t = (size_t)B * N * N * cap;
    CU(dalloc(&g->d_ls, 4 * v + 2 * w + t + (size_t)B * (N + 3)));
    double* q = g->d_ls;
    g->ls.L0 = q; q += v;
    g->ls.L2 = q; q += v;
    g->ls.R0 = q; q += v;
    g->ls.R2 = q; q += v;
    g->ls.L1 = q; q += w;
    g->ls.R1 = q; q += w;
    g->ls.T = q; q += t;
    g->ls.coef = q;
    // backward slots: as many ops in flight as a layer has, within half the free memory
    g->ws_slot = (size_t)12 * ld * cap + (size_t)2 * ld * ld + (size_t)kGateBwdParts * 256;
    // mixed path: slices of both operands of one product per slot, every dimension <= ld
    const size_t oz_bytes = (size_t)256 * ((oz_slice_bytes(ld, ld, c->oz_bf16) + 255) / 256);
    const size_t oz_ints = oz_exp_ints(ld);
    const size_t oz_slot = c->mixed ? 2 * oz_bytes + 2 * oz_ints * sizeof(int) + sizeof(OzProblem) : 0;
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    const int want = B * c->max_layer;
    int s = (int)std::max<size_t>(
        1, std::min<size_t>(want, free_b / 2 / (g->ws_slot * sizeof(double) + oz_slot)));
    if (c->cfg.max_slots > 0) s = std::min(s, c->cfg.max_slots);
    CU(dalloc(&g->d_ws, (size_t)s * g->ws_slot));
    if (c->mixed) {
        CU(dalloc(&g->d_oz, (size_t)s * oz_slot));
        unsigned char* q8 = g->d_oz;
        g->oz.as = q8;
        q8 += (size_t)s * oz_bytes;
        g->oz.bs = q8;
        q8 += (size_t)s * oz_bytes;
        g->oz.probs = reinterpret_cast<OzProblem*>(q8);   // 256-byte aligned: oz_bytes is a multiple
        q8 += (size_t)s * sizeof(OzProblem);
        g->oz.ea = reinterpret_cast<int*>(q8);
        g->oz.eb = g->oz.ea + (size_t)s * oz_ints;
        g->oz.slot_bytes = oz_bytes;
        g->oz.exp_ints = oz_ints;
    }
    CU(dalloc(&g->d_bd, (size_t)s));
    CU(dalloc(&g->d_bg, (size_t)kBwdGemms * s));
    CU(dalloc(&g->d_bc, (size_t)5 * s));
    CU(cudaMallocHost((void**)&g->h_bd, sizeof(BwdDesc) * s));
    CU(cudaMallocHost((void**)&g->h_bg, sizeof(GemmDesc) * kBwdGemms * s));
    CU(cudaMallocHost((void**)&g->h_bc, sizeof(Copy2D) * 5 * s));
    g->bslots = s;
    g->alloc_B = B;
    g->alloc_N = N;
    g->alloc_cap = cap;
    g->alloc_ops = c->n_ops;
    g->alloc_P = P;
    return MPDO_OK;
}

GemmDesc gd(int M, int N, int K, const double* A, int lda, int a_trans, const double* Bm, int ldb, int b_trans,
            double* C, int ldc, const double* D = nullptr, int ldd = 0) {
    return GemmDesc{M, N, K, A, lda, 0, Bm, ldb, 0, b_trans, C, ldc, 1.0, D ? 1.0 : 0.0, D, ldd, 0, 0, a_trans};
}

// backward passes of one chunk of ops (disjoint sites)
int run_bwd_chunk(mpdo_ctx* c, GradState* g, const std::vector<const TapeRec*>& recs) {
    const int nops = (int)recs.size();
    const int N = c->N, cap = c->cap, ld = c->ld, S = g->bslots;
    BwdDesc* bd = g->h_bd;
    GemmDesc* bg = g->h_bg;
    Copy2D* bc = g->h_bc;
    int mx[kBwdGemms][3] = {};
    int max_pack = 1, max_unpack = 1, max_cl = 1;
    for (int s = 0; s < nops; ++s) {
        const TapeRec& t = *recs[s];
        const int m = 4 * t.cl, n = 4 * t.cr, cc = std::min(m, n), k = t.k, cm = t.cm;
        double* w = g->d_ws + (size_t)s * g->ws_slot;
        double* Ap = w;                 w += (size_t)ld * cap;   // B-bar_p' (m x k), then A-bar (m x cm)
        double* Vb = w;                 w += (size_t)ld * cap;   // V-bar (k x n), then B-bar (cm x n)
        double* K = w;                  w += (size_t)ld * cap;
        double* Om = w;                 w += (size_t)ld * cap;
        double* Mk = w;                 w += (size_t)ld * cap;
        double* S2 = w;                 w += (size_t)2 * ld * cap;
        double* S3 = w;                 w += (size_t)2 * ld * cap;
        double* TT = w;                 w += (size_t)2 * ld * cap;
        double* X1 = w;                 w += (size_t)ld * ld;
        double* X2 = w;                 w += (size_t)ld * ld;
        double* gp = w;
        double* lbar_p = g->d_lbar + ((size_t)t.b * N + t.p) * cap;
        BwdDesc& d = bd[s];
        d.cl = t.cl;
        d.cm = cm;
        d.cr = t.cr;
        d.m = m;
        d.n = n;
        d.c = cc;
        d.k = k;
        d.is_gate = c->layers[t.layer][t.idx].kind == 0;
        d.G = c->d_gates + ((size_t)t.b * c->n_ops + t.op) * 256;
        d.thetap = t.slot.thetap;
        d.V = t.slot.V;
        d.s = t.slot.s;
        d.lam = t.p > 0 ? t.slot.lam : nullptr;
        d.sbar = lbar_p;
        d.lbar_left = t.p > 0 ? g->d_lbar + ((size_t)t.b * N + t.p - 1) * cap : nullptr;
        d.Vbar = Vb;
        d.K = K;
        d.Om = Om;
        d.Mk = Mk;
        d.S2 = S2;
        d.S3 = S3;
        d.X1 = X1;
        d.X2 = X2;
        d.gpart = gp;
        d.gacc = g->d_gacc + ((size_t)t.b * c->n_ops + t.op) * 256;
        double* sb_p = g->d_sbar + ((size_t)t.b * N + t.p) * site_elems(c);
        double* sb_q = g->d_sbar + ((size_t)t.b * N + t.p + 1) * site_elems(c);
        // pack the cotangents of the op's outputs
        bc[2 * s] = Copy2D{sb_p, Ap, m, k, cap, k, 1.0};             // B-bar_p'  (cl, 4, k) -> m x k
        bc[2 * s + 1] = Copy2D{sb_q, Vb, 4 * k, t.cr, cap, t.cr, 1.0};   // B-bar_{p+1}' (k, 4, cr) -> k x n
        // unpack the cotangents of its inputs; lambda_p (before the op) is not an input
        bc[2 * nops + 3 * s] = Copy2D{Ap, sb_p, m, cm, cm, cap, 1.0};
        bc[2 * nops + 3 * s + 1] = Copy2D{Vb, sb_q, 4 * cm, t.cr, t.cr, cap, 1.0};
        bc[2 * nops + 3 * s + 2] = Copy2D{nullptr, lbar_p, 1, cap, cap, cap, 0.0};
        max_pack = std::max(max_pack, std::max(m, 4 * k));
        max_unpack = std::max(max_unpack, std::max(m, 4 * cm));
        max_cl = std::max(max_cl, t.cl);
        const double* Ac = t.slot.A;
        const double* Bc = t.slot.B;
        GemmDesc gl[kBwdGemms] = {
            gd(k, n, m, Ap, k, 1, t.slot.thetap, n, 0, Vb, n, Vb, n),      // 0: V-bar = Y-bar + B-bar_p'^T Theta'
            gd(cc, k, n, t.slot.V, n, 0, Vb, n, 1, K, k),                   // 1: K = V V-bar^T
            gd(k, n, cc, Mk, cc, 0, t.slot.V, n, 0, S3, n, Vb, n),         // 2: H_k = Mk V + S^-2 V-bar
            gd(k, n, cc, Om, k, 1, t.slot.V, n, 0, S2 + (size_t)k * n, n),  // 3: Om^T V
            gd(m, 2 * k, n, t.slot.thetap, n, 0, S2, n, 1, TT, 2 * k),     // 4: [Theta' V_k, Theta' V Om]
            gd(m, n, 2 * k, TT, 2 * k, 0, S3, n, 0, X1, n),                // 5: Theta' H
            gd(m, n, k, Ap, k, 0, t.slot.V, n, 0, X2, n, X1, n),           // 6: Theta'-bar
            gd(m, n, cm, Ac, cm, 0, Bc, n, 0, X1, n),                      // 7: Theta = A B
            gd(m, cm, n, X2, n, 0, Bc, n, 1, Ap, cm),                      // 8: A-bar = Theta-bar B^T
            gd(cm, n, m, Ac, cm, 1, X2, n, 0, Vb, n),                      // 9: B-bar = A^T Theta-bar
        };
        for (int q = 0; q < kBwdGemms; ++q) {
            gl[q].status = c->d_status + t.b;
            bg[(size_t)q * S + s] = gl[q];
            mx[q][0] = std::max(mx[q][0], gl[q].M);
            mx[q][1] = std::max(mx[q][1], gl[q].N);
            mx[q][2] = std::max(mx[q][2], gl[q].K);
        }
    }
    CU(cudaMemcpyAsync(g->d_bd, bd, sizeof(BwdDesc) * nops, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(g->d_bg, bg, sizeof(GemmDesc) * kBwdGemms * S, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(g->d_bc, bc, sizeof(Copy2D) * 5 * nops, cudaMemcpyHostToDevice, c->st));
    // The mixed path runs products 4, 6, 7, 8 and 9 on the tensor cores (slice
    // products, oz_gemm.cu), the others on the FP64 pipe (gemm.cu).  The slice
    // products bound their error by 2^-46 of the largest entry of a row of A
    // times the largest of a column of B, where FP64 bounds each term by its
    // own size; that is as good wherever the terms of a sum have comparable
    // sizes.  Products 0-3 feed S_k^-2 (V-bar - V_c K^T), a difference of
    // nearly equal parts scaled by up to (s_0 / s_k)^2, and product 5 sums
    // along K the rows of H_k (scale ~ s^-2) with those of V_k (scale 1), so
    // that V_k's share sits below the slices' resolution: with them on the
    // tensor cores a directional derivative of the N = 24 ring moved by 1e-3
    // of itself.
    const unsigned long long timeout_ns = (unsigned long long)c->cfg.barrier_timeout_ms * 1000000ull;
    auto gemm = [&](int q) {
        const bool tc = c->mixed && (q == 4 || q >= 6);
        return tc ? launch_gemm_tc(g->d_bg + (size_t)q * S, nops, mx[q][0], mx[q][1], mx[q][2], g->oz, c->oz_bf16,
                                   timeout_ns, c->st)
                  : launch_gemm(g->d_bg + (size_t)q * S, nops, mx[q][0], mx[q][1], false, c->st);
    };
    CU(launch_copy2d(g->d_bc, 2 * nops, max_pack, c->st));
    CU(gemm(0));
    CU(gemm(1));
    CU(launch_svd_bwd_coeffs(g->d_bd, nops, kBroadening, kDegenerate, c->st));
    CU(gemm(2));
    CU(gemm(3));
    CU(gemm(4));
    CU(gemm(5));
    CU(launch_lambda_bwd(g->d_bd, nops, max_cl, c->st));
    CU(gemm(6));
    CU(gemm(7));
    CU(launch_gate_bwd(g->d_bd, nops, kGateBwdParts, c->st));
    CU(gemm(8));
    CU(gemm(9));
    CU(launch_copy2d(g->d_bc + 2 * nops, 3 * nops, max_unpack, c->st));
    CU(cudaStreamSynchronize(c->st));   // the host descriptor buffers are reused by the next chunk
    return MPDO_OK;
}


// tape layout of step s from its checkpointed dims and recorded ranks
int plan_tape(mpdo_ctx* c, GradState* g, int s, std::vector<std::vector<TapeRec>>& recs) {
    const int N = c->N;
    std::vector<int> dims = g->steps[s].dims;
    recs.assign(c->layers.size(), {});
    size_t off = 0;
    struct Pending {
        int li, j;
        size_t oA, oB, oL, oT, oV, oS;
    };
    std::vector<Pending> pend;
    for (int li = 0; li < (int)c->layers.size(); ++li) {
        for (const Item& it : layer_items(c, li)) {
            const Op& op = c->layers[li][it.idx];
            const int b = it.b, p = op.p;
            int* dm = &dims[(size_t)b * (N + 1)];
            TapeRec r{};
            r.b = b;
            r.layer = li;
            r.idx = it.idx;
            r.op = c->layer_op0[li] + it.idx;
            r.p = p;
            r.cl = dm[p];
            r.cm = dm[p + 1];
            r.cr = dm[p + 2];
            r.k = g->ranks[(size_t)b * g->n_steps * c->n_ops + (size_t)s * c->n_ops + r.op];
            const size_t m = 4 * (size_t)r.cl, n = 4 * (size_t)r.cr, cc = std::min(m, n);
            if (r.k < 1 || r.k > c->chi_max[b] || r.k > (int)cc) return fail(MPDO_ESTATE, "recorded rank out of range");
            Pending pd{li, (int)recs[li].size(), 0, 0, 0, 0, 0, 0};
            auto take = [&](size_t cnt) {
                const size_t o = off;
                off += (cnt + 31) & ~(size_t)31;
                return o;
            };
            pd.oA = take(m * r.cm);
            pd.oB = take((size_t)4 * r.cm * r.cr);
            pd.oL = take((size_t)r.cl);
            pd.oT = take(m * n);
            pd.oV = take(cc * n);
            pd.oS = take(cc);
            pend.push_back(pd);
            recs[li].push_back(r);
            dm[p + 1] = r.k;
        }
    }
    if (off > g->tape_cap) {
        if (g->d_tape) cudaFree(g->d_tape);
        g->d_tape = nullptr;
        g->tape_cap = 0;
        CU(dalloc(&g->d_tape, off));
        g->tape_cap = off;
    }
    for (const Pending& pd : pend) {
        TapeRec& r = recs[pd.li][pd.j];
        r.slot = TapeSlot{g->d_tape + pd.oA, g->d_tape + pd.oB, g->d_tape + pd.oL,
                          g->d_tape + pd.oT, g->d_tape + pd.oV, g->d_tape + pd.oS};
    }
    return MPDO_OK;
}

}  // namespace

}  // namespace mpdo

extern "C" {

namespace {
// the gradient's forward and backward keep every singular vector (the SVD
// backward uses the complete V), so no Jacobi pair is skipped meanwhile
struct FullSvdScope {
    mpdo_ctx* c;
    explicit FullSvdScope(mpdo_ctx* x) : c(x) { c->full_svd = true; }
    ~FullSvdScope() { c->full_svd = false; }
};
}  // namespace

int mpdo_grad_forward(mpdo_ctx* c, int n_steps) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (n_steps < 1) return fail(MPDO_EINVAL, "n_steps must be >= 1");
    if (sites_f32(c)) return fail(MPDO_EINVAL, "the gradient needs MPDO_STORE_F64 site storage");
    FullSvdScope full(c);
    if (!c->grad) {
        c->grad = new (std::nothrow) GradState();
        if (!c->grad) return fail(MPDO_ENOMEM, "host allocation failed");
    }
    GradState* g = c->grad;
    g->recorded = false;
    g->ck.reset();
    g->steps.assign(n_steps + 1, StepRecord{});
    g->n_steps = n_steps;
    if (g->d_traces) cudaFree(g->d_traces);
    g->d_traces = nullptr;
    CU(dalloc(&g->d_traces, (size_t)n_steps * c->B));
    c->rank_steps = n_steps;
    c->rank_log.assign((size_t)c->B * n_steps * c->n_ops, 0);
    for (int step = 0; step < n_steps; ++step) {
        int rc = save_state(c, g, g->steps[step]);
        if (rc) return rc;
        for (int li = 0; li < (int)c->layers.size(); ++li) {
            std::vector<Item> items = layer_items(c, li);
            const size_t cs = (size_t)chunk_ops(c);
            for (size_t s0 = 0; s0 < items.size(); s0 += cs) {
                std::vector<Item> chunk(items.begin() + s0, items.begin() + std::min(items.size(), s0 + cs));
                rc = run_chunk(c, chunk, step, nullptr, nullptr, true);
                if (rc) return rc;
            }
        }
        rc = normalize_trace(c);
        if (rc) return rc;
        CU(cudaMemcpyAsync(g->d_traces + (size_t)step * c->B, c->d_trace, sizeof(double) * c->B,
                           cudaMemcpyDeviceToDevice, c->st));
    }
    int rc = save_state(c, g, g->steps[n_steps]);
    if (rc) return rc;
    g->ranks = c->rank_log;
    rc = check_status_code(c);
    if (rc) return rc;
    g->recorded = true;
    g->gen = c->gen;
    return MPDO_OK;
}

int mpdo_grad_backward(mpdo_ctx* c, const double* zbar, const double* wbar, double* grad, double* loss) {
    if (!c || !grad) return fail(MPDO_EINVAL, "ctx and grad must not be NULL");
    CU(cudaSetDevice(c->dev));
    GradState* g = c->grad;
    if (!g || !g->recorded) return fail(MPDO_ESTATE, "mpdo_grad_forward must come first");
    if (g->gen != c->gen) return fail(MPDO_ESTATE, "the state changed since mpdo_grad_forward");
    FullSvdScope full(c);
    const int B = c->B, N = c->N, cap = c->cap, P = 6 * N + 2 * c->nb;
    int rc = alloc_backward(c, g);
    if (rc) return rc;
    // loss weights: a[b][i] and the symmetric W[b][i][j] from the upper triangle of wbar
    std::vector<double> a((size_t)B * N, 0.0), W((size_t)B * N * N, 0.0);
    for (int b = 0; b < B; ++b) {
        for (int i = 0; i < N; ++i) {
            const double v = zbar ? zbar[(size_t)b * N + i] : 0.0;
            if (!std::isfinite(v)) return fail(MPDO_EINVAL, "zbar must be finite");
            a[(size_t)b * N + i] = v;
        }
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                const double v = wbar ? wbar[((size_t)b * N + i) * N + j] : 0.0;
                if (!std::isfinite(v)) return fail(MPDO_EINVAL, "wbar must be finite");
                W[((size_t)b * N + i) * N + j] = W[((size_t)b * N + j) * N + i] = v;
            }
    }
    CU(cudaMemcpyAsync(g->d_a, a.data(), sizeof(double) * a.size(), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(g->d_W, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemsetAsync(g->d_lbar, 0, sizeof(double) * B * N * cap, c->st));
    CU(cudaMemsetAsync(g->d_gacc, 0, sizeof(double) * B * c->n_ops * 256, c->st));
    CU(cudaMemsetAsync(g->d_sbar, 0, sizeof(double) * B * N * site_elems(c), c->st));
    // loss cotangent at the final state (the context holds it after the forward)
    CU(launch_loss_cotangent(c->d_sites, c->d_dims, N, B, cap, g->d_a, g->d_W, g->ls, g->d_sbar, c->st));
    std::vector<double> traces((size_t)g->n_steps * B), coef((size_t)B * (N + 3));
    CU(cudaMemcpyAsync(traces.data(), g->d_traces, sizeof(double) * traces.size(), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(coef.data(), g->ls.coef, sizeof(double) * coef.size(), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    std::vector<std::vector<TapeRec>> recs;
    for (int s = g->n_steps - 1; s >= 0; --s) {
        // B_0 <- B_0 / t at the end of step s
        if (c->cfg.force_trace) {
            rc = ensure_copy_descs(c, g, B);
            if (rc) return rc;
            const std::vector<int>& de = g->steps[s + 1].dims;
            int nc = 0;
            for (int b = 0; b < B; ++b) {
                const double t = traces[(size_t)s * B + b];
                if (!std::isfinite(t) || t == 0.0) continue;
                double* s0 = g->d_sbar + (size_t)b * N * site_elems(c);
                g->h_cp[nc++] = Copy2D{s0, s0, 4, de[(size_t)b * (N + 1) + 1], cap, cap, 1.0 / t};
            }
            CU(cudaMemcpyAsync(g->d_cp, g->h_cp, sizeof(Copy2D) * nc, cudaMemcpyHostToDevice, c->st));
            CU(launch_copy2d(g->d_cp, nc, 4, c->st));
        }
        rc = restore_state(c, g, g->steps[s]);
        if (rc) return rc;
        rc = plan_tape(c, g, s, recs);
        if (rc) return rc;
        // recompute the step, taping every op
        for (int li = 0; li < (int)c->layers.size(); ++li) {
            const std::vector<TapeRec>& L = recs[li];
            const size_t cs = (size_t)chunk_ops(c);
            for (size_t s0 = 0; s0 < L.size(); s0 += cs) {
                const size_t s1 = std::min(L.size(), s0 + cs);
                std::vector<Item> chunk;
                std::vector<int> forced;
                std::vector<TapeSlot> tape;
                for (size_t q = s0; q < s1; ++q) {
                    chunk.push_back(Item{L[q].b, L[q].layer, L[q].idx});
                    forced.push_back(L[q].k);
                    tape.push_back(L[q].slot);
                }
                rc = run_chunk(c, chunk, s, forced.data(), tape.data(), false);
                if (rc) return rc;
            }
        }
        // backward through the layers in reverse
        for (int li = (int)c->layers.size() - 1; li >= 0; --li) {
            const std::vector<TapeRec>& L = recs[li];
            for (size_t s0 = 0; s0 < L.size(); s0 += g->bslots) {
                const size_t s1 = std::min(L.size(), s0 + (size_t)g->bslots);
                std::vector<const TapeRec*> chunk;
                for (size_t q = s0; q < s1; ++q) chunk.push_back(&L[q]);
                rc = run_bwd_chunk(c, g, chunk);
                if (rc) return rc;
            }
        }
    }
    CU(launch_param_grad(c->d_specs, B * c->n_ops, N, c->nb, c->d_params, g->d_gacc, g->d_contrib, B, c->n_ops,
                         g->d_grad, c->st));
    CU(cudaMemcpyAsync(grad, g->d_grad, sizeof(double) * B * P, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (loss)
        for (int b = 0; b < B; ++b) loss[b] = coef[(size_t)b * (N + 3) + N + 2];
    // back to the final state of the forward run
    rc = restore_state(c, g, g->steps[g->n_steps]);
    if (rc) return rc;
    return check_status_code(c);
}

int mpdo_grad(mpdo_ctx* c, int n_steps, const double* zbar, const double* wbar, double* grad, double* loss) {
    int rc = mpdo_grad_forward(c, n_steps);
    if (rc) return rc;
    return mpdo_grad_backward(c, zbar, wbar, grad, loss);
}

}  // extern "C"
