// C ABI of libmpdo: context, validation, the Trotter-step driver and the
// measurement entry points (declared and documented in include/mpdo.h).
#include <mpdo.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "internal.h"

using namespace mpdo;

namespace {

thread_local std::string g_err;
}  // namespace

namespace mpdo {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace mpdo

namespace mpdo {
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
}  // namespace mpdo

namespace {
// rho(t0) site vectors: v[b][q][4] -> site (b, q), element [0][s][0]
__global__ void init_product_kernel(void* sites, int f32, const double* v, int N, int cap) {
    const int b = blockIdx.x, q = threadIdx.x;
    if (q >= N) return;
    const size_t base = ((size_t)b * N + q) * (size_t)cap * 4 * cap;
    for (int s = 0; s < 4; ++s) site_st(sites, base + (size_t)s * cap, v[((size_t)b * N + q) * 4 + s], f32);
}

}  // namespace


namespace mpdo {

void free_all(mpdo_ctx* c) {
    release_slots(c);
    void* ptrs[] = {c->d_sites, c->d_lam,  c->d_dims,  c->d_status, c->d_maxdisc, c->d_trace, c->d_params,
                    c->d_gates, c->d_specs, c->d_envL,  c->d_envR,   c->d_full,    c->d_one_a, c->d_one_b,
                    c->d_out,   c->d_q,     c->d_pairs, c->d_need,   c->d_jb_table, c->d_gq,
                    c->d_wstack, c->d_part};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->grad) grad_free(c->grad);
    c->grad = nullptr;
    if (c->graph) graph_free(c->graph);
    c->graph = nullptr;
}

int release_slots(mpdo_ctx* c) {
    void* ptrs[] = {c->d_thetap, c->d_W,    c->d_Z,     c->d_Yk,    c->d_snorm, c->d_desc,  c->d_cta,
                    c->d_sync,   c->d_sweeps, c->d_pre_ok, c->d_W0,  c->d_E,     c->d_Q,     c->d_W32,
                    c->d_U32,    c->d_gemm,  c->d_copy,  c->d_oz_as, c->d_oz_bs, c->d_oz_ea, c->d_oz_eb,
                    c->d_oz};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c->d_thetap = c->d_W = c->d_Z = c->d_Yk = c->d_snorm = nullptr;
    c->d_W0 = c->d_E = c->d_Q = nullptr;
    c->d_W32 = c->d_U32 = nullptr;
    c->d_gemm = nullptr;
    c->d_copy = nullptr;
    c->d_oz_as = c->d_oz_bs = nullptr;
    c->d_oz_ea = c->d_oz_eb = nullptr;
    c->d_oz = nullptr;
    if (c->h_gemm) cudaFreeHost(c->h_gemm);
    c->h_gemm = nullptr;
    if (c->h_copy) cudaFreeHost(c->h_copy);
    c->h_copy = nullptr;
    c->d_desc = nullptr;
    c->d_cta = nullptr;
    c->d_sync = nullptr;
    c->d_sweeps = nullptr;
    c->d_pre_ok = nullptr;
    if (c->h_desc) cudaFreeHost(c->h_desc);
    if (c->h_cta) cudaFreeHost(c->h_cta);
    c->h_desc = nullptr;
    c->h_cta = nullptr;
    c->slots = 0;
    return MPDO_OK;
}

}  // namespace mpdo

namespace {

int alloc_slots(mpdo_ctx* c, int want) {
    release_slots(c);
    const size_t mat = (size_t)c->ld * c->ld;
    size_t per_slot_bytes = (3 * mat + (size_t)c->cap * c->ld + 2 * c->ld) * sizeof(double);
    if (c->mixed) {
        c->oz_slot_bytes = oz_slice_bytes(c->ld, c->ld, c->oz_bf16);
        per_slot_bytes += 3 * mat * sizeof(double) + 2 * mat * sizeof(float) + 2 * c->oz_slot_bytes +
                          2 * oz_exp_ints(c->ld) * sizeof(int);
    }
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = free_b / 2;
    int s = std::max(1, std::min(want, (int)std::min<size_t>(budget / per_slot_bytes, 1 << 20)));
    if (c->cfg.max_slots > 0) s = std::min(s, c->cfg.max_slots);
    s = std::min(s, c->jacobi_resident);   // every op of a chunk needs at least one co-resident Jacobi CTA
    if ((size_t)s * per_slot_bytes > free_b) return fail(MPDO_ENOMEM, "not enough device memory for one op slot");
    c->slots = s;
    CU(dalloc(&c->d_thetap, (size_t)s * mat));
    CU(dalloc(&c->d_W, (size_t)s * mat));
    CU(dalloc(&c->d_Z, (size_t)s * mat));
    CU(dalloc(&c->d_Yk, (size_t)s * c->cap * c->ld));
    CU(dalloc(&c->d_snorm, (size_t)s * 2 * c->ld));
    CU(dalloc(&c->d_sweeps, (size_t)s));
    CU(dalloc(&c->d_pre_ok, (size_t)s));
    c->h_sweeps.assign(s, 0);
    CU(dalloc(&c->d_desc, (size_t)s));
    const int gcap = std::max(std::max(c->jacobi_resident, c->qr_resident), s);
    CU(dalloc(&c->d_cta, (size_t)3 * (2 * gcap + s)));
    CU(dalloc(&c->d_sync, jacobi_sync_words(s)));
    CU(cudaMallocHost((void**)&c->h_desc, sizeof(OpDesc) * s));
    CU(cudaMallocHost((void**)&c->h_cta, sizeof(int) * 3 * (2 * gcap + s)));
    CU(dalloc(&c->d_copy, (size_t)4 * s));
    CU(cudaMallocHost((void**)&c->h_copy, sizeof(Copy2D) * 4 * s));
    if (c->mixed) {
        CU(dalloc(&c->d_W0, (size_t)s * mat));
        CU(dalloc(&c->d_E, (size_t)s * mat));
        CU(dalloc(&c->d_Q, (size_t)s * mat));
        CU(dalloc(&c->d_W32, (size_t)s * mat));
        CU(dalloc(&c->d_U32, (size_t)s * mat));
        CU(dalloc(&c->d_oz_as, (size_t)s * c->oz_slot_bytes));
        CU(dalloc(&c->d_oz_bs, (size_t)s * c->oz_slot_bytes));
        CU(dalloc(&c->d_oz_ea, (size_t)s * oz_exp_ints(c->ld)));
        CU(dalloc(&c->d_oz_eb, (size_t)s * oz_exp_ints(c->ld)));
        CU(dalloc(&c->d_oz, (size_t)s));
    }
    return MPDO_OK;
}

}  // namespace

namespace mpdo {

void prof_collect(mpdo_ctx* c, int k, double flops, int kernels) {
    if (!c->prof) return;
    float ms = 0.0f;
    if (cudaEventSynchronize(c->ev[2 * k + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]) == cudaSuccess)
        c->prof_ms[k] += ms;
    c->prof_launch[k] += kernels;
    c->prof_flops[k] += flops;
}

int check_status_code(mpdo_ctx* c) {
    std::vector<int> st(c->B);
    CU(cudaMemcpyAsync(st.data(), c->d_status, sizeof(int) * c->B, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    int any = 0;
    for (int v : st) any |= v;
    if (any & MPDO_ST_CAPACITY) return fail(MPDO_ECAPACITY, "a Jacobi block size did not fit its kernel");
    if (any & MPDO_ST_TIMEOUT) return fail(MPDO_ETIMEOUT, "a device-side wait timed out");
    if (any & MPDO_ST_NONFINITE) return fail(MPDO_ENONFINITE, "non-finite values in some instance");
    if (any & MPDO_ST_NOCONV) return fail(MPDO_ENOCONV, "Jacobi SVD hit its sweep limit in some instance");
    return MPDO_OK;
}

int plan_jacobi(mpdo_ctx* c, const OpDesc* h, int nops, bool fp32, int* hbase, int& total) {
    const int R = c->jacobi_resident;
    std::vector<double> work(nops);
    double wsum = 0.0;
    for (int s = 0; s < nops; ++s) {
        work[s] = (double)h[s].c * h[s].c * (double)h[s].L;
        wsum += work[s];
    }
    std::vector<int> G(nops, 1);
    total = 0;
    for (int s = 0; s < nops; ++s) {
        const OpDesc& d = h[s];
        const int pairs = jacobi_pairs_per_round(d.c, fp32 ? d.jb32 : d.jb);
        int g = (int)std::floor((double)R * work[s] / std::max(wsum, 1.0));
        g = std::max(1, std::min(pairs, g));
        const int passes = (pairs + g - 1) / g;      // block pairs per CTA per round
        g = (pairs + passes - 1) / passes;           // fewest CTAs with that many passes
        G[s] = g;
        total += g;
    }
    while (total > R) {   // trim the largest groups until everything is co-resident
        int arg = (int)(std::max_element(G.begin(), G.end()) - G.begin());
        if (G[arg] <= 1) return fail(MPDO_ECAPACITY, "more ops in flight than co-resident Jacobi CTAs");
        G[arg]--;
        total--;
    }
    int t = 0;
    for (int s = 0; s < nops; ++s) {
        hbase[2 * total + s] = G[s];
        for (int g = 0; g < G[s]; ++g, ++t) {
            hbase[t] = s;
            hbase[total + t] = g;
        }
    }
    return MPDO_OK;
}

std::vector<Item> layer_items(mpdo_ctx* c, int li) {
    std::vector<int> order(c->B);
    for (int b = 0; b < c->B; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return c->chi_max[x] > c->chi_max[y]; });
    std::vector<Item> items;
    for (int b : order)
        for (int i = 0; i < (int)c->layers[li].size(); ++i) items.push_back(Item{b, li, i});
    return items;
}

int chunk_ops(mpdo_ctx* c) {
    const auto mm = std::minmax_element(c->chi_max.begin(), c->chi_max.end());
    if (*mm.first == *mm.second) return c->slots;
    return std::max(1, std::min(c->slots, std::max(16, c->jacobi_resident / 4)));
}

void fill_desc(mpdo_ctx* c, const Item& it, int s, OpDesc& d) {
    const int N = c->N, cap = c->cap, ld = c->ld;
    const size_t mat = (size_t)ld * ld;
    const Op& op = c->layers[it.layer][it.idx];
    const int b = it.b, p = op.p;
    const int* dm = &c->h_dims[(size_t)b * (N + 1)];
    d = OpDesc{};
    d.b = b;
    d.op = c->layer_op0[it.layer] + it.idx;
    d.p = p;
    d.cl = dm[p];
    d.cm = dm[p + 1];
    d.cr = dm[p + 2];
    d.m = 4 * d.cl;
    d.n = 4 * d.cr;
    d.transposed = 0;                 // the QR step leaves min(m, n) rows of length n
    d.c = std::min(d.m, d.n);
    d.L = d.n;
    d.chi_max = c->chi_max[b];
    d.cutoff = c->cutoff[b];
    d.G = c->d_gates + ((size_t)b * c->n_ops + d.op) * 256;
    d.A = site_v(c, b, p);
    d.B = site_v(c, b, p + 1);
    d.site_f32 = sites_f32(c);
    d.lam_left = p > 0 ? c->d_lam + ((size_t)b * N + (p - 1)) * cap : nullptr;
    d.lam_out = c->d_lam + ((size_t)b * N + p) * cap;
    d.thetap = c->d_thetap + (size_t)s * mat;
    d.W = c->d_W + (size_t)s * mat;
    d.Z = nullptr;
    d.Acm = c->d_Z + (size_t)s * mat;
    d.Yk = c->d_Yk + (size_t)s * cap * ld;
    d.snorm = c->d_snorm + (size_t)s * 2 * ld;
    d.k_out = c->d_dims + (size_t)b * (N + 1) + p + 1;
    d.status = c->d_status + b;
    d.max_disc = c->d_maxdisc + b;
    d.rank_log = nullptr;
    d.jb = tuned_block_rows(c, d.cl, d.cr, false, jacobi_block_rows(d.L, d.c, 8));
    d.jb32 = tuned_block_rows(c, d.cl, d.cr, true, jacobi_block_rows_f32(d.L, d.c));
    d.sweeps_out = c->d_sweeps + s;
    d.pre_ok = c->mixed ? c->d_pre_ok + s : nullptr;
    d.forced_k = 0;
    d.full_svd = c->full_svd ? 1 : 0;
    d.tape_V = nullptr;
    d.tape_s = nullptr;
    d.W0 = c->mixed ? c->d_W0 + (size_t)s * mat : d.W;
    d.W32 = c->mixed ? c->d_W32 + (size_t)s * mat : nullptr;
    d.U32 = c->mixed ? c->d_U32 + (size_t)s * mat : nullptr;
    d.E = c->mixed ? c->d_E + (size_t)s * mat : nullptr;
    d.Q = c->mixed ? c->d_Q + (size_t)s * mat : nullptr;
    d.Zinit = nullptr;
    d.oz_as = c->mixed ? c->d_oz_as + (size_t)s * c->oz_slot_bytes : nullptr;
    d.oz_bs = c->mixed ? c->d_oz_bs + (size_t)s * c->oz_slot_bytes : nullptr;
    d.oz_ea = c->mixed ? c->d_oz_ea + (size_t)s * oz_exp_ints(ld) : nullptr;
    d.oz_eb = c->mixed ? c->d_oz_eb + (size_t)s * oz_exp_ints(ld) : nullptr;
}

int run_chunk(mpdo_ctx* c, const std::vector<Item>& items, int step, const int* forced, const TapeSlot* tape,
              bool log_ranks) {
    const int nops = (int)items.size();
    const int N = c->N, cap = c->cap, ld = c->ld;
    std::vector<double> work(nops), qwork(nops);
    for (int s = 0; s < nops; ++s) {
        const Item& it = items[s];
        OpDesc& d = c->h_desc[s];
        fill_desc(c, it, s, d);
        int fk = forced ? forced[s] : 0;
        if (!forced && step < c->forced_steps)
            fk = c->forced[((size_t)d.b * c->forced_steps + step) * c->n_ops + d.op];
        d.forced_k = fk;
        d.tape_V = tape ? tape[s].V : nullptr;
        if (tape) d.full_svd = 1;
        d.tape_s = tape ? tape[s].s : nullptr;
        work[s] = (double)d.c * d.c * (double)d.L;
        qwork[s] = (double)d.m * d.n * d.c;
    }
    CU(cudaMemcpyAsync(c->d_desc, c->h_desc, sizeof(OpDesc) * nops, cudaMemcpyHostToDevice, c->st));
    if (tape) {
        // inputs of every op (sites p, p+1, lambda_{p-1}) before the merge
        // overwrites them, and Theta' after it
        Copy2D* hc = c->h_copy;
        int nc = 0, max_rows = 1;
        for (int s = 0; s < nops; ++s) {
            const OpDesc& d = c->h_desc[s];
            // (the gradient runs on FP64 site storage only)
            hc[nc++] = Copy2D{static_cast<const double*>(d.A), tape[s].A, 4 * d.cl, d.cm, cap, d.cm, 1.0};
            hc[nc++] = Copy2D{static_cast<const double*>(d.B), tape[s].B, 4 * d.cm, d.cr, cap, d.cr, 1.0};
            if (d.lam_left) hc[nc++] = Copy2D{d.lam_left, tape[s].lam, 1, d.cl, cap, d.cl, 1.0};
            max_rows = std::max(max_rows, 4 * std::max(d.cl, d.cm));
        }
        for (int s = 0; s < nops; ++s) {
            const OpDesc& d = c->h_desc[s];
            hc[nc + s] = Copy2D{d.thetap, tape[s].thetap, d.m, d.n, ld, d.n, 1.0};
        }
        CU(cudaMemcpyAsync(c->d_copy, hc, sizeof(Copy2D) * (nc + nops), cudaMemcpyHostToDevice, c->st));
        CU(launch_copy2d(c->d_copy, nc, max_rows, c->st));
    }
    double fl_merge = 0.0, fl_svd = 0.0;
    for (int s = 0; s < nops; ++s) {
        const OpDesc& d = c->h_desc[s];
        fl_merge += 32.0 * d.cl * d.cm * d.cr + 512.0 * d.cl * d.cr;
        const double nn = 4.0 * std::max(d.cl, d.cr);
        fl_svd += 21.0 * nn * nn * nn;
    }
    const unsigned long long timeout_ns = (unsigned long long)c->cfg.barrier_timeout_ms * 1000000ull;
    ProfScope p_merge(c, K_MERGE);
    if (c->mixed) {
        CU(launch_oz_ops(c->d_desc, nops, OZ_MERGE, c->d_oz, cap, c->oz_bf16, timeout_ns, c->st));
        CU(launch_gate_weight(c->d_desc, nops, cap, c->st));
    } else {
        CU(launch_merge_gate(c->d_desc, nops, cap, c->st));
    }
    p_merge.stop();
    if (tape) {
        int nc = 0, max_rows = 1;
        for (int s = 0; s < nops; ++s) {
            const OpDesc& d = c->h_desc[s];
            nc += 2 + (d.lam_left ? 1 : 0);
            max_rows = std::max(max_rows, d.m);
        }
        CU(launch_copy2d(c->d_copy + nc, nops, max_rows, c->st));
    }

    const int gcap = std::max(std::max(c->jacobi_resident, c->qr_resident), c->slots);
    double qr_flops_chunk = 0.0;
    int qr_kernels_chunk = 1;
    // Jacobi launch plan: share the co-resident CTAs among the ops in
    // proportion to their work; h_cta/d_cta hold [op of each CTA | rank | CTAs per op]
    auto plan = [&](bool fp32, int* hbase, int& total) -> int {
        return plan_jacobi(c, c->h_desc, nops, fp32, hbase, total);
    };
    auto run_jacobi = [&](bool fp32, int slot) -> int {
        int total = 0;
        int* hbase = c->h_cta + (size_t)slot * (2 * gcap + c->slots);
        int* dbase = c->d_cta + (size_t)slot * (2 * gcap + c->slots);
        int rc = plan(fp32, hbase, total);
        if (rc) return rc;
        CU(cudaMemcpyAsync(dbase, hbase, sizeof(int) * (2 * total + nops), cudaMemcpyHostToDevice, c->st));
        CU(cudaMemsetAsync(c->d_sync, 0, sizeof(unsigned) * jacobi_sync_words(nops), c->st));
        CU(launch_jacobi(c->d_desc, nops, dbase, dbase + total, dbase + 2 * total, c->d_sync, total,
                         fp32 ? kMaxSweepsCap / 2 : c->cfg.jacobi_max_sweeps, fp32 ? 0.0 : fp64_jacobi_tol(c),
                         timeout_ns, ld, fp32, c->st, precond_rho(c)));
        return MPDO_OK;
    };
    CU(cudaMemsetAsync(c->d_sweeps, 0, sizeof(int) * nops, c->st));
    // Householder QR of every theta~ (R's rows go to W0)
    {
        const int R = c->qr_resident;
        const int QW = qr_threads() / 32;
        double wsum = 0.0;
        for (double w : qwork) wsum += w;
        std::vector<int> G(nops, 1);
        int total = 0;
        for (int s = 0; s < nops; ++s) {
            const OpDesc& d = c->h_desc[s];
            const int need = std::max(1, (d.n + QW - 1) / QW);
            int g = (int)std::floor((double)R * qwork[s] / std::max(wsum, 1.0));
            G[s] = std::max(1, std::min(need, g));
            total += G[s];
        }
        while (total > R) {
            int arg = (int)(std::max_element(G.begin(), G.end()) - G.begin());
            if (G[arg] <= 1) return fail(MPDO_ECAPACITY, "more ops in flight than co-resident QR CTAs");
            G[arg]--;
            total--;
        }
        int* hbase = c->h_cta + (size_t)2 * (2 * gcap + c->slots);
        int* dbase = c->d_cta + (size_t)2 * (2 * gcap + c->slots);
        // fault injection (host side): leave out the last CTA of the first op that
        // has two or more, while its group still counts it, so that the op's first
        // barrier cannot complete and its CTAs give up after barrier_timeout_ms
        int drop_op = -1;
        if (c->inject == MPDO_FAULT_DROP_CTA)
            for (int s = 0; s < nops && drop_op < 0; ++s)
                if (G[s] >= 2) drop_op = s;
        const int launched = total - (drop_op >= 0 ? 1 : 0);
        int t = 0;
        for (int s = 0; s < nops; ++s) {
            hbase[2 * launched + s] = G[s];
            const int run = G[s] - (s == drop_op ? 1 : 0);
            for (int g = 0; g < run; ++g, ++t) {
                hbase[t] = s;
                hbase[launched + t] = g;
            }
        }
        if (drop_op >= 0) c->inject = 0;
        total = launched;
        double fl_qr = 0.0;
        for (int s = 0; s < nops; ++s) {
            const OpDesc& d = c->h_desc[s];
            fl_qr += 4.0 * d.m * d.n * d.c - 2.0 * (d.m + d.n) * d.c * d.c + 4.0 / 3.0 * d.c * d.c * d.c;
        }
        qr_flops_chunk = fl_qr;
        if (c->mixed && c->cfg.qr_blocked && qrb_fits(cap)) {
            // mixed path: blocked QR, trailing updates on the tensor cores
            int r_max = 1;
            for (int s = 0; s < nops; ++s) r_max = std::max(r_max, c->h_desc[s].c);
            ProfScope p_qr(c, K_QR);
            CU(launch_qr_blocked(c->d_desc, nops, cap, c->d_oz, c->oz_bf16, timeout_ns, c->st, r_max));
            p_qr.stop();
            qr_kernels_chunk = qrb_kernels(cap, r_max);
        } else {
            CU(cudaMemcpyAsync(dbase, hbase, sizeof(int) * (2 * total + nops), cudaMemcpyHostToDevice, c->st));
            CU(cudaMemsetAsync(c->d_sync, 0, sizeof(unsigned) * jacobi_sync_words_per_op() * nops, c->st));
            ProfScope p_qr(c, K_QR);
            CU(launch_qr(c->d_desc, dbase, dbase + total, dbase + 2 * total, c->d_sync, total, timeout_ns, ld,
                         c->st));
            p_qr.stop();
        }
    }
    double fl_gemm = 0.0;
    if (c->mixed) {
        // FP32 preconditioning Jacobi on (W32 | U32)
        ProfScope p_j32(c, K_JACOBI32);
        int rc = run_jacobi(true, 1);
        if (rc) return rc;
        p_j32.stop();
        // E = U U^T - I, Q = U - E U / 2 (one Newton-Schulz step), W = Q W0, all
        // FP64-accurate tensor-core products (oz_gemm.cu)
        for (int s = 0; s < nops; ++s) {
            const OpDesc& d = c->h_desc[s];
            fl_gemm += 2.0 * d.c * d.c * d.c * 2 + 2.0 * d.c * d.c * d.L;
        }
        ProfScope p_gemm(c, K_GEMM);
        CU(launch_oz_ops(c->d_desc, nops, OZ_E, c->d_oz, cap, c->oz_bf16, timeout_ns, c->st));
        CU(launch_oz_ops(c->d_desc, nops, OZ_Q, c->d_oz, cap, c->oz_bf16, timeout_ns, c->st));
        CU(launch_oz_ops(c->d_desc, nops, OZ_W, c->d_oz, cap, c->oz_bf16, timeout_ns, c->st));
        p_gemm.stop();
    }
    ProfScope p_jac(c, K_JACOBI);
    {
        int rc = run_jacobi(false, 0);
        if (rc) return rc;
    }
    p_jac.stop();
    ProfScope p_tr(c, K_TRUNC);
    CU(launch_truncate(c->d_desc, nops, cap, c->st));
    p_tr.stop();
    ProfScope p_rec(c, K_RECON);
    if (c->mixed)
        CU(launch_oz_ops(c->d_desc, nops, OZ_RECON, c->d_oz, cap, c->oz_bf16, timeout_ns, c->st));
    else
        CU(launch_reconstruct(c->d_desc, nops, cap, c->st));
    p_rec.stop();
    // new bond dimensions back to the host (the next chunk's shapes depend on them)
    CU(cudaMemcpyAsync(c->h_dims.data(), c->d_dims, sizeof(int) * c->h_dims.size(), cudaMemcpyDeviceToHost,
                       c->st));
    if (c->prof) CU(cudaMemcpyAsync(c->h_sweeps.data(), c->d_sweeps, sizeof(int) * nops, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (c->prof) {
        int crit = 0, crit32 = 0;
        for (int s = 0; s < nops; ++s) {
            c->prof_sweeps += c->h_sweeps[s] & 0xffff;
            c->prof_sweeps32 += c->h_sweeps[s] >> 16;
            c->prof_svds += 1;
            crit = std::max(crit, c->h_sweeps[s] & 0xffff);
            crit32 = std::max(crit32, c->h_sweeps[s] >> 16);
        }
        c->prof_crit += crit;
        c->prof_crit32 += crit32;
        c->prof_chunks += 1;
    }
    double fl_rec = 0.0;
    for (int s = 0; s < nops; ++s) {
        const OpDesc& d = c->h_desc[s];
        fl_rec += 32.0 * d.cl * d.cr * c->h_dims[(size_t)d.b * (N + 1) + c->layers[items[s].layer][items[s].idx].p + 1];
    }
    // kernels per stage: a tensor-core product is three (operand set-up,
    // slicing, slice products), the merge adds the gate/weight kernel
    prof_collect(c, K_MERGE, fl_merge, c->mixed ? 4 : 1);
    prof_collect(c, K_QR, qr_flops_chunk, qr_kernels_chunk);
    prof_collect(c, K_JACOBI, fl_svd, 1);
    if (c->mixed) {
        prof_collect(c, K_JACOBI32, 0.0, 1);
        prof_collect(c, K_GEMM, fl_gemm, 9);
    }
    prof_collect(c, K_TRUNC, 0.0, 1);
    prof_collect(c, K_RECON, fl_rec, c->mixed ? 3 : 1);
    for (int s = 0; s < nops && log_ranks; ++s) {
        const Item& it = items[s];
        const Op& op = c->layers[it.layer][it.idx];
        const int k = c->h_dims[(size_t)it.b * (N + 1) + op.p + 1];
        const size_t per_b = (size_t)c->rank_steps * c->n_ops;
        c->rank_log[(size_t)it.b * per_b + (size_t)step * c->n_ops + c->layer_op0[it.layer] + it.idx] = k;
    }
    return MPDO_OK;
}

int normalize_trace(mpdo_ctx* c) {
    ProfScope p_trace(c, K_TRACE);
    CU(launch_trace_normalize(c->d_sites, sites_f32(c), c->d_dims, c->N, c->B, c->cap, c->cfg.force_trace, c->d_trace,
                              c->d_status, c->st));
    p_trace.stop();
    prof_collect(c, K_TRACE, 0.0, 1);
    return MPDO_OK;
}

}  // namespace mpdo

namespace {

int validate_model(mpdo_ctx* c, const mpdo_model* m) {
    const int N = c->N, B = c->B;
    if (!m) return fail(MPDO_EINVAL, "model is NULL");
    if (!m->h_x || !m->h_z || !m->g0 || !m->g2 || !m->J || !m->bond_i || !m->bond_j || !m->chi_max || !m->cutoff)
        return fail(MPDO_EINVAL, "model: a required array is NULL");
    if (m->n_bonds < 1) return fail(MPDO_EINVAL, "model: n_bonds must be >= 1");
    for (int b = 0; b < B; ++b) {
        if (m->chi_max[b] < 1) return fail(MPDO_EINVAL, "model: chi_max must be >= 1");
        if (m->chi_max[b] > c->cap) return fail(MPDO_ECAPACITY, "model: chi_max exceeds chi_cap");
        if (!(m->cutoff[b] >= 0.0) || !std::isfinite(m->cutoff[b]))
            return fail(MPDO_EINVAL, "model: cutoff must be finite and >= 0");
        for (int q = 0; q < N; ++q) {
            const size_t i = (size_t)b * N + q;
            const double g1 = m->g1 ? m->g1[i] : 0.0;
            if (!(m->g0[i] >= 0.0) || !(m->g2[i] >= 0.0) || !(g1 >= 0.0))
                return fail(MPDO_EINVAL, "model: rates g0, g1, g2 must be >= 0");
            const double hy = m->h_y ? m->h_y[i] : 0.0;
            if (!std::isfinite(m->h_x[i]) || !std::isfinite(hy) || !std::isfinite(m->h_z[i]) ||
                !std::isfinite(m->g0[i]) || !std::isfinite(m->g2[i]) || !std::isfinite(g1))
                return fail(MPDO_EINVAL, "model: non-finite on-site parameter");
        }
        for (int k = 0; k < m->n_bonds; ++k) {
            const size_t i = (size_t)b * m->n_bonds + k;
            if (!std::isfinite(m->J[i]) || (m->Jz && !std::isfinite(m->Jz[i])))
                return fail(MPDO_EINVAL, "model: non-finite coupling");
        }
    }
    if (m->init_pauli) {
        if (strlen(m->init_pauli) != (size_t)(2 * N))
            return fail(MPDO_EINVAL, "model: init_pauli must have 2N characters");
        for (int q = 0; q < N; ++q) {
            const char s = m->init_pauli[2 * q], a = m->init_pauli[2 * q + 1];
            if ((s != '+' && s != '-') || !strchr("xyzXYZ", a))
                return fail(MPDO_EINVAL, "model: init_pauli entries must be +x,-x,+y,-y,+z,-z");
        }
    }
    return MPDO_OK;
}

int pauli_comp(char ch) {
    switch (ch) {
        case 'I': case 'i': return 0;
        case 'X': case 'x': return 1;
        case 'Y': case 'y': return 2;
        case 'Z': case 'z': return 3;
        default: return -1;
    }
}

}  // namespace

extern "C" {

const char* mpdo_last_error(void) { return g_err.c_str(); }

int mpdo_config_default(mpdo_config* cfg) {
    if (!cfg) return fail(MPDO_EINVAL, "cfg is NULL");
    memset(cfg, 0, sizeof(*cfg));
    cfg->batch = 1;
    cfg->precision = MPDO_FP64;
    cfg->storage = MPDO_STORE_F64;
    cfg->trotter_order = 2;
    cfg->force_trace = 1;
    cfg->jacobi_max_sweeps = 100;
    cfg->jacobi_tol = 0.0;
    cfg->barrier_timeout_ms = 4000;
    cfg->max_slots = 0;
    cfg->device = -1;
    return MPDO_OK;
}

int mpdo_init(mpdo_ctx** out, const mpdo_config* cfg, void* cuda_stream) {
    if (!out || !cfg) return fail(MPDO_EINVAL, "out and cfg must not be NULL");
    *out = nullptr;
    if (cfg->n_qubits < 3) return fail(MPDO_EINVAL, "n_qubits must be >= 3");
    if (cfg->batch < 1) return fail(MPDO_EINVAL, "batch must be >= 1");
    if (!(cfg->precond_rho <= 1.0)) return fail(MPDO_EINVAL, "precond_rho must be a number <= 1");
    if (cfg->chi_cap < 1 || cfg->chi_cap > kMaxChi) return fail(MPDO_EINVAL, "chi_cap must be in [1, 512]");
    if (cfg->precision != MPDO_FP64 && cfg->precision != MPDO_MIXED_TF32 && cfg->precision != MPDO_MIXED_BF16X3)
        return fail(MPDO_EINVAL, "precision must be MPDO_FP64, MPDO_MIXED_TF32 or MPDO_MIXED_BF16X3");
    if (cfg->storage != MPDO_STORE_F64 && cfg->storage != MPDO_STORE_F32)
        return fail(MPDO_EINVAL, "storage must be MPDO_STORE_F64 or MPDO_STORE_F32");
    if (cfg->trotter_order != 2 && cfg->trotter_order != 4)
        return fail(MPDO_EINVAL, "trotter_order must be 2 or 4 (symmetric compositions have even order)");
    if (cfg->jacobi_max_sweeps < 1 || cfg->jacobi_max_sweeps > kMaxSweepsCap)
        return fail(MPDO_EINVAL, "jacobi_max_sweeps must be in [1, 128]");
    if (cfg->barrier_timeout_ms < 1) return fail(MPDO_EINVAL, "barrier_timeout_ms must be >= 1");
    int dev = cfg->device;
    if (dev < 0) CU(cudaGetDevice(&dev));
    CU(cudaSetDevice(dev));
    mpdo_ctx* c = new (std::nothrow) mpdo_ctx();
    if (!c) return fail(MPDO_ENOMEM, "host allocation failed");
    c->dev = dev;
    c->mixed = cfg->precision != MPDO_FP64;
    c->oz_bf16 = cfg->precision == MPDO_MIXED_BF16X3;
    c->cfg = *cfg;
    c->st = (cudaStream_t)cuda_stream;
    c->N = cfg->n_qubits;
    c->B = cfg->batch;
    c->cap = cfg->chi_cap;
    c->ld = 4 * cfg->chi_cap;
    const int N = c->N, B = c->B;
    auto bail = [&](int code) {
        free_all(c);
        delete c;
        return code;
    };
    cudaError_t e;
    if ((e = dalloc(&c->d_sites, ((size_t)B * N * site_elems(c) * site_esize(c) + 7) / 8)) != cudaSuccess ||
        (e = dalloc(&c->d_lam, (size_t)B * N * c->cap)) != cudaSuccess ||
        (e = dalloc(&c->d_dims, (size_t)B * (N + 1))) != cudaSuccess ||
        (e = dalloc(&c->d_status, (size_t)B)) != cudaSuccess ||
        (e = dalloc(&c->d_maxdisc, (size_t)B)) != cudaSuccess ||
        (e = dalloc(&c->d_trace, (size_t)B)) != cudaSuccess ||
        (e = dalloc(&c->d_envL, (size_t)B * (N + 1) * c->cap)) != cudaSuccess ||
        (e = dalloc(&c->d_envR, (size_t)B * (N + 1) * c->cap)) != cudaSuccess ||
        (e = dalloc(&c->d_full, (size_t)B * N * N)) != cudaSuccess ||
        (e = dalloc(&c->d_wstack, two_stack_doubles(N, B, c->cap))) != cudaSuccess ||
        (e = dalloc(&c->d_part, two_part_doubles(N, B, c->cap))) != cudaSuccess ||
        (e = dalloc(&c->d_one_a, (size_t)B * N * 4)) != cudaSuccess ||
        (e = dalloc(&c->d_one_b, (size_t)B * N)) != cudaSuccess ||
        (e = dalloc(&c->d_out, (size_t)B * N * N)) != cudaSuccess ||
        (e = dalloc(&c->d_q, (size_t)N)) != cudaSuccess ||
        (e = dalloc(&c->d_pairs, (size_t)3 * N * N)) != cudaSuccess ||
        (e = dalloc(&c->d_need, (size_t)N)) != cudaSuccess) {
        fail(e == cudaErrorMemoryAllocation ? MPDO_ENOMEM : MPDO_ECUDA,
             std::string("device allocation: ") + cudaGetErrorString(e));
        return bail(e == cudaErrorMemoryAllocation ? MPDO_ENOMEM : MPDO_ECUDA);
    }
    if ((e = oz_prepare()) != cudaSuccess || (e = qrb_prepare()) != cudaSuccess) {
        fail(MPDO_ECUDA, std::string("tensor-core kernel set-up: ") + cudaGetErrorString(e));
        return bail(MPDO_ECUDA);
    }
    if ((e = qr_max_resident(&c->qr_resident)) != cudaSuccess || c->qr_resident < 1) {
        fail(MPDO_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
        return bail(MPDO_ECUDA);
    }
    if ((e = jacobi_max_resident(&c->jacobi_resident)) != cudaSuccess || c->jacobi_resident < 1) {
        fail(MPDO_ECUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
        return bail(MPDO_ECUDA);
    }
    for (auto& ev : c->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
            fail(MPDO_ECUDA, std::string("event create: ") + cudaGetErrorString(e));
            return bail(MPDO_ECUDA);
        }
    c->h_dims.assign((size_t)B * (N + 1), 1);
    *out = c;
    return MPDO_OK;
}

int mpdo_build_gates(mpdo_ctx* c, const mpdo_model* m, double dt) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    CU(cudaSetDevice(c->dev));
    if (!std::isfinite(dt)) return fail(MPDO_EINVAL, "dt must be finite");
    int rc = validate_model(c, m);
    if (rc) return rc;
    const int N = c->N, B = c->B, nb = m->n_bonds;
    std::vector<int> bi(m->bond_i, m->bond_i + nb), bj(m->bond_j, m->bond_j + nb);
    std::vector<Layer> layers;
    std::vector<double> weights;
    std::string err = build_schedule(N, bi, bj, layers, weights);
    if (!err.empty()) return fail(MPDO_EINVAL, "bond graph: " + err);
    if (c->cfg.trotter_order == 4) {
        // Suzuki's symmetric triple jump: S2(w1 dt) S2(w0 dt) S2(w1 dt), w0 + 2 w1 = 1
        const double w1 = 1.0 / (2.0 - std::cbrt(2.0)), w0 = 1.0 - 2.0 * w1;
        std::vector<Layer> four;
        for (double w : {w1, w0, w1})
            for (Layer L : layers) {
                for (auto& o : L) o.frac *= w;
                four.push_back(L);
            }
        layers.swap(four);
    }
    c->layers = layers;
    c->weights = weights;
    c->nb = nb;
    c->layer_op0.clear();
    c->n_ops = c->n_swaps = c->max_layer = 0;
    for (auto& L : layers) {
        c->layer_op0.push_back(c->n_ops);
        c->n_ops += (int)L.size();
        c->max_layer = std::max(c->max_layer, (int)L.size());
        for (auto& o : L) c->n_swaps += o.kind;
    }
    c->chi_max.assign(m->chi_max, m->chi_max + B);
    c->cutoff.assign(m->cutoff, m->cutoff + B);
    // parameters
    const int P = 6 * N + 2 * nb;
    std::vector<double> hp((size_t)B * P, 0.0);
    for (int b = 0; b < B; ++b) {
        double* dst = &hp[(size_t)b * P];
        for (int q = 0; q < N; ++q) {
            const size_t i = (size_t)b * N + q;
            dst[0 * N + q] = m->h_x[i];
            dst[1 * N + q] = m->h_y ? m->h_y[i] : 0.0;
            dst[2 * N + q] = m->h_z[i];
            dst[3 * N + q] = m->g0[i];
            dst[4 * N + q] = m->g1 ? m->g1[i] : 0.0;
            dst[5 * N + q] = m->g2[i];
        }
        for (int k = 0; k < nb; ++k) {
            dst[6 * N + k] = m->J[(size_t)b * nb + k];
            dst[6 * N + nb + k] = m->Jz ? m->Jz[(size_t)b * nb + k] : 0.0;
        }
    }
    std::vector<GateSpec> specs;
    specs.reserve((size_t)B * c->n_ops);
    for (int b = 0; b < B; ++b)
        for (auto& L : layers)
            for (auto& o : L)
                specs.push_back(GateSpec{b, o.kind, o.qa, o.qb, o.bond, o.frac * dt, weights[o.qa], weights[o.qb]});
    // (re)allocate graph-sized buffers
    if (c->d_params) cudaFree(c->d_params);
    if (c->d_gates) cudaFree(c->d_gates);
    if (c->d_specs) cudaFree(c->d_specs);
    c->d_params = nullptr;
    c->d_gates = nullptr;
    c->d_specs = nullptr;
    CU(dalloc(&c->d_params, hp.size()));
    CU(dalloc(&c->d_gates, (size_t)B * c->n_ops * 256));
    CU(dalloc(&c->d_specs, specs.size()));
    CU(cudaMemcpyAsync(c->d_params, hp.data(), sizeof(double) * hp.size(), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(c->d_specs, specs.data(), sizeof(GateSpec) * specs.size(), cudaMemcpyHostToDevice, c->st));
    CU(launch_build_gates(c->d_specs, (int)specs.size(), N, nb, c->d_params, c->d_gates, c->st));
    const int want = B * c->max_layer;
    if (c->slots < want) {
        rc = alloc_slots(c, want);
        if (rc) return rc;
    }
    // initial product state (Sec. 2.2): site vector (1, +-1 at a)/sqrt2, chi = 1
    const double r2 = 1.0 / std::sqrt(2.0);
    std::vector<double> v0((size_t)B * N * 4, 0.0);
    for (int b = 0; b < B; ++b)
        for (int q = 0; q < N; ++q) {
            double* v = &v0[((size_t)b * N + q) * 4];
            v[0] = r2;
            if (m->init_pauli) {
                const double sg = m->init_pauli[2 * q] == '+' ? 1.0 : -1.0;
                v[pauli_comp(m->init_pauli[2 * q + 1])] += sg * r2;
            } else {
                v[3] += r2;
            }
        }
    CU(cudaMemsetAsync(c->d_sites, 0, site_esize(c) * (size_t)B * N * site_elems(c), c->st));
    CU(cudaMemcpyAsync(c->d_one_a, v0.data(), sizeof(double) * v0.size(), cudaMemcpyHostToDevice, c->st));
    init_product_kernel<<<B, 64, 0, c->st>>>(c->d_sites, sites_f32(c), c->d_one_a, N, c->cap);
    CU(cudaGetLastError());
    std::vector<double> ones((size_t)B * N * c->cap, 1.0);
    CU(cudaMemcpyAsync(c->d_lam, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, c->st));
    c->h_dims.assign((size_t)B * (N + 1), 1);
    CU(cudaMemcpyAsync(c->d_dims, c->h_dims.data(), sizeof(int) * c->h_dims.size(), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemsetAsync(c->d_status, 0, sizeof(int) * B, c->st));
    CU(cudaMemsetAsync(c->d_maxdisc, 0, sizeof(double) * B, c->st));
    CU(cudaMemsetAsync(c->d_trace, 0, sizeof(double) * B, c->st));
    CU(cudaStreamSynchronize(c->st));
    c->built = true;
    ++c->gen;
    ++c->layout;
    c->forced.clear();
    c->forced_steps = 0;
    return MPDO_OK;
}

int mpdo_init_graph_state(mpdo_ctx* c, const int* pairs, int n_pairs) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (n_pairs < 0 || (n_pairs > 0 && !pairs)) return fail(MPDO_EINVAL, "pairs must hold n_pairs >= 0 pairs");
    const int N = c->N, B = c->B;
    for (int k = 0; k < n_pairs; ++k) {
        const int i = pairs[2 * k], j = pairs[2 * k + 1];
        if (i < 0 || j < 0 || i >= N || j >= N || i == j) return fail(MPDO_EINVAL, "pair indices out of range or i == j");
    }
    // |+x> on every qubit: site vector (1, 1, 0, 0) / sqrt2, bond dimensions 1
    const double r2 = 1.0 / std::sqrt(2.0);
    std::vector<double> v0((size_t)B * N * 4, 0.0);
    for (size_t q = 0; q < (size_t)B * N; ++q) v0[4 * q] = v0[4 * q + 1] = r2;
    CU(cudaMemsetAsync(c->d_sites, 0, site_esize(c) * (size_t)B * N * site_elems(c), c->st));
    CU(cudaMemcpyAsync(c->d_one_a, v0.data(), sizeof(double) * v0.size(), cudaMemcpyHostToDevice, c->st));
    init_product_kernel<<<B, 64, 0, c->st>>>(c->d_sites, sites_f32(c), c->d_one_a, N, c->cap);
    CU(cudaGetLastError());
    std::vector<double> ones((size_t)B * N * c->cap, 1.0);
    CU(cudaMemcpyAsync(c->d_lam, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice, c->st));
    c->h_dims.assign((size_t)B * (N + 1), 1);
    CU(cudaMemcpyAsync(c->d_dims, c->h_dims.data(), sizeof(int) * c->h_dims.size(), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemsetAsync(c->d_status, 0, sizeof(int) * B, c->st));
    CU(cudaMemsetAsync(c->d_maxdisc, 0, sizeof(double) * B, c->st));
    CU(cudaStreamSynchronize(c->st));
    ++c->gen;
    if (n_pairs == 0) return MPDO_OK;
    // Pauli-basis superoperators: CZ (rho -> CZ rho CZ, by traces of Pauli products)
    // and SWAP, as 16 x 16 two-site gates G[(a,b), (c,d)]
    using cd = std::complex<double>;
    const cd I(0.0, 1.0);
    const cd P[4][2][2] = {{{1, 0}, {0, 1}}, {{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
    const double czd[4] = {1.0, 1.0, 1.0, -1.0};
    std::vector<double> cz(256, 0.0), sw(256, 0.0);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int cc = 0; cc < 4; ++cc)
                for (int d = 0; d < 4; ++d) {
                    // Tr[(P_a x P_b) CZ (P_c x P_d) CZ] / 4; CZ is diagonal
                    cd tr = 0.0;
                    for (int x = 0; x < 4; ++x)
                        for (int y = 0; y < 4; ++y) {
                            const cd pab = P[a][x >> 1][y >> 1] * P[b][x & 1][y & 1];
                            const cd pcd = P[cc][y >> 1][x >> 1] * P[d][y & 1][x & 1];
                            tr += pab * czd[y] * pcd * czd[x];
                        }
                    cz[(a * 4 + b) * 16 + cc * 4 + d] = tr.real() / 4.0;
                }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) sw[(b * 4 + a) * 16 + a * 4 + b] = 1.0;
    // op list: per pair, swaps bring j next to i, CZ on (i, i+1), swaps back
    std::vector<Layer> L;
    std::vector<int> at(N);
    for (int q = 0; q < N; ++q) at[q] = q;
    auto push = [&](int kind, int p) {
        L.push_back(Layer{Op{kind, p, at[p], at[p + 1], -1, 0.0}});
        if (kind == 1) std::swap(at[p], at[p + 1]);
    };
    for (int k = 0; k < n_pairs; ++k) {
        const int i = std::min(pairs[2 * k], pairs[2 * k + 1]), j = std::max(pairs[2 * k], pairs[2 * k + 1]);
        for (int p = j - 1; p >= i + 1; --p) push(1, p);
        push(0, i);
        for (int p = i + 1; p <= j - 1; ++p) push(1, p);
    }
    const int nops = (int)L.size();
    std::vector<double> hg((size_t)B * nops * 256);
    for (int b = 0; b < B; ++b)
        for (int o = 0; o < nops; ++o)
            std::copy_n((L[o][0].kind == 0 ? cz : sw).data(), 256, hg.data() + ((size_t)b * nops + o) * 256);
    double* d_g = nullptr;
    CU(dalloc(&d_g, hg.size()));
    CU(cudaMemcpyAsync(d_g, hg.data(), sizeof(double) * hg.size(), cudaMemcpyHostToDevice, c->st));
    // run the ops through the step's machinery on the graph-state op list
    std::vector<Layer> keep_layers;
    keep_layers.swap(c->layers);
    std::vector<int> keep_op0;
    keep_op0.swap(c->layer_op0);
    const int keep_n_ops = c->n_ops;
    double* keep_gates = c->d_gates;
    const int keep_forced = c->forced_steps;
    c->layers = L;
    c->layer_op0.resize(nops);
    for (int o = 0; o < nops; ++o) c->layer_op0[o] = o;
    c->n_ops = nops;
    c->d_gates = d_g;
    c->forced_steps = 0;
    int rc = MPDO_OK;
    for (int li = 0; li < nops && rc == MPDO_OK; ++li) {
        const std::vector<Item> items = layer_items(c, li);
        const size_t cs = (size_t)chunk_ops(c);
        for (size_t s0 = 0; s0 < items.size() && rc == MPDO_OK; s0 += cs) {
            std::vector<Item> chunk(items.begin() + s0, items.begin() + std::min(items.size(), s0 + cs));
            rc = run_chunk(c, chunk, 0, nullptr, nullptr, false);
        }
    }
    cudaStreamSynchronize(c->st);
    c->layers.swap(keep_layers);
    c->layer_op0.swap(keep_op0);
    c->n_ops = keep_n_ops;
    c->d_gates = keep_gates;
    c->forced_steps = keep_forced;
    cudaFree(d_g);
    if (rc) return rc;
    return check_status_code(c);
}

int mpdo_trotter_step(mpdo_ctx* c, int n_steps) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (n_steps < 0) return fail(MPDO_EINVAL, "n_steps must be >= 0");
    c->rank_steps = n_steps;
    c->rank_log.assign((size_t)c->B * n_steps * c->n_ops, 0);
    ++c->gen;
    for (int step = 0; step < n_steps; ++step) {
        for (int li = 0; li < (int)c->layers.size(); ++li) {
            const std::vector<Item> items = layer_items(c, li);
            const size_t cs = (size_t)chunk_ops(c);
            for (size_t s0 = 0; s0 < items.size(); s0 += cs) {
                std::vector<Item> chunk(items.begin() + s0, items.begin() + std::min(items.size(), s0 + cs));
                int rc = run_chunk(c, chunk, step, nullptr, nullptr, true);
                if (rc) return rc;
            }
        }
        int rc = normalize_trace(c);
        if (rc) return rc;
    }
    return check_status_code(c);
}

int mpdo_measure_1q(mpdo_ctx* c, const int* qubits, int nq, char comp, double* out, int out_on_device) {
    if (!c || !qubits || !out) return fail(MPDO_EINVAL, "NULL argument");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    const int a = pauli_comp(comp);
    if (a < 0) return fail(MPDO_EINVAL, "comp must be one of I, X, Y, Z");
    if (nq < 0 || nq > c->N) return fail(MPDO_EINVAL, "nq must be in [0, N]");
    for (int k = 0; k < nq; ++k)
        if (qubits[k] < 0 || qubits[k] >= c->N) return fail(MPDO_EINVAL, "qubit index out of range");
    if (nq == 0) return MPDO_OK;
    CU(cudaMemcpyAsync(c->d_q, qubits, sizeof(int) * nq, cudaMemcpyHostToDevice, c->st));
    CU(launch_environments(c->d_sites, sites_f32(c), c->d_dims, c->N, c->B, c->cap, c->d_envL, c->d_envR, c->st));
    double* dst = out_on_device ? out : c->d_out;
    CU(launch_measure_1q(c->d_sites, sites_f32(c), c->d_dims, c->N, c->B, c->cap, c->d_envL, c->d_envR, c->d_q, nq,
                         a, dst, c->st));
    if (!out_on_device) {
        CU(cudaMemcpyAsync(out, c->d_out, sizeof(double) * nq * c->B, cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
    }
    return MPDO_OK;
}

int mpdo_measure_2q(mpdo_ctx* c, const int* pairs, int np, const char comp[2], int connected, double* out,
                    int out_on_device) {
    if (!c || !pairs || !out || !comp) return fail(MPDO_EINVAL, "NULL argument");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    const int ca = pauli_comp(comp[0]), cb = pauli_comp(comp[1]);
    if (ca < 0 || cb < 0) return fail(MPDO_EINVAL, "comp entries must be I, X, Y, Z");
    const int N = c->N, B = c->B;
    if (np < 0 || np > N * N) return fail(MPDO_ECAPACITY, "np must be in [0, N*N]");
    if (np == 0) return MPDO_OK;
    for (int k = 0; k < np; ++k) {
        const int i = pairs[2 * k], j = pairs[2 * k + 1];
        if (i < 0 || j < 0 || i >= N || j >= N || i == j) return fail(MPDO_EINVAL, "pair indices out of range or i == j");
    }
    CU(launch_environments(c->d_sites, sites_f32(c), c->d_dims, N, B, c->cap, c->d_envL, c->d_envR, c->st));
    std::vector<int> allq(N);
    for (int q = 0; q < N; ++q) allq[q] = q;
    CU(cudaMemcpyAsync(c->d_q, allq.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c->st));
    CU(launch_measure_1q(c->d_sites, sites_f32(c), c->d_dims, N, B, c->cap, c->d_envL, c->d_envR, c->d_q, N, ca,
                         c->d_one_a, c->st));
    CU(launch_measure_1q(c->d_sites, sites_f32(c), c->d_dims, N, B, c->cap, c->d_envL, c->d_envR, c->d_q, N, cb,
                         c->d_one_b, c->st));
    double* dst = out_on_device ? out : c->d_out;
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: pairs with i < j; pass 1: pairs with i > j, evaluated as (j, i) with swapped components
        std::vector<int> trip;
        std::vector<unsigned char> need(N, 0);
        for (int k = 0; k < np; ++k) {
            int i = pairs[2 * k], j = pairs[2 * k + 1];
            if ((pass == 0) != (i < j)) continue;
            if (pass == 1) std::swap(i, j);
            trip.push_back(i);
            trip.push_back(j);
            trip.push_back(k);
            need[i] = 1;
        }
        if (trip.empty()) continue;
        const int x = pass == 0 ? ca : cb, y = pass == 0 ? cb : ca;
        CU(cudaMemcpyAsync(c->d_need, need.data(), N, cudaMemcpyHostToDevice, c->st));
        CU(launch_measure_2q(c->d_sites, sites_f32(c), c->d_dims, N, B, c->cap, c->d_envL, c->d_envR, x, y, c->d_need,
                             c->d_wstack, c->d_part, c->d_full, c->st));
        CU(cudaMemcpyAsync(c->d_pairs, trip.data(), sizeof(int) * trip.size(), cudaMemcpyHostToDevice, c->st));
        const double* oa = pass == 0 ? c->d_one_a : c->d_one_b;
        const double* ob = pass == 0 ? c->d_one_b : c->d_one_a;
        CU(launch_gather_2q(c->d_full, oa, ob, c->d_pairs, (int)trip.size() / 3, np, N, B, connected, dst, c->st));
        CU(cudaStreamSynchronize(c->st));   // host vectors above are reused by the next pass
    }
    if (!out_on_device) {
        CU(cudaMemcpyAsync(out, dst, sizeof(double) * (size_t)np * B, cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
    }
    return MPDO_OK;
}

int mpdo_status(mpdo_ctx* c, int* status, double* max_discarded, int* chi, double* trace_before) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    CU(cudaSetDevice(c->dev));
    const int B = c->B, N = c->N;
    if (status) CU(cudaMemcpyAsync(status, c->d_status, sizeof(int) * B, cudaMemcpyDeviceToHost, c->st));
    if (max_discarded) CU(cudaMemcpyAsync(max_discarded, c->d_maxdisc, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st));
    if (trace_before) CU(cudaMemcpyAsync(trace_before, c->d_trace, sizeof(double) * B, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(c->h_dims.data(), c->d_dims, sizeof(int) * c->h_dims.size(), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (chi)
        for (int b = 0; b < B; ++b)
            for (int p = 0; p < N - 1; ++p) chi[(size_t)b * (N - 1) + p] = c->h_dims[(size_t)b * (N + 1) + p + 1];
    return MPDO_OK;
}

int mpdo_set_state(mpdo_ctx* c, int b, const int* dims, const double* tensors) {
    if (!c || !dims || !tensors) return fail(MPDO_EINVAL, "NULL argument");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    const int N = c->N;
    if (b < 0 || b >= c->B) return fail(MPDO_EINVAL, "instance out of range");
    if (dims[0] != 1 || dims[N] != 1) return fail(MPDO_EINVAL, "dims[0] and dims[N] must be 1");
    for (int p = 1; p < N; ++p)
        if (dims[p] < 1 || dims[p] > c->chi_max[b]) return fail(MPDO_ECAPACITY, "bond dimension out of [1, chi_max]");
    // compact rows (l, s) of length cr, copied into rows of length chi_cap
    const size_t es = site_esize(c);
    std::vector<float> f32;
    if (sites_f32(c)) {
        size_t tot = 0;
        for (int p = 0; p < N; ++p) tot += (size_t)dims[p] * 4 * dims[p + 1];
        f32.assign(tensors, tensors + tot);
    }
    size_t off = 0;
    for (int p = 0; p < N; ++p) {
        const int cl = dims[p], cr = dims[p + 1];
        const void* src = sites_f32(c) ? (const void*)(f32.data() + off) : (const void*)(tensors + off);
        CU(cudaMemcpy2DAsync(site_v(c, b, p), es * c->cap, src, es * cr, es * cr, (size_t)4 * cl,
                             cudaMemcpyHostToDevice, c->st));
        off += (size_t)cl * 4 * cr;
    }
    std::vector<double> ones((size_t)N * c->cap, 1.0);
    CU(cudaMemcpyAsync(c->d_lam + (size_t)b * N * c->cap, ones.data(), sizeof(double) * ones.size(),
                       cudaMemcpyHostToDevice, c->st));
    for (int p = 0; p <= N; ++p) c->h_dims[(size_t)b * (N + 1) + p] = dims[p];
    CU(cudaMemcpyAsync(c->d_dims, c->h_dims.data(), sizeof(int) * c->h_dims.size(), cudaMemcpyHostToDevice, c->st));
    CU(cudaStreamSynchronize(c->st));
    ++c->gen;
    return MPDO_OK;
}

int mpdo_get_state(mpdo_ctx* c, int b, int* dims, double* tensors, long long cap_elems) {
    if (!c || !dims) return fail(MPDO_EINVAL, "NULL argument");
    CU(cudaSetDevice(c->dev));
    if (b < 0 || b >= c->B) return fail(MPDO_EINVAL, "instance out of range");
    const int N = c->N;
    CU(cudaMemcpyAsync(c->h_dims.data(), c->d_dims, sizeof(int) * c->h_dims.size(), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    long long need = 0;
    for (int p = 0; p <= N; ++p) dims[p] = c->h_dims[(size_t)b * (N + 1) + p];
    for (int p = 0; p < N; ++p) need += (long long)dims[p] * 4 * dims[p + 1];
    if (!tensors) return MPDO_OK;
    if (need > cap_elems) return fail(MPDO_ECAPACITY, "tensor buffer too small");
    const size_t es = site_esize(c);
    std::vector<float> f32(sites_f32(c) ? (size_t)need : 0);
    size_t off = 0;
    for (int p = 0; p < N; ++p) {
        const int cl = dims[p], cr = dims[p + 1];
        void* dst = sites_f32(c) ? (void*)(f32.data() + off) : (void*)(tensors + off);
        CU(cudaMemcpy2DAsync(dst, es * cr, site_v(c, b, p), es * c->cap, es * cr, (size_t)4 * cl,
                             cudaMemcpyDeviceToHost, c->st));
        off += (size_t)cl * 4 * cr;
    }
    CU(cudaStreamSynchronize(c->st));
    if (sites_f32(c))
        for (size_t i = 0; i < f32.size(); ++i) tensors[i] = f32[i];
    return MPDO_OK;
}

int mpdo_op_counts(mpdo_ctx* c, int* n_ops, int* n_swaps, int* n_layers) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (n_ops) *n_ops = c->n_ops;
    if (n_swaps) *n_swaps = c->n_swaps;
    if (n_layers) *n_layers = (int)c->layers.size();
    return MPDO_OK;
}

int mpdo_rank_log(mpdo_ctx* c, int* k, long long cap) {
    if (!c || !k) return fail(MPDO_EINVAL, "NULL argument");
    if ((long long)c->rank_log.size() > cap) return fail(MPDO_ECAPACITY, "rank log buffer too small");
    std::copy(c->rank_log.begin(), c->rank_log.end(), k);
    return MPDO_OK;
}

int mpdo_force_ranks(mpdo_ctx* c, const int* k, int n_steps) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (!k || n_steps <= 0) {
        c->forced.clear();
        c->forced_steps = 0;
        return MPDO_OK;
    }
    const size_t per_b = (size_t)n_steps * c->n_ops;
    for (int b = 0; b < c->B; ++b)
        for (size_t i = 0; i < per_b; ++i) {
            const int v = k[(size_t)b * per_b + i];
            if (v < 1 || v > c->chi_max[b]) return fail(MPDO_EINVAL, "forced rank outside [1, chi_max]");
        }
    c->forced.assign(k, k + (size_t)c->B * per_b);
    c->forced_steps = n_steps;
    return MPDO_OK;
}

int mpdo_gates(mpdo_ctx* c, int b, double* out, long long cap) {
    if (!c || !out) return fail(MPDO_EINVAL, "NULL argument");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (b < 0 || b >= c->B) return fail(MPDO_EINVAL, "instance out of range");
    const long long need = (long long)c->n_ops * 256;
    if (need > cap) return fail(MPDO_ECAPACITY, "gate buffer too small");
    CU(cudaMemcpyAsync(out, c->d_gates + (size_t)b * c->n_ops * 256, sizeof(double) * need, cudaMemcpyDeviceToHost,
                       c->st));
    CU(cudaStreamSynchronize(c->st));
    return MPDO_OK;
}

int mpdo_schedule(int n, int n_bonds, const int* bond_i, const int* bond_j, int* ops, long long cap, int* n_ops) {
    if (!bond_i || !bond_j || !n_ops) return fail(MPDO_EINVAL, "NULL argument");
    if (n < 2 || n_bonds < 1) return fail(MPDO_EINVAL, "need n >= 2 and n_bonds >= 1");
    std::vector<int> bi(bond_i, bond_i + n_bonds), bj(bond_j, bond_j + n_bonds);
    std::vector<Layer> layers;
    std::vector<double> w;
    std::string err = build_schedule(n, bi, bj, layers, w);
    if (!err.empty()) return fail(MPDO_EINVAL, "bond graph: " + err);
    long long k = 0;
    for (size_t li = 0; li < layers.size(); ++li)
        for (const Op& o : layers[li]) {
            if (ops) {
                if ((k + 1) * 7 > cap) return fail(MPDO_ECAPACITY, "ops buffer too small");
                int* r = ops + k * 7;
                r[0] = (int)li;
                r[1] = o.kind;
                r[2] = o.p;
                r[3] = o.qa;
                r[4] = o.qb;
                r[5] = o.bond;
                r[6] = (int)std::lround(o.frac * 2.0);
            }
            ++k;
        }
    *n_ops = (int)k;
    return MPDO_OK;
}

int mpdo_inject_fault(mpdo_ctx* c, int kind) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    if (kind != 0 && kind != MPDO_FAULT_DROP_CTA) return fail(MPDO_EINVAL, "unknown fault kind");
    c->inject = kind;
    return MPDO_OK;
}

int mpdo_profile_enable(mpdo_ctx* c, int on) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    c->prof = on != 0;
    return MPDO_OK;
}

int mpdo_profile_read(mpdo_ctx* c, double* ms, long long* launches, double* flops, int kmax, int reset) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    for (int k = 0; k < std::min(kmax, kProfKinds); ++k) {
        if (ms) ms[k] = c->prof_ms[k];
        if (launches) launches[k] = c->prof_launch[k];
        if (flops) flops[k] = c->prof_flops[k];
    }
    if (reset) {
        for (int k = 0; k < kProfKinds; ++k) {
            c->prof_ms[k] = 0.0;
            c->prof_launch[k] = 0;
            c->prof_flops[k] = 0.0;
        }
        c->prof_sweeps = c->prof_svds = c->prof_sweeps32 = 0;
        c->prof_crit = c->prof_crit32 = c->prof_chunks = 0;
    }
    return MPDO_OK;
}

int mpdo_profile_sweeps(mpdo_ctx* c, long long* sweeps, long long* svds, long long* sweeps_fp32) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    if (sweeps) *sweeps = c->prof_sweeps;
    if (svds) *svds = c->prof_svds;
    if (sweeps_fp32) *sweeps_fp32 = c->prof_sweeps32;
    return MPDO_OK;
}

int mpdo_profile_sweeps_critical(mpdo_ctx* c, long long* crit, long long* crit_fp32, long long* chunks) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    if (crit) *crit = c->prof_crit;
    if (crit_fp32) *crit_fp32 = c->prof_crit32;
    if (chunks) *chunks = c->prof_chunks;
    return MPDO_OK;
}

void mpdo_destroy(mpdo_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

}  // extern "C"
