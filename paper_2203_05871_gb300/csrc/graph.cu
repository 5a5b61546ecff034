// One Trotter step as a CUDA graph (mpdo_trotter_step_graph).
//
// mpdo_trotter_step reads the new bond dimensions back to the host after every
// chunk of ops, to size the next chunk's launches exactly.  Here nothing goes
// back to the host inside a step: every chunk starts with a planner kernel that
// reads the bond dimensions on the device and writes the dimension fields of
// the chunk's op descriptors, the co-resident CTA plans of the cooperative QR
// and Jacobi launches (the host plan's proportional-to-work rule; the launch
// has every resident CTA and the unassigned ones return at once); the
// tensor-core products build their problem shapes from the descriptors on the
// device as well, and every other launch has a capacity-sized grid
// whose CTAs outside an op's shape return at once.  The step is captured once
// per layout (op list and workspaces) and replayed; ranks are collected on the
// device.
#include <mpdo.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ctx.h"
#include "internal.h"

using namespace mpdo;

namespace mpdo {

namespace {

// Shares R co-resident CTAs among the ops of a chunk in proportion to their
// work, each op between 1 and cap_s CTAs (the host plan's rule).  out: [R] op
// of each CTA (-1: unused, the CTA returns at once), [R] rank within the op,
// [nops] CTAs per op.  Returns 0, or 1 if R < nops.
__device__ int plan_ctas(const double* work, const int* cap, int nops, int R, int* out) {
    int* G = out + 2 * R;
    double wsum = 0.0;
    for (int s = 0; s < nops; ++s) wsum += work[s];
    int total = 0;
    for (int s = 0; s < nops; ++s) {
        int g = (int)floor((double)R * work[s] / fmax(wsum, 1.0));
        g = max(1, min(cap[s], g));
        const int passes = (cap[s] + g - 1) / g;
        g = (cap[s] + passes - 1) / passes;
        G[s] = g;
        total += g;
    }
    while (total > R) {
        int arg = 0;
        for (int s = 1; s < nops; ++s)
            if (G[s] > G[arg]) arg = s;
        if (G[arg] <= 1) return 1;
        G[arg]--;
        total--;
    }
    int t = 0;
    for (int s = 0; s < nops; ++s)
        for (int g = 0; g < G[s]; ++g, ++t) {
            out[t] = s;
            out[R + t] = g;
        }
    for (; t < R; ++t) {
        out[t] = -1;
        out[R + t] = 0;
    }
    return 0;
}

constexpr int kMaxChunk = 1024;

__global__ void __launch_bounds__(256) plan_chunk_kernel(OpDesc* descs, int nops, const int* dims, int N, int Rj,
                                                         int Rq, int* cta64, int* cta32, int* ctaqr, int mixed,
                                                         const int* jb_table, int chi_cap, int* error) {
    __shared__ double work[kMaxChunk];
    __shared__ int cap[kMaxChunk];
    for (int s = threadIdx.x; s < nops; s += blockDim.x) {
        OpDesc& d = descs[s];
        const int* dm = dims + (size_t)d.b * (N + 1);
        d.cl = dm[d.p];
        d.cm = dm[d.p + 1];
        d.cr = dm[d.p + 2];
        d.m = 4 * d.cl;
        d.n = 4 * d.cr;
        d.c = min(d.m, d.n);
        d.L = d.n;
        d.jb = jacobi_block_rows(d.L, d.c, 8);
        d.jb32 = jacobi_block_rows_f32(d.L, d.c);
        if (jb_table) {   // autotuned rows per block of this (chi_l, chi_r) class
            const int* t = jb_table + ((size_t)d.cl * (chi_cap + 1) + d.cr) * 2;
            if (t[0] > 0) d.jb = t[0];
            if (t[1] > 0) d.jb32 = t[1];
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int bad = 0;
    for (int s = 0; s < nops; ++s) {
        const OpDesc& d = descs[s];
        work[s] = (double)d.c * d.c * (double)d.L;
        cap[s] = jacobi_pairs_per_round(d.c, d.jb);
    }
    bad |= plan_ctas(work, cap, nops, Rj, cta64);
    if (mixed) {
        for (int s = 0; s < nops; ++s) cap[s] = jacobi_pairs_per_round(descs[s].c, descs[s].jb32);
        bad |= plan_ctas(work, cap, nops, Rj, cta32);
    }
    for (int s = 0; s < nops; ++s) {
        const OpDesc& d = descs[s];
        work[s] = (double)d.m * d.n * d.c;
        cap[s] = max(1, (d.n + kQrWarps - 1) / kQrWarps);
    }
    bad |= plan_ctas(work, cap, nops, Rq, ctaqr);
    if (bad) *error = 1;
}

// klog[b * n_ops + op] = the rank the op chose
__global__ void klog_kernel(const OpDesc* descs, int nops, int n_ops, int* klog) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nops; s += gridDim.x * blockDim.x) {
        const OpDesc& d = descs[s];
        klog[(size_t)d.b * n_ops + d.op] = *d.k_out;
    }
}

struct Chunk {
    int nops = 0;
    OpDesc* d_desc = nullptr;
    int *d_cta64 = nullptr, *d_cta32 = nullptr, *d_ctaqr = nullptr;
};

}  // namespace

struct GraphState {
    long long layout = -1;
    cudaStream_t cap_st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<std::vector<Chunk>> chunks;   // per layer
    int* d_klog = nullptr;                    // [B][n_ops] ranks of the last replayed step
    int* d_error = nullptr;
    int Rj = 0, Rq = 0;
};

namespace {

void release(GraphState* g) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->exec = nullptr;
    g->graph = nullptr;
    for (auto& L : g->chunks)
        for (auto& ch : L) {
            void* ptrs[] = {ch.d_desc, ch.d_cta64, ch.d_cta32, ch.d_ctaqr};
            for (void* p : ptrs)
                if (p) cudaFree(p);
        }
    g->chunks.clear();
    if (g->d_klog) cudaFree(g->d_klog);
    if (g->d_error) cudaFree(g->d_error);
    g->d_klog = nullptr;
    g->d_error = nullptr;
    g->layout = -1;
}

// queue one step on stream st (captured)
int enqueue_step(mpdo_ctx* c, GraphState* g, cudaStream_t st) {
    const int cap = c->cap, ld = c->ld;
    const unsigned long long timeout_ns = (unsigned long long)c->cfg.barrier_timeout_ms * 1000000ull;
    for (auto& L : g->chunks)
        for (auto& ch : L) {
            const int nops = ch.nops;
            plan_chunk_kernel<<<1, 256, 0, st>>>(ch.d_desc, nops, c->d_dims, c->N, g->Rj, g->Rq, ch.d_cta64,
                                                 ch.d_cta32, ch.d_ctaqr, c->mixed ? 1 : 0, c->d_jb_table, cap,
                                                 g->d_error);
            CU(cudaGetLastError());
            CU(cudaMemsetAsync(c->d_sweeps, 0, sizeof(int) * nops, st));
            if (c->mixed) {
                CU(launch_oz_ops(ch.d_desc, nops, OZ_MERGE, c->d_oz, cap, c->oz_bf16, timeout_ns, st));
                CU(launch_gate_weight(ch.d_desc, nops, cap, st));
            } else {
                CU(launch_merge_gate(ch.d_desc, nops, cap, st));
            }
            const size_t sync_bytes = sizeof(unsigned) * jacobi_sync_words(nops);
            CU(cudaMemsetAsync(c->d_sync, 0, sync_bytes, st));
            if (c->mixed && c->cfg.qr_blocked && qrb_fits(cap))
                CU(launch_qr_blocked(ch.d_desc, nops, cap, c->d_oz, c->oz_bf16, timeout_ns, st, 0));
            else
                CU(launch_qr(ch.d_desc, ch.d_ctaqr, ch.d_ctaqr + g->Rq, ch.d_ctaqr + 2 * g->Rq, c->d_sync, g->Rq,
                             timeout_ns, ld, st));
            if (c->mixed) {
                CU(cudaMemsetAsync(c->d_sync, 0, sync_bytes, st));
                CU(launch_jacobi(ch.d_desc, nops, ch.d_cta32, ch.d_cta32 + g->Rj, ch.d_cta32 + 2 * g->Rj, c->d_sync,
                                 g->Rj, kMaxSweepsCap / 2, 0.0, timeout_ns, ld, true, st, precond_rho(c)));
                CU(launch_oz_ops(ch.d_desc, nops, OZ_E, c->d_oz, cap, c->oz_bf16, timeout_ns, st));
                CU(launch_oz_ops(ch.d_desc, nops, OZ_Q, c->d_oz, cap, c->oz_bf16, timeout_ns, st));
                CU(launch_oz_ops(ch.d_desc, nops, OZ_W, c->d_oz, cap, c->oz_bf16, timeout_ns, st));
            }
            CU(cudaMemsetAsync(c->d_sync, 0, sync_bytes, st));
            CU(launch_jacobi(ch.d_desc, nops, ch.d_cta64, ch.d_cta64 + g->Rj, ch.d_cta64 + 2 * g->Rj, c->d_sync, g->Rj,
                             c->cfg.jacobi_max_sweeps, fp64_jacobi_tol(c), timeout_ns, ld, false, st, precond_rho(c)));
            CU(launch_truncate(ch.d_desc, nops, cap, st));
            if (c->mixed)
                CU(launch_oz_ops(ch.d_desc, nops, OZ_RECON, c->d_oz, cap, c->oz_bf16, timeout_ns, st));
            else
                CU(launch_reconstruct(ch.d_desc, nops, cap, st));
            klog_kernel<<<(nops + 127) / 128, 128, 0, st>>>(ch.d_desc, nops, c->n_ops, g->d_klog);
            CU(cudaGetLastError());
        }
    CU(launch_trace_normalize(c->d_sites, sites_f32(c), c->d_dims, c->N, c->B, cap, c->cfg.force_trace, c->d_trace,
                              c->d_status, st));
    return MPDO_OK;
}

int build_graph(mpdo_ctx* c, GraphState* g) {
    release(g);
    if (!g->cap_st) CU(cudaStreamCreateWithFlags(&g->cap_st, cudaStreamNonBlocking));
    g->Rj = c->jacobi_resident;
    g->Rq = c->qr_resident;
    CU(dalloc(&g->d_klog, (size_t)c->B * c->n_ops));
    CU(dalloc(&g->d_error, 1));
    CU(cudaMemsetAsync(g->d_error, 0, sizeof(int), c->st));
    g->chunks.assign(c->layers.size(), {});
    for (int li = 0; li < (int)c->layers.size(); ++li) {
        const std::vector<Item> items = layer_items(c, li);
        const size_t cs = (size_t)chunk_ops(c);
        for (size_t s0 = 0; s0 < items.size(); s0 += cs) {
            const int nops = (int)std::min(cs, items.size() - s0);
            if (nops > kMaxChunk || nops > std::min(g->Rj, g->Rq))
                return fail(MPDO_ECAPACITY, "graph step: more ops in one chunk than co-resident CTAs");
            Chunk ch;
            ch.nops = nops;
            std::vector<OpDesc> h(nops);
            for (int s = 0; s < nops; ++s) fill_desc(c, items[s0 + s], s, h[s]);
            CU(dalloc(&ch.d_desc, (size_t)nops));
            CU(dalloc(&ch.d_cta64, (size_t)2 * g->Rj + nops));
            CU(dalloc(&ch.d_ctaqr, (size_t)2 * g->Rq + nops));
            if (c->mixed) CU(dalloc(&ch.d_cta32, (size_t)2 * g->Rj + nops));
            CU(cudaMemcpyAsync(ch.d_desc, h.data(), sizeof(OpDesc) * nops, cudaMemcpyHostToDevice, c->st));
            CU(cudaStreamSynchronize(c->st));
            g->chunks[li].push_back(ch);
        }
    }
    CU(cudaStreamSynchronize(c->st));
    CU(cudaStreamBeginCapture(g->cap_st, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(c, g, g->cap_st);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->cap_st, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(MPDO_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    g->graph = graph;
    CU(cudaGraphInstantiate(&g->exec, g->graph, 0));
    g->layout = c->layout;
    return MPDO_OK;
}

}  // namespace

void graph_free(GraphState* g) {
    if (!g) return;
    release(g);
    if (g->cap_st) cudaStreamDestroy(g->cap_st);
    delete g;
}

}  // namespace mpdo

extern "C" int mpdo_trotter_step_graph(mpdo_ctx* c, int n_steps) {
    if (!c) return fail(MPDO_EINVAL, "ctx is NULL");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (n_steps < 0) return fail(MPDO_EINVAL, "n_steps must be >= 0");
    if (c->forced_steps > 0) return fail(MPDO_EINVAL, "forced ranks are not supported by the graph step");
    if (!c->graph) {
        c->graph = new (std::nothrow) GraphState();
        if (!c->graph) return fail(MPDO_ENOMEM, "host allocation failed");
    }
    GraphState* g = c->graph;
    if (g->layout != c->layout || !g->exec) {
        int rc = build_graph(c, g);
        if (rc) return rc;
    }
    const size_t per = (size_t)c->B * c->n_ops;
    int* d_all = nullptr;
    CU(dalloc(&d_all, std::max<size_t>(1, per * n_steps)));
    for (int step = 0; step < n_steps; ++step) {
        cudaError_t e = cudaGraphLaunch(g->exec, c->st);
        if (e != cudaSuccess) {
            cudaFree(d_all);
            return fail(MPDO_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
        }
        e = cudaMemcpyAsync(d_all + per * step, g->d_klog, sizeof(int) * per, cudaMemcpyDeviceToDevice, c->st);
        if (e != cudaSuccess) {
            cudaFree(d_all);
            return fail(MPDO_ECUDA, std::string("rank copy: ") + cudaGetErrorString(e));
        }
    }
    std::vector<int> all(per * n_steps), err(1);
    cudaError_t e1 = cudaMemcpyAsync(all.data(), d_all, sizeof(int) * all.size(), cudaMemcpyDeviceToHost, c->st);
    cudaError_t e2 = cudaMemcpyAsync(err.data(), g->d_error, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    cudaError_t e3 = cudaMemcpyAsync(c->h_dims.data(), c->d_dims, sizeof(int) * c->h_dims.size(),
                                     cudaMemcpyDeviceToHost, c->st);
    cudaError_t e4 = cudaStreamSynchronize(c->st);
    cudaFree(d_all);
    for (cudaError_t e : {e1, e2, e3, e4})
        if (e != cudaSuccess) return fail(MPDO_ECUDA, std::string("graph step: ") + cudaGetErrorString(e));
    if (err[0]) return fail(MPDO_ECAPACITY, "graph step: more ops in flight than co-resident CTAs");
    c->rank_steps = n_steps;
    c->rank_log.assign(per * n_steps, 0);
    for (int step = 0; step < n_steps; ++step)
        for (int b = 0; b < c->B; ++b)
            for (int op = 0; op < c->n_ops; ++op)
                c->rank_log[((size_t)b * n_steps + step) * c->n_ops + op] = all[per * step + (size_t)b * c->n_ops + op];
    ++c->gen;
    return check_status_code(c);
}
