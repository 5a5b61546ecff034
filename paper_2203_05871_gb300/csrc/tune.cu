// Autotuner of the Jacobi SVD's rows per block, per (chi_l, chi_r) class
// (mpdo_autotune).
//
// The one-sided Jacobi stages two blocks of b rows per block pair (jacobi.cu:
// both in shared memory, or for the FP32 pass on rows of at most 1024
// elements one in shared memory and one in registers).  Larger blocks mean fewer rounds and barriers per sweep and
// more work per shared-memory load; smaller ones more block pairs per round,
// i.e. more CTAs per op.  The best b depends on the row length, the number of
// rows and how many ops share the GPU, so it is measured: for every class the
// tuner fills as many workspace slots as a layer has ops in flight with a
// seeded graded matrix of the class's shape (rows scaled like the rows of a
// pivoted R; at most 16 slots), and times the Jacobi launch for every b that fits (FP64 pass,
// and the FP32 pass of the mixed path), keeping the fastest.  The winners go
// to a (chi_l, chi_r) table that both the host-planned and the graph step
// read.  Different b change the order of the rotations, so results change at
// rounding level only.
#include <mpdo.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "ctx.h"
#include "internal.h"

using namespace mpdo;

namespace mpdo {

namespace {

int time_jacobi(mpdo_ctx* c, std::vector<OpDesc>& h, bool fp32, int b, double* ms_out) {
    const int nops = (int)h.size();
    const int ld = c->ld;
    for (auto& d : h) (fp32 ? d.jb32 : d.jb) = b;
    // pristine rows back into W0 (and W) from Theta' (holding the synthetic input)
    for (const auto& d : h) {
        CU(cudaMemcpy2DAsync(d.W0, sizeof(double) * ld, d.thetap, sizeof(double) * ld, sizeof(double) * d.L, d.c,
                             cudaMemcpyDeviceToDevice, c->st));
        if (d.W != d.W0)
            CU(cudaMemcpy2DAsync(d.W, sizeof(double) * ld, d.thetap, sizeof(double) * ld, sizeof(double) * d.L, d.c,
                                 cudaMemcpyDeviceToDevice, c->st));
    }
    CU(cudaMemcpyAsync(c->d_desc, h.data(), sizeof(OpDesc) * nops, cudaMemcpyHostToDevice, c->st));
    int total = 0;
    const int gcap = std::max(std::max(c->jacobi_resident, c->qr_resident), c->slots);
    int rc = plan_jacobi(c, h.data(), nops, fp32, c->h_cta, total);
    if (rc) return rc;
    CU(cudaMemcpyAsync(c->d_cta, c->h_cta, sizeof(int) * (2 * total + nops), cudaMemcpyHostToDevice, c->st));
    (void)gcap;
    const unsigned long long timeout_ns = (unsigned long long)c->cfg.barrier_timeout_ms * 1000000ull;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    CU(cudaMemsetAsync(c->d_sync, 0, sizeof(unsigned) * jacobi_sync_words(nops), c->st));
    CU(cudaEventRecord(e0, c->st));
    CU(launch_jacobi(c->d_desc, nops, c->d_cta, c->d_cta + total, c->d_cta + 2 * total, c->d_sync, total,
                     fp32 ? kMaxSweepsCap / 2 : c->cfg.jacobi_max_sweeps, fp32 ? 0.0 : fp64_jacobi_tol(c), timeout_ns, ld,
                     fp32, c->st, precond_rho(c)));
    CU(cudaEventRecord(e1, c->st));
    CU(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms;
    return MPDO_OK;
}

}  // namespace

}  // namespace mpdo

extern "C" int mpdo_autotune(mpdo_ctx* c, const int* classes, int n_classes, int* chosen) {
    if (!c || (!classes && n_classes > 0)) return fail(MPDO_EINVAL, "NULL argument");
    CU(cudaSetDevice(c->dev));
    if (!c->built) return fail(MPDO_ESTATE, "mpdo_build_gates must come first");
    if (n_classes < 0) return fail(MPDO_EINVAL, "n_classes must be >= 0");
    const int cap = c->cap, ld = c->ld;
    for (int i = 0; i < n_classes; ++i)
        if (classes[2 * i] < 1 || classes[2 * i] > cap || classes[2 * i + 1] < 1 || classes[2 * i + 1] > cap)
            return fail(MPDO_EINVAL, "class chi values must be in [1, chi_cap]");
    if (c->jb_table.empty()) c->jb_table.assign((size_t)(cap + 1) * (cap + 1) * 2, 0);
    // ops in flight while timing: a layer's worth, at most 16 (enough to share
    // the GPU the way a layer does, and keeps tuning to seconds)
    const int nops = std::max(1, std::min(std::min(c->slots, c->B * c->max_layer), 16));
    std::mt19937_64 rng(2203058712ull);
    std::normal_distribution<double> nd(0.0, 1.0);
    int* d_status = nullptr;
    CU(dalloc(&d_status, 1));
    for (int i = 0; i < n_classes; ++i) {
        const int cl = classes[2 * i], cr = classes[2 * i + 1];
        const int m = 4 * cl, n = 4 * cr, cc = std::min(m, n);
        // seeded graded rows (row j scaled by 10^(-10 j / cc)), one copy per slot in Theta'
        std::vector<double> rows((size_t)cc * ld, 0.0);
        for (int j = 0; j < cc; ++j) {
            const double sc = std::pow(10.0, -10.0 * j / std::max(cc, 1));
            for (int k = 0; k < n; ++k) rows[(size_t)j * ld + k] = sc * nd(rng);
        }
        std::vector<OpDesc> h(nops);
        for (int s = 0; s < nops; ++s) {
            OpDesc d{};
            d.b = 0;
            d.cl = cl;
            d.cr = cr;
            d.m = m;
            d.n = n;
            d.c = cc;
            d.L = n;
            d.chi_max = c->chi_max[0];
            d.cutoff = c->cutoff[0];
            const size_t mat = (size_t)ld * ld;
            d.thetap = c->d_thetap + (size_t)s * mat;
            d.W = c->d_W + (size_t)s * mat;
            d.W0 = c->mixed ? c->d_W0 + (size_t)s * mat : d.W;
            d.W32 = c->mixed ? c->d_W32 + (size_t)s * mat : nullptr;
            d.U32 = c->mixed ? c->d_U32 + (size_t)s * mat : nullptr;
            d.snorm = c->d_snorm + (size_t)s * 2 * ld;
            d.status = d_status;
            d.sweeps_out = c->d_sweeps + s;
            h[s] = d;
            CU(cudaMemcpyAsync(d.thetap, rows.data(), sizeof(double) * rows.size(), cudaMemcpyHostToDevice, c->st));
        }
        for (int pass = 0; pass < (c->mixed ? 2 : 1); ++pass) {
            const bool fp32 = pass == 1;
            const int rowlen = n;
            const int eb = 8;
            double best = 1e300;
            int best_b = fp32 ? jacobi_block_rows_f32(n, cc) : jacobi_block_rows(rowlen, cc, eb);
            for (int b = 1; b <= kJacobiMaxB; b *= 2) {
                if (fp32 ? !jacobi_f32_fits(b, n, cc) : (size_t)2 * b * rowlen * eb > (size_t)kJacobiRowBytes) break;
                if (b > 1 && b >= cc) break;
                if (fp32) {   // the FP32 pass starts from the FP64 rows of W0
                    for (auto& d : h) d.jb = jacobi_block_rows(n, cc, 8);
                }
                double t = 1e300;
                for (int rep = 0; rep < 2; ++rep) {
                    double ms = 0.0;
                    int rc = time_jacobi(c, h, fp32, b, &ms);
                    if (rc) {
                        cudaFree(d_status);
                        return rc;
                    }
                    t = std::min(t, ms);
                }
                if (t < best) {
                    best = t;
                    best_b = b;
                }
            }
            c->jb_table[((size_t)cl * (cap + 1) + cr) * 2 + pass] = best_b;
            if (chosen) chosen[2 * i + pass] = best_b;
        }
        if (!c->mixed && chosen) chosen[2 * i + 1] = 0;
    }
    cudaFree(d_status);
    if (!c->d_jb_table) CU(dalloc(&c->d_jb_table, c->jb_table.size()));
    CU(cudaMemcpyAsync(c->d_jb_table, c->jb_table.data(), sizeof(int) * c->jb_table.size(), cudaMemcpyHostToDevice,
                       c->st));
    CU(cudaStreamSynchronize(c->st));
    ++c->layout;   // a captured graph step is rebuilt with the table
    return MPDO_OK;
}
