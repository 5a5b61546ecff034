// mpdo_measure_1q_noalloc: single-qubit Pauli expectation values of MPO states
// that the caller keeps in its own device memory, for callers that must not
// allocate device memory: frameworks that hand all device memory to their own
// pool up front (a hidden cudaMalloc would fail or break their accounting),
// and code whose allocation rules forbid the runtime's allocator altogether.
//
// Same computation as mpdo_measure_1q (left/right identity environments,
// then E(comp at q) / E(I...I)), but the environment scratch lives in the
// file-scope device array below instead of a context allocation.  The array
// is created when the library is loaded on a device and is kept until the
// process exits.  Every call shares it: calls that overlap on the GPU (for
// example on two streams) race on it and must be serialised by the caller.
//
// The bond dimensions and qubit indices sit in the caller's device memory, so
// the host cannot check them.  A first kernel copies them into the scratch,
// clamped to valid ranges (dims to [1, chi_cap], dims[0] = dims[n] = 1, qubits
// to [0, n)), and records which instances and qubits were out of range; the
// environment and measurement kernels then only ever see the clamped copies,
// so every access stays inside the caller's arrays and the scratch.  A last
// kernel writes NaN to out[b][k] for every flagged instance b or qubit k.
#include <mpdo.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace mpdo {

// Capacity of the static scratch, in doubles (2 MiB).  A call needs both
// environment arrays, 2 * batch * (n_qubits + 1) * chi_cap doubles, followed by
// the clamped bond dimensions and qubits and their flags, batch * (n_qubits + 2)
// + 2 * nq ints (two per double, rounded up).
constexpr long long kNoallocScratchDoubles = 1ll << 18;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

namespace {

// Clamped copies of the caller's dims [B][n+1] and qubits [nq] (dims_s, q_s)
// and the out-of-range flags bad_b [B], bad_q [nq].  One CTA: the flags are
// cleared before any thread sets one.
__global__ void noalloc_sanitize_kernel(const int* dims, const int* qubits, int n, int B, int nq, int cap,
                                        int* dims_s, int* q_s, int* bad_b, int* bad_q) {
    for (int i = threadIdx.x; i < B; i += blockDim.x) bad_b[i] = 0;
    for (int i = threadIdx.x; i < nq; i += blockDim.x) bad_q[i] = 0;
    __syncthreads();
    const int total = B * (n + 1);
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int b = i / (n + 1), p = i % (n + 1);
        const int v = dims[i];
        const bool edge = p == 0 || p == n;
        const bool ok = edge ? v == 1 : (v >= 1 && v <= cap);
        dims_s[i] = edge ? 1 : min(max(v, 1), cap);
        if (!ok) atomicOr(bad_b + b, 1);
    }
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
        const int q = qubits[k];
        const bool ok = q >= 0 && q < n;
        q_s[k] = ok ? q : 0;
        if (!ok) bad_q[k] = 1;
    }
}

// out[b][k] = NaN where instance b or qubit k was out of range
__global__ void noalloc_flag_kernel(const int* bad_b, const int* bad_q, int B, int nq, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * nq) return;
    const int b = t / nq, k = t % nq;
    if (bad_b[b] || bad_q[k]) out[t] = __longlong_as_double(0x7ff8000000000000ll);
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

int fail(int code, const std::string& msg) {
    set_last_error("mpdo_measure_1q_noalloc: " + msg);
    return code;
}

}  // namespace

}  // namespace mpdo

using namespace mpdo;

extern "C" int mpdo_measure_1q_noalloc(const double* sites, const int* dims, int n_qubits, int batch, int chi_cap,
                                       const int* qubits, int nq, char comp, double* out, void* cuda_stream) {
    int a = -1;
    switch (comp) {
        case 'I': case 'i': a = 0; break;
        case 'X': case 'x': a = 1; break;
        case 'Y': case 'y': a = 2; break;
        case 'Z': case 'z': a = 3; break;
        default: break;
    }
    if (!sites || !dims || !qubits || !out) return fail(MPDO_EINVAL, "NULL pointer argument");
    if (a < 0) return fail(MPDO_EINVAL, "comp must be one of I, X, Y, Z");
    if (n_qubits < 1 || batch < 1 || nq < 0) return fail(MPDO_EINVAL, "need n_qubits >= 1, batch >= 1, nq >= 0");
    if (chi_cap < 1 || chi_cap > kMaxChi) return fail(MPDO_EINVAL, "chi_cap must be in [1, 512]");
    const long long env = 2ll * batch * (n_qubits + 1) * chi_cap;
    const long long ints = (long long)batch * (n_qubits + 2) + 2ll * nq;
    const long long need = env + (ints + 1) / 2;
    if (need > kNoallocScratchDoubles)
        return fail(MPDO_ECAPACITY, "2 * batch * (n_qubits + 1) * chi_cap doubles plus (batch * (n_qubits + 2) + 2 * nq) "
                                    "ints = " + std::to_string(need) + " doubles exceed the static scratch of " +
                                        std::to_string(kNoallocScratchDoubles) + " doubles");
    if (nq == 0) return MPDO_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(MPDO_ECUDA, "no usable current device");
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            // One-time set-up on this device (the device is current): the host-side
            // symbol is only a stand-in, the kernels need the device address.
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return fail(MPDO_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double* envL = scratch;
    double* envR = scratch + (size_t)batch * (n_qubits + 1) * chi_cap;
    int* dims_s = reinterpret_cast<int*>(scratch + env);
    int* q_s = dims_s + (size_t)batch * (n_qubits + 1);
    int* bad_b = q_s + nq;
    int* bad_q = bad_b + batch;
    noalloc_sanitize_kernel<<<1, 256, 0, st>>>(dims, qubits, n_qubits, batch, nq, chi_cap, dims_s, q_s, bad_b, bad_q);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_environments(sites, 0, dims_s, n_qubits, batch, chi_cap, envL, envR, st);
    if (e == cudaSuccess)
        e = launch_measure_1q(sites, 0, dims_s, n_qubits, batch, chi_cap, envL, envR, q_s, nq, a, out, st);
    if (e == cudaSuccess) {
        const int tot = batch * nq;
        noalloc_flag_kernel<<<(tot + 255) / 256, 256, 0, st>>>(bad_b, bad_q, batch, nq, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(MPDO_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return MPDO_OK;
}
