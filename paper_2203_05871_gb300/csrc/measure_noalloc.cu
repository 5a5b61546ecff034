// mpdo_measure_1q_noalloc: single-qubit Pauli expectation values of MPO states
// that the caller keeps in its own device memory, for callers that must not
// allocate device memory.  Such callers include code that runs while a
// stream is being captured into a CUDA graph, and frameworks that hand all
// device memory to their own pool up front, so a hidden cudaMalloc would fail
// or break their accounting.
//
// Same computation as mpdo_measure_1q (left/right identity environments,
// then E(comp at q) / E(I...I)), but the environment scratch lives in the
// file-scope device array below instead of a context allocation.  The array
// is created when the library is loaded on a device and is kept until the
// process exits.  Every call shares it: calls that overlap on the GPU (for
// example on two streams) race on it and must be serialised by the caller.
#include <mpdo.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace mpdo {

// Capacity of the static scratch, in doubles: both environment arrays,
// 2 * batch * (n_qubits + 1) * chi_cap <= kNoallocScratchDoubles (2 MiB).
constexpr long long kNoallocScratchDoubles = 1ll << 18;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

namespace {

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
    const long long need = 2ll * batch * (n_qubits + 1) * chi_cap;
    if (need > kNoallocScratchDoubles)
        return fail(MPDO_ECAPACITY, "2 * batch * (n_qubits + 1) * chi_cap = " + std::to_string(need) +
                                        " exceeds the static scratch of " + std::to_string(kNoallocScratchDoubles) +
                                        " doubles");
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
    cudaError_t e = launch_environments(sites, 0, dims, n_qubits, batch, chi_cap, envL, envR, st);
    if (e == cudaSuccess)
        e = launch_measure_1q(sites, 0, dims, n_qubits, batch, chi_cap, envL, envR, qubits, nq, a, out, st);
    if (e != cudaSuccess) return fail(MPDO_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return MPDO_OK;
}
