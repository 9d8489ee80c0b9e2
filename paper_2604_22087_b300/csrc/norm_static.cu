// Allocation-free residual norm.
//
// jetsci_norm2 keeps its first-pass partial sums in scratch that jetsci_mesh_create
// allocated.  Some callers cannot allocate device memory at all when they need the norm:
// their device memory is reserved up front by another runtime's pool (a solver library or
// an array framework that owns the GPU's memory), or they cannot afford the implicit
// device synchronisation of cudaMalloc inside a time-critical loop, and they may hold no
// mesh.  jetsci_norm2_static serves them: its scratch is a fixed file-scope device array
// (kStaticPartials doubles, 32 KiB) that every GPU which loads this library holds until
// the process exits, so a call allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "jetsci_internal.h"

namespace {

constexpr int64_t kStaticPartials = 4096;  // first-pass partials; n <= 4096 * 8192
constexpr int kMaxDevices = 128;

static __device__ __align__(256) double g_norm_scratch[kStaticPartials];

double *g_scratch_addr[kMaxDevices] = {};  // device address of g_norm_scratch, per device
std::mutex g_scratch_mu;

}  // namespace

using namespace jetsci;

extern "C" jetsci_status jetsci_norm2_static(const double *x_dev, int64_t n, double *out_dev, void *stream) {
    if (n < 0 || !out_dev || (n > 0 && !x_dev)) return fail(JETSCI_ERR_ARG, "invalid norm arguments");
    const int64_t max_n = kStaticPartials * (int64_t)kNormChunk;
    if (n > max_n)
        return fail(JETSCI_ERR_ARG, "jetsci_norm2_static: n = " + std::to_string(n) +
                                        " exceeds the static scratch limit of " + std::to_string(max_n) +
                                        " entries; use jetsci_norm2");
    int dev = -1;
    JETSCI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(JETSCI_ERR_ARG, "device ordinal out of range");
    double *scratch = nullptr;
    {
        // Set-up, once per device with that device current: in host code the symbol's name
        // is only a host-side stand-in, so the kernels get its device address.
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_norm_scratch)");
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    return launch_norm2(x_dev, n, scratch, kStaticPartials, out_dev, (cudaStream_t)stream);
}
