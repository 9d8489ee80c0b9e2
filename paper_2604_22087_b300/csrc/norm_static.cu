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

#include <string>

#include "jetsci_internal.h"

namespace {

constexpr int64_t kStaticPartials = 4096;  // first-pass partials; n <= 4096 * 8192

static __device__ __align__(256) double g_norm_scratch[kStaticPartials];

}  // namespace

using namespace jetsci;

extern "C" jetsci_status jetsci_norm2_static(const double *x_dev, int64_t n, double *out_dev, void *stream) {
    if (n < 0 || !out_dev || (n > 0 && !x_dev)) return fail(JETSCI_ERR_ARG, "invalid norm arguments");
    const int64_t max_n = kStaticPartials * (int64_t)kNormChunk;
    if (n > max_n)
        return fail(JETSCI_ERR_ARG, "jetsci_norm2_static: n = " + std::to_string(n) +
                                        " exceeds the static scratch limit of " + std::to_string(max_n) +
                                        " entries; use jetsci_norm2");
    // In host code the symbol's name is only a host-side stand-in: the kernels get its device
    // address in the current device's context.  It is looked up on every call (after the first
    // call on a device, which may load this library's device code, the lookup is a table
    // search), not cached, so that a cudaDeviceReset, which reloads the module possibly at
    // another address, leaves no stale pointer behind.
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_norm_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_norm_scratch)");
    return launch_norm2(x_dev, n, static_cast<double *>(p), kStaticPartials, out_dev, (cudaStream_t)stream);
}
