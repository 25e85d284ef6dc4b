// vor_noalloc.cu -- a build entry point that allocates no device memory.
//
// Some callers cannot allocate device memory when they need a diagram: a
// plug-in running inside a host application whose framework owns the whole
// device memory pool, or a real-time deployment that forbids device
// allocation after start-up (cudaMalloc can also synchronise the device,
// which such callers cannot afford).  vor_build_noalloc serves them: the
// caller still provides the sites and the output buffers, and the build's
// workspace is a fixed static array in device memory that every GPU loading
// this library keeps until the process exits.
//
// The array's name in host code is only a host-side stand-in for the device
// symbol, not a device address: a kernel handed it would fault or, where the
// GPU can reach host memory, silently use the wrong memory.  The device
// address is therefore looked up with cudaGetSymbolAddress on every call,
// with the caller's device current.  The address is not cached: it belongs
// to the context that is current at the call, and after cudaDeviceReset (or
// under another context on the same device) the module is loaded again at
// another address.  The lookup allocates nothing.
#include <cstring>

#include <cuda_runtime.h>

#include "vor.h"
#include "vor_internal.h"

namespace {

constexpr size_t kScratchBytes = VOR_NOALLOC_SCRATCH_BYTES;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch in the context current on the calling thread.
// Returns nullptr on failure.
void *scratch_address() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return nullptr;
    return p;
}

}  // namespace

extern "C" int vor_build_noalloc(const vor_site *d_sites, int64_t n, vor_box box,
                                 const vor_opts *opts, const vor_out *out, void *stream) {
    const int64_t need = vor_workspace_bytes(n, box, opts);
    if (need < 0) {
        if (box.w < 2 || box.h < 2 || box.w > (1 << 20) || box.h > (1 << 20))
            return VOR_E_BOX_TOO_LARGE;
        return VOR_E_INVALID_ARG;
    }
    if ((uint64_t)need > kScratchBytes) return VOR_E_SCRATCH_LIMIT;
    void *ws = scratch_address();
    if (!ws) return VOR_E_CUDA;
    // The build clears the parts of the workspace that must start at zero
    // (status header, bucket counts, probe histogram) on the stream itself.
    const int rc = vor_build_async(d_sites, n, box, opts, ws, (int64_t)kScratchBytes, out, stream);
    if (rc != VOR_OK) return rc;
    // waits for the stream and reads the build's status from the scratch
    return vor_status(ws, stream, nullptr);
}
