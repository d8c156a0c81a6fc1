// etics_noalloc.cu -- an SCF coefficient entry point that needs no workspace
// from the caller and allocates nothing.
//
// Some callers cannot hand the library a device buffer: a hard real-time
// loop where an allocation could block or fail at the wrong moment, or a host
// application that owns all device memory through its own budget and gives
// plug-in code no way to allocate.  For them etics_scf_coeffs_noalloc runs
// the ordinary coefficient pass with its scratch (the per-block FP64 partial
// sums) in a fixed array that is part of the library image itself.
#include <mutex>

#include "etics_internal.h"

namespace {

// File-scope scratch: every GPU that loads the library holds these bytes
// until the process exits.  Host code never uses the symbol directly (in
// host code it is only a stand-in); it asks the runtime for the device
// address once per device.
static __device__ __align__(256) unsigned char g_scf_scratch[ETICS_STATIC_SCRATCH_BYTES];

std::mutex g_scratch_mutex;
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scf_scratch on the current device (looked up on the
// first call for that device, with that device current).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ETICS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scf_scratch) != cudaSuccess || !p) return ETICS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return ETICS_OK;
}

}  // namespace

extern "C" int etics_scf_coeffs_noalloc(const void* posm, int64_t N, int n_max, int l_max,
                                        int precision, double* coeffs, void* stream) {
    if (N < 0 || (precision != ETICS_FP64 && precision != ETICS_MIXED) || !coeffs)
        return ETICS_ERR_ARG;
    if (n_max < 0 || l_max < 0) return ETICS_ERR_ARG;
    if (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    // the device lookups first, so that a failing CUDA call reads as
    // ETICS_ERR_CUDA and not as a bad argument
    void* scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc) return rc;
    const size_t need = etics_workspace_bytes(N, n_max, l_max, ETICS_SCF, precision);
    if (need == 0) return ETICS_ERR_CUDA;   // the arguments were checked above
    // the fixed array is too small for this expansion on this device
    if (need > (size_t)ETICS_STATIC_SCRATCH_BYTES) return ETICS_ERR_WORKSPACE;
    // The partial sums are written in full by every call before they are
    // read, so nothing in the array has to start at zero.
    return etics_scf_coeffs(posm, N, n_max, l_max, precision, coeffs, scratch,
                            (size_t)ETICS_STATIC_SCRATCH_BYTES, stream);
}
