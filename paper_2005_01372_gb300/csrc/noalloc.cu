// lsw_apply_operator_noalloc: the FFT operator with its scratch in a fixed
// device array instead of stream-ordered allocations.
//
// Some callers must not have the library allocate device memory while they
// run: applications that reserve all device memory up front for their own
// allocator, embedders whose memory budget is audited per call, and
// latency-critical loops that cannot absorb an allocation's cost or its
// possible failure mid-run.  For them this entry point computes exactly what
// lsw_apply_operator computes, with the scratch taken from a file-scope
// __device__ array of fixed size.
#include <cuda_runtime.h>

#include <mutex>

#include "lsw_internal.cuh"

namespace lsw {
namespace {

// 32 MiB of scratch.  Every GPU that loads the library holds this array until
// the process exits.  The operator needs 2 * nbatch * nz * nx complex values
// of its precision (e.g. 32 fields of 256 x 256 in FP32).
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// The array's device address on the current device.  In host code the
// symbol's name is only a host-side stand-in: handing it to a kernel would
// fault, or silently use the wrong memory where the GPU can reach host
// memory, so the address is looked up with the device current.
lsw_status lookup_scratch(int dev, void** out) {
    void* p = nullptr;
    LSW_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_ptr[dev] = p;
    *out = p;
    return LSW_OK;
}

lsw_status scratch_on_current_device(void** out) {
    int dev = 0;
    LSW_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LSW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_ptr[dev]) {
        *out = g_scratch_ptr[dev];
        return LSW_OK;
    }
    return lookup_scratch(dev, out);
}

}  // namespace

// Set-up, once per lsw_build_green on the current device: (re)load the
// array's address.  Looking it up also loads the library's device code on
// that device if it was not loaded yet, which is when the array is
// committed, so no later call of the entry point does either.  A device
// reset invalidates every handle built before it; the next lsw_build_green
// refreshes the address, so a cached address is never stale for a valid
// handle.
lsw_status noalloc_setup() {
    int dev = 0;
    LSW_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LSW_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    void* p = nullptr;
    return lookup_scratch(dev, &p);
}

}  // namespace lsw

using namespace lsw;

extern "C" lsw_status lsw_apply_operator_noalloc(const lsw_green* g, int prec, const double* chi, const void* u,
                                                 const void* u0, void* y, int nbatch, int mode, void* stream) {
    if (!g || !chi || nbatch < 0) return LSW_ERR_INVALID_ARG;
    if (mode < LSW_OP_FORWARD || mode > LSW_OP_ADJOINT) return LSW_ERR_INVALID_ARG;
    if (prec != LSW_C128 && prec != LSW_C64) return LSW_ERR_INVALID_ARG;
    if (nbatch == 0) return LSW_OK;
    if (!u || !y || y == u || (u0 && y == u0)) return LSW_ERR_INVALID_ARG;
    const size_t elem = prec == LSW_C128 ? sizeof(double2) : sizeof(float2);
    const size_t need = elem * 2 * (size_t)g->nz * g->nx * (size_t)nbatch;
    if (need > kNoAllocScratchBytes) return LSW_ERR_UNSUPPORTED_SIZE;
    if (mode != LSW_OP_FORWARD && mode != LSW_OP_RESIDUAL) u0 = nullptr;
    void* scratch = nullptr;
    LSW_TRY(scratch_on_current_device(&scratch));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // Pass A writes every entry of the scratch before passes B and C read it,
    // so nothing left by an earlier call needs clearing.
    OpGeom geo{g->nz, g->nx, chi, g->nz, nullptr, 1};
    if (prec == LSW_C128)
        return op_apply<double>(g, g->full, geo, mode, (const double2*)u, (const double2*)u0, (double2*)y, nbatch,
                                (double2*)scratch, st);
    return op_apply<float>(g, g->full, geo, mode, (const float2*)u, (const float2*)u0, (float2*)y, nbatch,
                           (float2*)scratch, st);
}
