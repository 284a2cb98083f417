// bras_apply_noalloc: the BRAS apply for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: code that owns all device memory through
// its own pool or caching allocator, latency-critical loops where an allocation's implicit
// device synchronisation is not acceptable, or hosts with a hard memory budget fixed up front.
// The regular bras_apply may (re)allocate its workspace for the partial sums of cell-block
// boundary dofs when nrhs grows; this variant never does.  Its partial sums live in one
// fixed, file-scope device array instead.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace bras {
namespace {

// 16 MiB: room for 2 Mi double / 4 Mi float partial sums (partials x nrhs).  Every GPU that
// loads this library keeps this array until the process exits.
constexpr size_t kScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's name
// is only a host-side stand-in, so the address is looked up once per device with that device
// current and cached.
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BRAS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BRAS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return BRAS_OK;
}

}  // namespace
}  // namespace bras

using namespace bras;

extern "C" int bras_apply_noalloc(const bras_ctx* ctx, int precision, const void* x, void* y, int nrhs,
                                  void* stream) {
    set_detail(-1);
    if (!ctx || !x || !y || nrhs < 1 || precision < 0 || precision > 2) return BRAS_ERR_INVALID;
    if (!has_precision(ctx, precision) || (precision == BRAS_FP64 && !has_fp64_bras(ctx))) return BRAS_ERR_PRECISION;
    const size_t w = precision == BRAS_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = part_entries(ctx, nrhs) * w;
    if (need > kScratchBytes) {
        set_detail((int64_t)need);
        return BRAS_ERR_TOO_LARGE;
    }
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != BRAS_OK) return rc;
    // Every partial slot the combine pass reads is written by exactly one block earlier in the
    // same call, so nothing in the shared array needs clearing between calls.  The dispatch is bras_apply's
    // own, so both calls run the same kernel and return the same bits.
    return dispatch_op(ctx, precision, OP_BRAS, x, y, scratch, nrhs, static_cast<cudaStream_t>(stream));
}
