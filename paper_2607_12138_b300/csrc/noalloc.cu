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
    if (!has_precision(ctx, precision)) return BRAS_ERR_PRECISION;
    const size_t w = precision == BRAS_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)ctx->npart * (size_t)nrhs * w;
    if (need > kScratchBytes) {
        set_detail((int64_t)need);
        return BRAS_ERR_TOO_LARGE;
    }
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != BRAS_OK) return rc;
    // Every slot the combine pass reads is written by exactly one block earlier in the same
    // call, so nothing in the shared array needs clearing between calls.
    LaunchCommon L = make_launch(ctx, precision, OP_BRAS);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t err;
    const bool h1 = ctx->space == BRAS_H1;
    if (precision == BRAS_FP64) {
        auto* xx = static_cast<const double*>(x);
        auto* yy = static_cast<double*>(y);
        auto* pp = static_cast<double*>(scratch);
        err = h1 ? launch_h1_f64(L, ctx->nloc, OP_BRAS, xx, yy, pp, nrhs, st)
                 : launch_pk_f64(L, ctx->nloc, OP_BRAS, xx, yy, pp, nrhs, st);
    } else {
        auto* xx = static_cast<const float*>(x);
        auto* yy = static_cast<float*>(y);
        auto* pp = static_cast<float*>(scratch);
        if (h1) err = launch_h1_f32(L, ctx->nloc, OP_BRAS, xx, yy, pp, nrhs, st);
        else if (precision == BRAS_BF16) err = launch_pk_bf16(L, ctx->nloc, OP_BRAS, xx, yy, pp, nrhs, st);
        else err = launch_pk_f32(L, ctx->nloc, OP_BRAS, xx, yy, pp, nrhs, st);
    }
    return err == cudaSuccess ? BRAS_OK : BRAS_ERR_CUDA;
}
