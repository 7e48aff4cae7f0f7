// Allocation-free variant of the convolution weight gradient.
//
// Some callers cannot allocate device memory at the point where they need this
// gradient: code that runs while a memory pool is frozen or fully reserved by
// another framework, a real-time control loop that forbids allocator calls (and
// their implicit synchronisation) after start-up, or an embedding host whose
// allocator is not the CUDA one.  The ordinary entry point asks the caller for a
// workspace; this one keeps its split partial sums in a fixed array that lives in
// the library's device image instead.
#include "squint.h"
#include "squint_ops.h"
#include "sq_kernels.cuh"

#include <cuda.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>

namespace sq {
extern thread_local std::string g_last_error;
}

namespace {

// 1 Mi floats (4 MiB): room for the split partials of every encoder layer of the
// training-shape workload (batch 512, 32 channels) with margin.  Each device that
// loads the library holds this array until the process exits.
constexpr int64_t kScratchFloats = int64_t(1) << 20;
static __device__ __align__(256) float g_wgrad_scratch[kScratchFloats];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

std::mutex g_mu;
// (device ordinal, context id) -> device address of g_wgrad_scratch in that context.  The
// context id is unique within the process, so a context torn down and created again
// (cudaDeviceReset) gets a fresh lookup instead of a stale address.
std::map<std::pair<int, unsigned long long>, float*> g_scratch_addr;

// Id of the calling thread's current context, from the driver (resolved once).
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_ctx = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    CUcontext ctx = nullptr;
    if (!get_ctx || !get_id || get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current device's context, looked up once
// per context (the host-side name is only a handle for the runtime, not an address).
float* scratch_on_current_device(int* rc) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { *rc = SQUINT_ECUDA; return nullptr; }
    unsigned long long ctx_id = 0;
    std::lock_guard<std::mutex> lk(g_mu);
    if (current_context_id(&ctx_id)) {
        auto it = g_scratch_addr.find(std::make_pair(dev, ctx_id));
        if (it != g_scratch_addr.end()) return it->second;
    }
    // the lookup also makes the device's context current on this thread if none was
    float* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_wgrad_scratch);
    if (e != cudaSuccess || !ptr) {
        sq::g_last_error = std::string("cudaGetSymbolAddress of the weight-gradient scratch failed: ") +
                           cudaGetErrorString(e);
        *rc = SQUINT_ECUDA;
        return nullptr;
    }
    if (!current_context_id(&ctx_id)) {
        sq::g_last_error = "weight-gradient scratch: the current CUDA context could not be identified";
        *rc = SQUINT_ECUDA;
        return nullptr;
    }
    g_scratch_addr[std::make_pair(dev, ctx_id)] = ptr;
    return ptr;
}

}  // namespace

extern "C" {

int64_t squint_op_conv3x3_wgrad_noalloc_max(void) { return kScratchFloats; }

int squint_op_conv3x3_wgrad_noalloc(int nimg, int cin, int h, int w, int cout, int stride, const float* x,
                                    const float* dy, float* dw, float* db, void* stream) {
    if (nimg < 0 || cin < 1 || cout < 1 || h < 3 || w < 3 || stride < 1 || !x || !dy || !dw || !db)
        return SQUINT_EINVAL;
    sq::ConvShape sh{};
    sh.nimg = nimg; sh.Cin = cin; sh.H = h; sh.W = w; sh.Cout = cout; sh.stride = stride;
    sh.OH = (h - 3) / stride + 1;
    sh.OW = (w - 3) / stride + 1;
    sh.x_img_stride = (int64_t)cin * h * w;
    sh.y_img_stride = (int64_t)cout * sh.OH * sh.OW;
    const int64_t need = sq::conv_wgrad_workspace(sh);
    if (need > kScratchFloats) {
        sq::g_last_error = "conv3x3 weight gradient: these shapes need " + std::to_string(need) +
                           " scratch floats, more than the fixed " + std::to_string(kScratchFloats);
        return SQUINT_EINVAL;
    }
    // an error some earlier call left pending is reported as such, not as this launch's
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        sq::g_last_error = std::string("a CUDA error from an earlier call is pending: ") + cudaGetErrorString(pending);
        return SQUINT_ECUDA;
    }
    int rc = SQUINT_OK;
    float* scratch = scratch_on_current_device(&rc);
    if (!scratch) return rc;
    // every partial the reduction reads is written by this call first: nothing to clear
    sq::launch_conv_wgrad<float>(sh, dy, x, dw, db, scratch, (cudaStream_t)stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        sq::g_last_error = std::string("conv3x3 weight gradient launch: ") + cudaGetErrorString(e);
        return SQUINT_ECUDA;
    }
    return SQUINT_OK;
}

}  // extern "C"
