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

#include <map>
#include <mutex>
#include <string>

namespace sq {
extern thread_local std::string g_last_error;
}

namespace {

// 1 Mi floats (4 MiB): room for the split partials of every encoder layer of the
// training-shape workload (batch 512, 32 channels) with margin.  Each device that
// loads the library holds this array until the process exits.
constexpr int64_t kScratchFloats = int64_t(1) << 20;
static __device__ __align__(256) float g_wgrad_scratch[kScratchFloats];

std::mutex g_mu;
std::map<int, float*> g_scratch_addr;   // device ordinal -> device address of g_wgrad_scratch

// Device address of the scratch array on the current device, looked up once per
// device (the host-side name is only a handle for the runtime, not an address).
float* scratch_on_current_device(int* rc) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { *rc = SQUINT_ECUDA; return nullptr; }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch_addr.find(dev);
    if (it != g_scratch_addr.end()) return it->second;
    float* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_wgrad_scratch);
    if (e != cudaSuccess || !ptr) {
        sq::g_last_error = std::string("cudaGetSymbolAddress of the weight-gradient scratch failed: ") +
                           cudaGetErrorString(e);
        *rc = SQUINT_ECUDA;
        return nullptr;
    }
    g_scratch_addr[dev] = ptr;
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
    int rc = SQUINT_OK;
    float* scratch = scratch_on_current_device(&rc);
    if (!scratch) return rc;
    // every partial the reduction reads is written by this call first: nothing to clear
    sq::launch_conv_wgrad<float>(sh, dy, x, dw, db, scratch, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? SQUINT_OK : SQUINT_ECUDA;
}

}  // extern "C"
