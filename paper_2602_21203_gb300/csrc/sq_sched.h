// Building blocks of the launch schedule shared by the update and inference.
#pragma once

#include "sq_internal.h"
#include "sq_tc.cuh"

namespace sq {

// An activation or gradient matrix: FP32 rows plus an optional BF16 shadow
// (the operand the tensor-core GEMMs read).
struct Mat {
    float* f = nullptr;
    int64_t ld = 0;
    __nv_bfloat16* h = nullptr;
    int64_t ldh = 0;
    Mat rows(int64_t r0) const {
        Mat m = *this;
        if (m.f) m.f += r0 * ld;
        if (m.h) m.h += r0 * ldh;
        return m;
    }
};

// A linear layer of one parameter set: FP32 weight [out, in] and bias, BF16 padded
// copy of the weight, and the LayerNorm that follows it (g == null: output layer).
struct LayerRef {
    const float* w = nullptr;
    const float* b = nullptr;
    const __nv_bfloat16* wh = nullptr;
    int64_t ldh = 0;
    const uint8_t* w8 = nullptr;     // e4m3 copy (FP8 mode), row stride ld8, scale *s8
    int64_t ld8 = 0;
    const float* s8 = nullptr;
    const uint8_t* sf8 = nullptr;    // MX block scales of w8 (MX-FP8 mode)
    int in = 0, out = 0;
    const float* g = nullptr;
    const float* beta = nullptr;
};
using MlpRef = std::vector<LayerRef>;

// Collects dense contractions of one kind and launches them as one grouped
// kernel: CUDA-core FP32 (plain path) or tcgen05 BF16 (tensor-core path).
class GemmBuilder {
public:
    GemmBuilder(squint_handle* h, cudaStream_t s, bool bf16, bool split = true)
        : h_(h), s_(s), bf_(bf16), split_(split) {}
    ~GemmBuilder() { flush(); }
    // Y = X W^T + b   (Yh: optional BF16 copy of Y).  With `ln` (tensor-core path only),
    // the LayerNorm (+ReLU) of Y's rows is computed in the same kernel; returns whether
    // it was (otherwise the caller runs the LayerNorm kernel).
    bool fwd(const Mat& X, int rows, const LayerRef& W, float* Y, int64_t ldy, __nv_bfloat16* Yh = nullptr,
             int64_t ldyh = 0, const LnProblem* ln = nullptr, bool relu = false);
    // dX[:, 0:ncols] = sum_q dY_q W_q[:, col0:col0+ncols]  (* (mask > 0))
    void dx(const Mat* dY, const LayerRef* W, int n_pairs, int rows, int col0, int ncols, float* dX, int64_t ldx,
            const float* mask = nullptr, int64_t ldm = 0);
    // dW = dY^T X
    void dw(const Mat& dY, int rows, const Mat& X, const LayerRef& W, float* dW);
    void flush();

private:
    squint_handle* h_;
    cudaStream_t s_;
    bool bf_;
    bool split_;
    std::vector<GemmProblem> fp_;
    GemmLayout lay_ = kKK;
    std::vector<TcGemm> tc_;
    std::vector<TcGemm> tcln_;       // problems with the LayerNorm epilogue (launched apart)
    std::vector<TcGemm> tc8ln_;
    std::vector<TcGemm> tc8_;        // FP8 forward problems; A is quantised at flush
    std::vector<QuantItem> q8_;
    int64_t arena_used_ = 0;
    double qbytes_ = 0;
    double flops_ = 0;
    const char* kind_ = "gemm";
};

// Times the launches made while it lives (kernel profiling only; no-op otherwise).
struct ProfScope {
    squint_handle* h;
    cudaStream_t s;
    int idx = -1;
    ProfScope(squint_handle* hh, cudaStream_t ss, const char* name, double work, int unit) : h(hh), s(ss) {
        if (!h->prof) return;
        squint_handle::ProfEntry e{name, nullptr, nullptr, work, unit, h->lane_of(s)};
        cudaEventCreate(&e.a);
        cudaEventCreate(&e.b);
        squint_handle::record_timing(e.a, s);
        h->prof->push_back(e);
        idx = (int)h->prof->size() - 1;
    }
    ~ProfScope() {
        if (idx >= 0) squint_handle::record_timing((*h->prof)[idx].b, s);
    }
};

// Forward of E parameter sets of one MLP shape on `rows` rows of X (split = false: no
// K split in the tensor-core GEMMs, so each row's result is independent of the others).
// On the BF16 path the whole chain is one fused launch when its shape allows (each row's
// result is independent of the other rows there too).
// keep = false: only the output is needed (no backward through this evaluation), so the
// hidden layers' activations need not be saved.  r0 (one parameter set only): the rows
// are rows r0 .. r0 + rows of the buffers (outputs and saves), X already pointing at them.
void mlp_forward(squint_handle* h, MlpBufs& mb, const MlpRef* sets, int E, const Mat& X, int rows, bool bf16,
                 cudaStream_t s, bool split = true, bool keep = true, int r0 = 0);
// Layer view of canonical layer `ly` in the online parameters (base == params), the
// target copy (target == true) or an inference snapshot (base == a policy buffer; its
// BF16 weight copy, if any, is filled in by the caller).
LayerRef layer_ref(squint_handle* h, const Lin& ly, bool target, const float* base = nullptr);
MlpRef mlp_ref(squint_handle* h, const std::vector<Lin>& layers, bool target, const float* base = nullptr);
GemmProblem lin_fwd(const float* X, int64_t ldx, int rows, const float* W, const float* b, int in, int out, float* Y,
                    int64_t ldy);

}  // namespace sq
