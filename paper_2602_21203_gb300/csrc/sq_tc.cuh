// BF16 tensor-core GEMM interface (tcgen05 + TMA, sm_103a).
#pragma once

#include "sq_common.cuh"

namespace sq {

// A BF16 (or FP8 e4m3) operand in global memory.  K-major: element (mn, k) at
// ptr[mn * ld + k]; MN-major: element (mn, k) at ptr[k * ld + mn].  ptr 16-byte
// aligned, ld x element size a multiple of 16 bytes.
struct TcOperand {
    const void* ptr;
    int64_t ld;
    bool mn_major;
};

// D[M, N] = sum over pairs q of A_q[M, K] B_q[N, K]^T (+ bias[n]) (* (mask[m, n] > 0)),
// FP32 accumulation; D written as FP32 (c, ldc) and/or BF16 (cbf, ldcbf).
struct TcGemm {
    int M, N, K;
    int n_pairs;              // 1 or 2
    TcOperand a[2], b[2];
    const float* bias;
    float* c; int64_t ldc;
    __nv_bfloat16* cbf; int64_t ldcbf;
    const float* mask; int64_t ldmask;
    int accumulate;           // c += D instead of c = D
    // fp8 = 1: A and B are e4m3 (K-major, one pair) holding x / scale per tensor; D is
    // scaled back by *scale_a * *scale_b before the bias (device scalars).  fp8 = 2
    // (MX-FP8): A and B are e4m3 with block scales sf_a / sf_b in the atoms written by
    // launch_quantize_mx (per 32 elements of K of each row of A and of B), applied by the
    // block-scaled MMAs (kind::mxf8f6f4).
    int fp8;
    const float* scale_a; const float* scale_b;
    const uint8_t* sf_a; const uint8_t* sf_b;
    // LayerNorm of each output row fused into the epilogue (ln_g non-null): c receives
    // D + bias (the pre-activation), then y = (D - mean) rstd g + beta, ReLU if ln_relu,
    // goes to ln_post (FP32, row stride N) and ln_posth (BF16, row stride N), with the
    // row statistics in ln_mean / ln_rstd.  The N columns of a row block form one
    // cluster whose CTAs exchange row sums through distributed shared memory; needs
    // N <= 128 x tc_max_cluster(), no K split, and cbf == nullptr.
    const float* ln_g; const float* ln_beta;
    float* ln_post; __nv_bfloat16* ln_posth;
    float* ln_mean; float* ln_rstd;
    float ln_eps; int ln_relu;
};
// Largest cluster the GEMM kernel can be launched with on this device (after tc_prepare).
int tc_max_cluster();

// Per-tensor e4m3 quantisation of BF16 rows (current scaling): scale = amax / 448,
// dst = e4m3(x / scale) rounded to nearest, pad columns zero, *scale written.
// Two launches per batch: block maxima of |x| into `part`, then every block takes
// the maximum over those partials (no atomics: the scale is the same every run).
struct QuantItem {
    const __nv_bfloat16* src; int64_t src_ld;
    int rows, cols;
    uint8_t* dst; int64_t dst_ld;   // dst_ld >= cols, a multiple of 16
    float* scale;
    uint8_t* sf = nullptr;          // MX-FP8: block-scale atoms (launch_quantize_mx)
};
constexpr int kQuantMaxItems = 8;
constexpr int kF8Scales = 64;         // activation scales per stream arena (FP8 learner)
constexpr int kQuantBlocks = 64;      // row blocks per item in the amax pass
int64_t quant_workspace();            // floats of `part`
void launch_quantize_e4m3(const QuantItem* items, int n, float* part, cudaStream_t s);
// MX-FP8 (block-scaled e4m3, OCP MX layout of one scale per 32 elements of a row): one
// launch.  Per 32-element block of a row, scale 2^e with e the smallest integer such that
// max|x| <= 448 2^e (e >= -127), UE8M0 byte e + 127; dst = e4m3(x 2^-e) rounded to
// nearest even, pad columns zero.  The scale bytes go to `sf` in the atoms the GEMM
// reads: for row r and 32-column block j, atom (r / 128) * ceil(cols / 128) + j / 4 of
// 512 bytes, byte (r % 32) * 16 + ((r % 128) / 32) * 4 + j % 4 (rows up to the end of
// the last 128-row tile get zero bytes).  mx_scale_bytes(rows, cols) bytes.
int64_t mx_scale_bytes(int rows, int cols);
void launch_quantize_mx(const QuantItem* items, int n, cudaStream_t s);

// Launches one grouped kernel per up to 4 problems (all of one A/B majorness).  When
// the launch has few output tiles and a long K, the K range of each tile is split over
// a thread-block cluster of up to 8 CTAs; the CTAs add their partial tiles through
// distributed shared memory in rank order, so the result is the same on every run.
// Returns 0, or < 0 if a tensor map cannot describe an operand (alignment, extents).
// *err (device int) receives a nonzero code if a bounded wait gave up.
// allow_split = false keeps every output row's arithmetic independent of the other
// rows of the launch (no K split), e.g. for inference whose result must not depend
// on which requests share the batch.
// Bounded waits of a launch: `cycles` per wait (0: the default, about 2 s); `stall` (failure
// tests only) makes the producer issue no operand loads, so the first operand wait runs out.
struct TcWait { long long cycles; int stall; };
int launch_tc_gemm(const TcGemm* probs, int n_probs, int* err, cudaStream_t s, bool allow_split = true,
                   const TcWait* wait = nullptr);
// Opt the kernels in to their shared memory and resolve the tensor-map encoder (call outside capture).
void tc_prepare();

// 3x3 convolution, 32 -> 32 channels, stride 1, on padded-HWC BF16 activations
// (per image (H+4) x (W+4) rows of 32 channels, valid pixels at (y+2, x+2)).
// Forward: in = padded input (grid width Wp = W+4, in_rows = (H+4) Wp), off0 = 2 Wp + 2,
// w = forward filter layout.  Data gradient: in = padded gradient of the output
// (Wp = OW+4), off0 = 0, w = data-gradient filter layout, mask = padded activation
// below (outputs zeroed where it is <= 0).  Output pixel (oy, ox) < (out_h, out_w).
struct ConvTc {
    const __nv_bfloat16* in;
    int nimg, in_rows, Wp, out_h, out_w, off0;
    const __nv_bfloat16* w;
    const float* bias;
    int relu;
    const __nv_bfloat16* mask;
    __nv_bfloat16* out_phwc;
    float* out_chw;
    __nv_bfloat16* out_chw_bf;
};
int launch_conv32_tc(const ConvTc& c, int* err, cudaStream_t s);
// Weight gradient: x = padded layer input (Wp = W+4), dy = padded gradient at the
// layer's pre-activation (out_h x out_w); dw [32, 32, 3, 3] and db [32] written.
struct WgradTc {
    const __nv_bfloat16* x;
    const __nv_bfloat16* dy;
    int nimg, in_rows, Wp, out_h, out_w;
};
int64_t wgrad32_tc_workspace(int nimg);
int launch_wgrad32_tc(const WgradTc& c, float* work, float* dw, float* db, int* err, cudaStream_t s);
// The same in two parts: CTA i adds images [i per_cta, (i + 1) per_cta) into partial
// tile work[i] (kCh x (9 kCh + 1) floats); the reduce adds work[0 .. ctas) in order.
// wgrad32_per_cta(n) is the split launch_wgrad32_tc uses for n images, so a batch
// processed in chunks of a multiple of it, each chunk's partials written at its first
// image / per_cta, reduces to the same bits as one launch over the whole batch.
int wgrad32_per_cta(int nimg);
int launch_wgrad32_tc_partials(const WgradTc& c, int per_cta, float* work, int* err, cudaStream_t s);
void launch_wgrad32_reduce(const float* work, int ctas, float* dw, float* db, cudaStream_t s);
void conv_tc_prepare();
void launch_to_phwc(const float* src, int64_t img_stride, int nimg, int H, int W, __nv_bfloat16* dst, cudaStream_t s);
void launch_from_phwc(const __nv_bfloat16* src, int nimg, int H, int W, float* dst, cudaStream_t s);
// FP32 filter [32, 32, 3, 3] -> BF16 forward and data-gradient layouts (18432 B each).
void launch_conv_weight_cast(const float* w, __nv_bfloat16* fwd, __nv_bfloat16* bwd, cudaStream_t s);

// FP32 rows -> BF16 rows of a padded matrix (columns cols..dst_ld-1 set to zero).
struct CastItem { const float* src; int64_t src_ld; int rows, cols; __nv_bfloat16* dst; int64_t dst_ld; };
void launch_cast_rows(const CastItem* items, int n, cudaStream_t s);

}  // namespace sq
