// BF16 tensor-core GEMM interface (tcgen05 + TMA, sm_103a).
#pragma once

#include "sq_common.cuh"

namespace sq {

// A BF16 operand in global memory.  K-major: element (mn, k) at ptr[mn * ld + k];
// MN-major: element (mn, k) at ptr[k * ld + mn].  ptr 16-byte aligned, ld a multiple of 8.
struct TcOperand {
    const __nv_bfloat16* ptr;
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
};

// Launches one grouped kernel per up to 4 problems (all of one A/B majorness).
// Returns 0, or < 0 if a tensor map cannot describe an operand (alignment, extents).
// *err (device int) receives a nonzero code if a bounded wait gave up.
int launch_tc_gemm(const TcGemm* probs, int n_probs, int* err, cudaStream_t s);
// Opt the kernels in to their shared memory and resolve the tensor-map encoder (call outside capture).
void tc_prepare();

// FP32 rows -> BF16 rows of a padded matrix (columns cols..dst_ld-1 set to zero).
struct CastItem { const float* src; int64_t src_ld; int rows, cols; __nv_bfloat16* dst; int64_t dst_ld; };
void launch_cast_rows(const CastItem* items, int n, cudaStream_t s);

}  // namespace sq
