// Fused LayerNorm-MLP forward on tcgen05 (sm_103a): one launch evaluates a whole head
// chain  Linear -> LayerNorm -> ReLU -> ... -> Linear  for blocks of 128 rows.
#pragma once

#include "sq_tc.cuh"

namespace sq {

constexpr int kMlpMaxHidden = 3;
constexpr int kMlpMaxProbs = 2;

// Saved activations of one hidden layer (each optional): the pre-activation W h + b
// (FP32, row stride H), the LayerNorm + ReLU output (FP32 and BF16, row stride H) and
// the row statistics.
struct MlpTcSave {
    float* pre; float* post; __nv_bfloat16* posth; float* mean; float* rstd;
};

// One parameter set evaluated on M rows of X.  Hidden layer l: w[l] [H, in_l] BF16
// (in_0 = kin, in_l = H), row stride ldw[l], bias[l], LayerNorm gain g[l] and shift
// beta[l]; the output layer: w[nh] [nout, H], bias[nh].  out: FP32 [M, nout], row
// stride ldo.  X: BF16 [M, kin], row stride ldx (a multiple of 8).
struct MlpTcProblem {
    int M;
    const __nv_bfloat16* x; int64_t ldx; int kin;
    const __nv_bfloat16* w[kMlpMaxHidden + 1]; int64_t ldw[kMlpMaxHidden + 1];
    const float* bias[kMlpMaxHidden + 1];
    const float* g[kMlpMaxHidden]; const float* beta[kMlpMaxHidden];
    MlpTcSave save[kMlpMaxHidden];
    float* out; int64_t ldo;
};

// Whether the fused kernel takes this shape: 1 <= nh <= 3 hidden layers of equal width
// H (a multiple of 32, at most 1024), 1 <= nout <= 256, kin <= 1024.
bool mlp_tc_supported(int nh, int H, int nout, int kin);
// Cluster size (CTAs sharing a row block, each computing H / CL columns of every hidden
// layer) the launcher would pick for H; `force` (1, 2, 4 or 8) if the shape allows it.
int mlp_tc_cluster(int H, int nout, int force = 0);
// Launches the n (<= 2) problems as one grid.  Returns 0, or < 0 if a shape or operand
// cannot be described (the caller then uses the layer-by-layer path).
int launch_mlp_tc(const MlpTcProblem* p, int n, int nh, int H, int nout, float eps, int* err, const TcWait* wait,
                  cudaStream_t s, int force_cluster = 0);
void mlp_tc_prepare();

// Backward through the same head (the input-gradient chain; its weight gradients are
// left to GEMMs): dout BF16 [M, nout] (row stride ld_dout, a multiple of 8); the weights
// as in the forward; the forward's saves of every hidden layer (pre-activation and
// LayerNorm + ReLU output FP32 with row stride H, row statistics).  Per hidden layer,
// optionally: dpre_bf, the gradient at its pre-activation in BF16 [M, H], and colpart,
// [ceil(M / 128)][3][H] per 128-row block column sums of dn xhat, dn and dpre (dn the
// gradient at the LayerNorm output after the ReLU mask): the gain, shift and bias
// gradients once the row blocks are added.  dx FP32 [M, ncols] (row stride lddx)
// receives columns [c0, c0 + ncols) of the input gradient; ncols = 0 stops the chain at
// dpre_0 (then dpre_bf[0] is required and w[0] unused), for callers that form the input
// gradient themselves (e.g. summed over a critic pair).  With the LayerNorm shifts beta
// given (every hidden layer's, saves written by the fused forward, which rounds the
// LayerNorm output as fma(g, xhat, beta)), the ReLU mask is rebuilt from pre by the same
// expression and post is not read; without them post is required.
struct MlpTcBwdProblem {
    int M;
    const __nv_bfloat16* dout; int64_t ld_dout;
    const __nv_bfloat16* w[kMlpMaxHidden + 1]; int64_t ldw[kMlpMaxHidden + 1];
    const float* g[kMlpMaxHidden]; const float* beta[kMlpMaxHidden];
    const float* pre[kMlpMaxHidden]; const float* post[kMlpMaxHidden];
    const float* mean[kMlpMaxHidden]; const float* rstd[kMlpMaxHidden];
    __nv_bfloat16* dpre_bf[kMlpMaxHidden];
    float* colpart[kMlpMaxHidden];
    float* dx; int64_t lddx;
};
// Shapes the fused backward takes: those of the forward, c0 a multiple of 8, and ncols
// either a multiple of 64 per CTA of the cluster, at most 64, or 0.
// force_cluster (1, 2, 4 or 8): the cluster size to use if the shape allows it.
bool mlp_bwd_tc_supported(int nh, int H, int nout, int kin, int c0, int ncols, int force_cluster = 0);
int launch_mlp_bwd_tc(const MlpTcBwdProblem* p, int n, int nh, int H, int nout, int kin, int c0, int ncols, int* err,
                      const TcWait* wait, cudaStream_t s, int force_cluster = 0);
void mlp_bwd_tc_prepare();

}  // namespace sq
