// Kernel launch interfaces of the Squint CUDA library.
#pragma once

#include "sq_common.cuh"

namespace sq {

// ---------------------------------------------------------------- front end
// Steps a1-a4 of one update: minibatch slots, gathers, random shift, squint.
struct CopyDst {
    float* ptr;      // destination rows
    int64_t ld;      // row stride (elements)
    int col;         // first column
    int which;       // 0: proprio[idx], 1: proprio[nxt], 2: action[idx]
    __nv_bfloat16* ptr_h;   // optional BF16 copy (same column, row stride ld_h)
    int64_t ld_h;
};
struct FrontendArgs {
    const uint8_t* obs;
    const float* proprio;
    const float* action;
    const float* reward;
    const uint8_t* done;
    int64_t n_slots;
    int C, H, W, f, pad, P, A, B;
    uint64_t seed;
    const int64_t* update_idx;   // device scalar
    int idx_offset;              // draws of update *update_idx + idx_offset (1: the next one)
    float* x;                    // [2B, C, Hs, Ws]: rows < B are o_t, rows >= B are o_{t+1}
    __nv_bfloat16* x_bf;         // optional BF16 copy of x
    uint16_t* sums;              // optional box sums, same layout
    int32_t* idx_out;            // [2B]: slot of o_t, then slot of o_{t+1}
    int32_t* shift_out;          // [2B, 2] (dx, dy)
    float* r_out;                // [B]
    float* d_out;                // [B]
    CopyDst dst[8];
    int n_dst;
    int* err;                    // device error word: a frame copy that never completed
};
void launch_frontend(const FrontendArgs& a, cudaStream_t s);

// Inference front end: squint without shift for a ragged batch of requests.
struct ActFrontArgs {
    const uint8_t* const* obs;   // device array of per-request obs pointers
    const float* const* prop;    // device array of per-request proprio pointers
    const int32_t* row_req;      // [rows]: request of each row
    const int32_t* row_in_req;   // [rows]: row within its request
    int rows, C, H, W, f, P;
    float* x;                    // [rows, C, Hs, Ws]
    float* xin; int64_t ld_xin; int col;   // proprio goes to xin[row, col:col+P]
};
void launch_act_frontend(const ActFrontArgs& a, cudaStream_t s);
// Opt the front-end kernels in to `frame_bytes` of dynamic shared memory (call once, outside capture).
void frontend_prepare(size_t frame_bytes);
// Squint at insert: n uint8 frames [n, C, H, W] -> rounded f x f area means [C, H/f, W/f]
// into ring slots (slot0 + i) mod n_slots of a uint8 ring [n_slots, C, H/f, W/f].
void launch_squint_store(const uint8_t* src, int n, int C, int H, int W, int f, uint8_t* ring, int64_t slot0,
                         int64_t n_slots, cudaStream_t s);

// ---------------------------------------------------------------- dense contractions (CUDA cores)
// C(m,n) [+]= sum_s sum_k A_s(m,k) B_s(n,k) (+ bias[n]) (* (mask(m,n) > 0)).
struct GemmProblem {
    int M, N, K;
    const void* A;
    int64_t sa_m, sa_k;
    const void* B;
    int64_t sb_n, sb_k;
    void* C;
    int64_t sc_m, sc_n;
    const void* bias;          // [N] or null
    const void* mask;          // or null
    int64_t sm_m, sm_n;
    int accumulate;            // 1: C += result
    int n_sum;                 // summed operand pairs (>= 1)
    int64_t a_sum, b_sum;      // element offset between summed pairs
};
// Operand layouts: KK = A and B k-contiguous; KN = A k-contiguous, B n-contiguous;
// MN = A m-contiguous, B n-contiguous.
enum GemmLayout { kKK = 0, kKN = 1, kMN = 2 };
template <typename T>
void launch_gemm(const GemmProblem* probs, int n_probs, GemmLayout layout, cudaStream_t s);

// Valid 3x3 convolution (NCHW), implicit GEMM on CUDA cores.
struct ConvShape {
    int nimg, Cin, H, W, Cout, stride, OH, OW;
    int64_t x_img_stride;      // elements between images of the input (default Cin*H*W)
    int64_t y_img_stride;      // elements between images of the output (default Cout*OH*OW)
};
// First encoder layer (Cin <= 16, any stride, Cout = 32) with ReLU, written as padded-HWC
// BF16 (grid width OW + 4) for the tensor-core layers; x is NCHW FP32.
void launch_conv0_phwc(const ConvShape& sh, const float* x, const float* w, const float* b, __nv_bfloat16* out,
                       cudaStream_t s);
// The same layer on tensor cores (BF16 operands, FP32 accumulation; Cin <= 16, Cout = 32):
// 0, or < 0 if the shape is outside its range.  A bounded wait that gives up records its
// code in *err.
int launch_conv0_tc(const ConvShape& sh, const float* x, const float* w, const float* b, __nv_bfloat16* out,
                    int* err, cudaStream_t s);
template <typename T>
void launch_conv_fwd(const ConvShape& sh, const T* x, const T* w, const T* b, T* y, bool relu, cudaStream_t s);
// dx = conv-transpose(dy, w) (* (mask > 0) if mask given; mask has the layout of dx).
template <typename T>
void launch_conv_dgrad(const ConvShape& sh, const T* dy, const T* w, T* dx, const T* mask, cudaStream_t s);
// dw, db from dy and x; workspace of conv_wgrad_workspace(sh) elements of T.
int64_t conv_wgrad_workspace(const ConvShape& sh);
template <typename T>
void launch_conv_wgrad(const ConvShape& sh, const T* dy, const T* x, T* dw, T* db, T* work, cudaStream_t s);
// The same for a 32-output layer with Cin * 9 + 1 <= 32 whose output gradient is the
// padded-HWC BF16 image (grid (OH + 4) x (OW + 4), 32 channels) of the tensor-core path;
// returns -1 for other shapes.
int launch_conv_wgrad_phwc(const ConvShape& sh, const __nv_bfloat16* dy_phwc, const float* x, float* dw, float* db,
                           float* work, cudaStream_t s);

// ---------------------------------------------------------------- LayerNorm
struct LnProblem {
    int rows, n;
    const float* pre;  int64_t ld_pre;     // input
    const float* g;    const float* beta;  // affine
    float* out;        int64_t ld_out;     // output (ReLU applied if relu)
    __nv_bfloat16* out_bf; int64_t ld_out_bf;  // optional BF16 copy of out
    float* mean;       float* rstd;        // [rows] statistics
};
void launch_ln_fwd(const LnProblem* p, int n_probs, bool relu, float eps, cudaStream_t s);
struct LnBwdProblem {
    int rows, n;
    const float* dout; int64_t ld_dout;    // gradient w.r.t. the LN(+ReLU) output
    const float* out;  int64_t ld_out;     // forward output (ReLU mask) or null
    const float* pre;  int64_t ld_pre;
    const float* mean; const float* rstd;
    const float* g;
    float* dpre;       int64_t ld_dpre;    // gradient w.r.t. pre (written)
    __nv_bfloat16* dpre_bf; int64_t ld_dpre_bf;  // optional BF16 copy of dpre
    float* dg; float* dbeta;               // column sums (written) or null
    float* dbias;                          // sum of dpre over rows (linear bias grad) or null
    // Deferred column sums: with `terms` set, the row kernel writes dn xh and dn of every
    // element to terms[0 .. rows n) and terms[rows n .. 2 rows n) (row stride n) instead
    // of reducing them, and launch_ln_bwd_cols adds them (and dpre) up later, e.g. on
    // another stream beside the weight-gradient GEMMs.
    float* terms;
};
// Column sums (dg, dbeta, dbias) need `work` of ln_bwd_workspace() floats (null: rows only).
// Its first kLnTickets words are ticket counters that must be zero before the first launch;
// every launch leaves them zero again.  Launches that share a workspace must be stream-ordered.
constexpr int kLnTickets = 64;
int64_t ln_bwd_workspace(const LnBwdProblem* p, int n_probs);
void launch_ln_bwd(const LnBwdProblem* p, int n_probs, float* work, cudaStream_t s);
// Opt the LayerNorm backward in to its shared memory (rows up to 2048 wide; call outside capture).
void ln_prepare();

// Column sums over rows: out[j] = sum_r in[r*ld + j] (deterministic order).
struct ColSumProblem { int rows, n; const float* in; int64_t ld; float* out; };
void launch_colsum(const ColSumProblem* p, int n_probs, cudaStream_t s);
// The deferred column sums of LayerNorm backward problems whose `terms` are set.
void launch_ln_bwd_cols(const LnBwdProblem* p, int n_probs, cudaStream_t s);

// ---------------------------------------------------------------- heads and losses
struct ActorHeadArgs {
    int rows, B, A;                 // rows = 2B: rows < B draw the target noise, rows >= B the actor noise
    const float* out; int64_t ld_out;   // [rows, 2A] mu | raw
    float lo, hi;
    uint64_t seed; const int64_t* update_idx;
    float* a_dst0; int64_t ld0;     // actions of rows < B
    float* a_dst1; int64_t ld1;     // actions of rows >= B
    __nv_bfloat16* a_dst0_h; int64_t ld0_h;   // optional BF16 copies
    __nv_bfloat16* a_dst1_h; int64_t ld1_h;
    float* logp;                    // [rows]
    float* eps;                     // [rows, A] saved noise
    const float* eps_in;            // optional: noise given instead of drawn
    int row0;                       // rows [row0, rows) are computed (0: all)
};
void launch_actor_head(const ActorHeadArgs& a, cudaStream_t s);

struct ActorHeadBwdArgs {
    int B, A;
    const float* out; int64_t ld_out;     // forward head inputs of the B actor rows
    const float* eps;                     // [B, A]
    const float* da; int64_t ld_da;       // dL/da rows (row stride ld_da; 0 means A)
    const float* da2;                     // optional second part of dL/da (same layout), added to da
    const float* log_alpha;               // dL/dlogp = exp(log_alpha)/B
    float lo, hi;
    float* dout;                          // [B, 2A]
    __nv_bfloat16* dout_bf; int64_t ld_dout_bf;   // optional BF16 copy
    const int32_t* do_actor;              // null: always run
    const float* dlogp_rows;              // optional per-row dL/dlogp instead of exp(log_alpha)/B
};
void launch_actor_head_bwd(const ActorHeadBwdArgs& a, cudaStream_t s);

struct C51TargetArgs {
    int B, K, E;
    const float* logits_bar;   // [E, B, K]
    const float* r; const float* d; const float* logp_next;
    const float* log_alpha;    // alpha = exp(*log_alpha); null: alpha_value
    float alpha_value;
    float gamma, v_min, v_max;
    float* m;                  // [B, K]; MSE critic (K = 1): the TD target y
    int cdq;                   // clipped double Q: per sample the target critic with the smaller mean
    int mse;                   // scalar critics (Eq. 1): y = r + gamma (1-d)(Q_bar - alpha log pi')
    // the update's step counters (null: left alone), advanced by one thread before any
    // reader of the update runs: steps [3] critic, actor, alpha; do_actor = whether the
    // actor steps in update *update_idx (every policy_freq-th)
    int32_t* steps; int32_t* do_actor; const int64_t* update_idx; int policy_freq;
};
void launch_c51_target(const C51TargetArgs& a, cudaStream_t s);

struct CeArgs {
    int B, K, E;
    const float* logits;       // [E, B, K]
    const float* m;            // [B, K]
    float v_min, v_max;
    float scale;               // dlogits = (softmax - m) * scale
    float* dlogits;            // [E, B, K]
    __nv_bfloat16* dlogits_bf; int64_t ld_bf;   // optional BF16 copy [E, B, ld_bf]
    float* row_loss;           // [E*B]
    float* row_q;              // [E*B]
    int mse;                   // scalar critics (Eq. 2): loss (Q - y)^2, dQ = 2 (Q - y) scale
};
void launch_ce(const CeArgs& a, cudaStream_t s);

struct ActorQArgs {
    int B, K, E;
    const float* logits;       // [E, B, K] critics on (z_sg, s, a~)
    float v_min, v_max;
    float* dlogits;            // [E, B, K] = -(1/(E B)) p (z - Q)
    __nv_bfloat16* dlogits_bf; int64_t ld_bf;   // optional BF16 copy [E, B, ld_bf]
    float* row_q;              // [E*B]
    const int32_t* do_actor;
    int cdq;                   // clipped double Q: the smaller critic per sample carries the gradient
    int mse;                   // scalar critics: Q is the output itself
};
void launch_actor_q(const ActorQArgs& a, cudaStream_t s);

// log-alpha step (Adam) from the actor log-probs at s_t, plus per-update statistics.
struct AlphaArgs {
    int B;
    const float* logp_t;          // [B]
    float* log_alpha; float* m; float* v;
    int32_t* steps;               // alpha count at steps[2]
    double lr, b1, b2, eps;
    float target_entropy;
    float* stats;                 // [8] per-update statistics
};
void launch_alpha_step(const AlphaArgs& a, cudaStream_t s);

struct StatsArgs {
    int B, E;
    const float* row_loss; const float* row_q;       // critic step
    const float* row_q_actor; const float* logp_t;   // actor step
    const float* log_alpha;
    const int32_t* do_actor;
    int64_t* update_idx;          // read into the statistics, then advanced by one
    float* stats;                 // [8]
    int cdq;                      // actor loss with the smaller critic per sample
};
void launch_stats(const StatsArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- optimiser
// A weight matrix inside an updated range whose padded BF16 copy is written by the same
// kernel: element (r, c) of the rows x cols block at offset `off` from the range start
// goes to dst[r * ld + c] (pad columns are left as they are).
struct BfSeg { int64_t off; int rows, cols; int64_t ld; __nv_bfloat16* dst; };
constexpr int kMaxBfSeg = 8;

struct AdamArgs {
    float* p; const float* g; float* m; float* v; int64_t n;
    const int32_t* step;          // device step count (already incremented)
    double lr, b1, b2, eps;
    const int32_t* enable;        // null or device flag
    __nv_bfloat16* p_bf;          // optional BF16 copy of p
    BfSeg seg[kMaxBfSeg];         // padded BF16 copies of the range's weight matrices
    int n_seg;
    // optional polyak of a target copy in the same pass: target[i] <- (1 - tau) target[i]
    // + tau p_new[i] for i < n, with the padded BF16 copies tseg (matrix k at seg[k]'s
    // offset and shape)
    float* target; float tau;
    BfSeg tseg[kMaxBfSeg];
    int n_tseg;
};
// 0, or -1 if the BF16 copies do not describe the range (overlapping or outside it).
int launch_adam(const AdamArgs& a, cudaStream_t s);

struct PolyakArgs {
    float* target; const float* src; int64_t n; float tau; int64_t* update_idx;
    BfSeg seg[kMaxBfSeg];         // padded BF16 copies of the target weight matrices
    int n_seg;
};
int launch_polyak(const PolyakArgs& a, cudaStream_t s);
// dx = dy * (y > 0), elementwise over n values.
template <typename T> void launch_relu_bwd(int64_t n, const T* dy, const T* y, T* dx, cudaStream_t s);

// Inference head: mean or sampled action per row of a ragged batch.
struct ActHeadArgs {
    int rows, A;
    const float* out; int64_t ld_out;
    const int32_t* row_req; const int32_t* row_in_req;
    const uint64_t* req_key; const int32_t* req_mode;
    float* const* req_actions;   // device array of per-request output pointers
    float lo, hi; uint64_t seed;
};
void launch_act_head(const ActHeadArgs& a, cudaStream_t s);

}  // namespace sq
