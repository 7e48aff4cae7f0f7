/*
 * squint_ops.h - layer operations of the Squint learner on caller-owned device
 * buffers.  They are the kernels the update is built from, exposed one by one so
 * that each forward and hand-written backward can be checked on its own (finite
 * differences in FP64, the FP64 oracle) and wrapped as autograd functions.
 *
 * Conventions: every pointer is a device pointer the caller owns; `stream` is a
 * cudaStream_t as void*; calls are asynchronous on it.  Return value 0, or
 * SQUINT_EINVAL (-1) for a bad argument / unsupported dtype, SQUINT_ECUDA (-3)
 * if the launch failed.  Row-major layouts throughout.
 */
#ifndef SQUINT_OPS_H
#define SQUINT_OPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SQUINT_DT_F32 0
#define SQUINT_DT_F64 1
#define SQUINT_DT_BF16 2   /* BF16 operands, FP32 accumulation and output (tensor cores) */

/*
 * C[m, n] (+)= sum_k A(m, k) B(n, k) + bias[n] for m < M, n < N.
 * A(m, k) = A[m * sa_m + k * sa_k], B(n, k) = B[n * sb_n + k * sb_k];
 * C[m * ldc + n].  F32/F64: A, B, C, bias of that type, any strides.
 * BF16: A and B BF16 with one unit stride each (sa_k == 1: K-major, sa_m == 1:
 * M-major; likewise for B), 16-byte aligned, the other stride a multiple of 8;
 * C and bias FP32.  This is the dense contraction of every linear layer (Sec. III:
 * critic and actor networks): forward X W^T, data gradient dY W, weight gradient dY^T X.
 * BF16 products with few 128 x 128 output tiles and a long K split K over a cluster of
 * CTAs whose partial tiles are added in a fixed order: repeated calls give identical bits.
 */
int squint_op_gemm(int dtype, int M, int N, int K, const void* A, int64_t sa_m, int64_t sa_k, const void* B,
                   int64_t sb_n, int64_t sb_k, void* C, int64_t ldc, const void* bias, int accumulate, void* stream);


/*
 * The input-gradient chain of the same head in one BF16 tensor-core launch (the
 * backward of the critic and actor MLPs in Alg. 1's critic and actor steps):
 *   dpost_{nh-1} = dout W_nh;  for l = nh-1 .. 0: dn = dpost_l (x) [post_l > 0],
 *   dxh = dn (x) g_l, dpre_l = rstd_l (dxh - mean_row(dxh) - xhat_l mean_row(dxh (x) xhat_l))
 *   with xhat_l = (pre_l - mean_l) rstd_l;  dpost_{l-1} = dpre_l W_l (l > 0);
 *   dx = dpre_0 W_0[:, c0 : c0 + ncols].
 * dout BF16 [M, nout] (row stride ld_dout, a multiple of 8); w, ldw as for
 * squint_op_mlp_bf16; g[l] FP32; pre[l], post[l] FP32 [M, H] and mean[l], rstd[l] [M]:
 * the forward's saves.  beta (optional, every hidden layer's LayerNorm shift): the mask
 * [post_l > 0] is rebuilt as [fma(g_l, xhat_l, beta_l) > 0], the rounding with which
 * squint_op_mlp_bf16 forms post_l, and post may be NULL; without beta post is read.
 * Every dpre_l is rounded to BF16 before the next product reads it.
 * Optional per hidden layer (NULL arrays or entries): dpre_bf[l] BF16 [M, H], and
 * colpart[l] FP32 [ceil(M / 128)][3][H], per 128-row block the column sums of dn xhat,
 * dn and dpre (FP32, before rounding), whose sums over the row blocks are the LayerNorm
 * gain, shift and the linear bias gradients.  dx FP32 [M, ncols] (row stride lddx).
 * Shapes: those of squint_op_mlp_bf16, c0 a multiple of 8, c0 + ncols <= kin, and ncols
 * a multiple of 64 per CTA of the cluster the kernel picks, or at most 64 (SQUINT_EINVAL
 * otherwise).
 */
int squint_op_mlp_bwd_bf16(int M, int kin, int nh, int H, int nout, const void* dout, int64_t ld_dout,
                           const void* const* w, const int64_t* ldw, const float* const* g,
                           const float* const* beta, const float* const* pre, const float* const* post,
                           const float* const* mean, const float* const* rstd, void* const* dpre_bf,
                           float* const* colpart, int c0, int ncols, float* dx, int64_t lddx, void* stream);

/*
 * FP32 rows to BF16 rows with round-to-nearest-even (the rounding of every BF16 operand
 * the tensor-core path reads): dst[r, c] = bf16(src[r, c]) for c < cols, and zero in the
 * pad columns cols <= c < ld_dst.  Row strides in elements.
 */
int squint_op_cast_bf16(int rows, int cols, const float* src, int64_t ld_src, void* dst, int64_t ld_dst,
                        void* stream);

/*
 * A whole LayerNorm MLP head in one BF16 tensor-core launch (the critic and actor MLPs,
 * Sec. IV "Normalization": nh hidden layers Linear -> LayerNorm -> ReLU, then a plain
 * Linear output layer; Alg. 1 evaluates them in every step of the update):
 *   h_0 = x;  pre_l = h_l W_l^T + bias_l;  h_{l+1} = ReLU(LN(pre_l) g_l + beta_l)  (l < nh)
 *   out = h_nh W_nh^T + bias_nh
 * x BF16 [M, kin] (row stride ldx >= kin, a multiple of 8, 16-byte aligned); w[l] BF16
 * [out_l, in_l] row-major with row stride ldw[l] (in_0 = kin, out_l = in_{l+1} = H,
 * out_nh = nout; strides multiples of 8); bias[l], g[l], beta[l] FP32.  Every hidden
 * layer's output is rounded to BF16 before the next layer reads it; accumulation and
 * LayerNorm statistics are FP32 (rstd = 1 / sqrt(var + eps), var the mean square
 * deviation).  out FP32 [M, nout] (row stride ldo).  Optional per hidden layer (arrays
 * of nh pointers, or NULL arrays / NULL entries): pre FP32 [M, H], post FP32 [M, H],
 * post_bf BF16 [M, H], mean and rstd [M].  Shapes: 1 <= nh <= 3, H a multiple of 32 up
 * to 1024, nout <= 256, kin <= 1024 (SQUINT_EINVAL outside).  cluster = 0 picks the
 * number of CTAs that share a 128-row block (each computing H / cluster columns); 1, 2,
 * 4 or 8 forces it when the shape allows.  Each row's result does not depend on the other
 * rows of the call.
 */
int squint_op_mlp_bf16(int M, int kin, int nh, int H, int nout, const void* x, int64_t ldx, const void* const* w,
                       const int64_t* ldw, const float* const* bias, const float* const* g,
                       const float* const* beta, float eps, float* out, int64_t ldo, float* const* pre,
                       float* const* post, void* const* post_bf, float* const* mean, float* const* rstd, int cluster,
                       void* stream);

/*
 * BF16 linear layer with its LayerNorm in one kernel (the hidden layers of the critic and
 * actor MLPs, Sec. IV "Normalization"): pre = A B^T + bias (A [M, K], B [N, K] BF16,
 * row-major, row strides lda, ldb >= K, multiples of 8), then per row
 * post = (pre - mean) rstd g + beta with rstd = 1 / sqrt(var + eps), ReLU if relu;
 * pre and post FP32 [M, N], post_bf (optional) BF16 [M, N], mean and rstd [M].  The
 * column tiles of each 128-row block run as one thread-block cluster and exchange row
 * sums through distributed shared memory; N up to 1024 (SQUINT_EINVAL above what the
 * device can co-schedule).
 */
int squint_op_gemm_layernorm(int M, int N, int K, const void* A, int64_t lda, const void* B, int64_t ldb,
                             const float* bias, const float* g, const float* beta, float eps, int relu, float* pre,
                             float* post, void* post_bf, float* mean, float* rstd, void* stream);

/*
 * FP8 (e4m3) GEMM with per-tensor scaling, FP32 accumulation (the reduced-precision
 * form tried for the forward linear layers): A [M, K] and B [N, K] are BF16, row
 * stride lda / ldb >= K; each is quantised as a whole, scale = max|x| / 448 and
 * x_q = e4m3(x / scale) rounded to nearest; then C[m, n] = scale_A scale_B
 * sum_k A_q(m, k) B_q(n, k) + bias[n] on tcgen05 (kind::f8f6f4).  `work`: caller-owned
 * device memory, 16-byte aligned, squint_op_gemm_fp8_workspace(M, N, K) bytes; it
 * holds the quantised operands and their scales (two floats at byte offset 2048).
 */
size_t squint_op_gemm_fp8_workspace(int M, int N, int K);
int squint_op_gemm_fp8(int M, int N, int K, const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                       int64_t ldc, const float* bias, void* work, size_t work_bytes, void* stream);

/*
 * MX-FP8 (block-scaled e4m3; OCP Microscaling format: one power-of-two scale per 32
 * consecutive elements of a row), the finer-grained form of the reduced-precision
 * forward layers.
 *
 * squint_op_quantize_mxfp8: BF16 src [rows, cols] (row stride ld >= cols) -> e4m3 codes
 * dst [rows, dst_ld] (dst_ld >= cols, a multiple of 16; columns cols .. dst_ld-1 zero)
 * and UE8M0 scale bytes `sf` (squint_op_mx_scale_bytes(rows, cols) bytes).  Block j of
 * row r (columns 32 j .. 32 j + 31) gets e = the smallest integer with
 * max|x| <= 448 2^e (448 = largest finite e4m3; e >= -127, e = -127 for an all-zero
 * block), byte e + 127 at sf[((r / 128) ceil(cols / 128) + j / 4) 512 + (r % 32) 16 +
 * ((r % 128) / 32) 4 + j % 4], and codes e4m3(x 2^-e) rounded to nearest even; scale
 * bytes of rows rows .. 128 ceil(rows / 128) - 1 are zero.  Bit-exact.
 *
 * squint_op_gemm_mxfp8: C[m, n] = sum_k 2^(ea(m, k/32) + eb(n, k/32)) A(m, k) B(n, k)
 * + bias[n] for e4m3 A [M, K] (row stride lda), B [N, K] (ldb) with scale bytes sfa,
 * sfb laid out as above (rows of A: M, rows of B: N, cols: K), FP32 accumulation on
 * tcgen05 (kind::mxf8f6f4, block-scaled MMAs).  A, B 16-byte aligned, lda, ldb
 * multiples of 16; bias may be NULL.  All pointers are caller-owned device memory;
 * both calls are asynchronous on `stream`.  SQUINT_EINVAL on bad sizes or alignment.
 */
int64_t squint_op_mx_scale_bytes(int rows, int cols);
int squint_op_quantize_mxfp8(int rows, int cols, const void* src, int64_t ld, void* dst, int64_t dst_ld, void* sf,
                             void* stream);
int squint_op_gemm_mxfp8(int M, int N, int K, const void* A, int64_t lda, const void* sfa, const void* B, int64_t ldb,
                         const void* sfb, float* C, int64_t ldc, const float* bias, void* stream);

/*
 * Squint at insert (Alg. 1 stores the transition with Downsample(o); Sec. IV
 * "Resolution Squinting": area downsampling): n uint8 frames src [n, C, H, W]
 * (H, W multiples of f) become their f x f area means rounded half up,
 * q = (S + f^2/2) / f^2 in integers, written to slots (slot0 + i) mod n_slots of the
 * uint8 ring [n_slots, C, H/f, W/f].  A learner whose ring holds such frames is
 * created with obs_h = H/f, obs_w = W/f, squint_f = 1 and the shift pad at that
 * resolution; it then reads x = q / 255 - 0.5.  Bit-exact integer arithmetic.
 */
int squint_op_squint_store(int n, int C, int H, int W, int f, const void* src, void* ring, int64_t slot0,
                           int64_t n_slots, void* stream);

/*
 * Valid 3x3 convolution, NCHW (the encoder layers, Sec. III "single shared CNN
 * encoder"): y[i,o,p,q] = b[o] + sum_{c,u,v} w[o,c,u,v] x[i,c,s p+u,s q+v], ReLU if relu.
 * x [nimg, cin, h, w], w [cout, cin, 3, 3], y [nimg, cout, oh, ow], oh = (h-3)/s+1.
 */
int squint_op_conv3x3_fwd(int dtype, int nimg, int cin, int h, int w, int cout, int stride, const void* x,
                          const void* wt, const void* b, void* y, int relu, void* stream);
/* Workspace (bytes) the backward below needs for these shapes. */
size_t squint_op_conv3x3_workspace(int dtype, int nimg, int cin, int h, int w, int cout, int stride);
/*
 * Backward of the convolution given dy at its pre-activation: dw, db (always) and
 * dx (if non-NULL; zeroed where dx_mask <= 0 when dx_mask is given).
 */
int squint_op_conv3x3_bwd(int dtype, int nimg, int cin, int h, int w, int cout, int stride, const void* x,
                          const void* wt, const void* dy, void* dx, const void* dx_mask, void* dw, void* db,
                          void* workspace, size_t workspace_bytes, void* stream);

/*
 * Tensor-core convolutions of the encoder's 32 -> 32 channel, stride-1 layers on the
 * padded-HWC BF16 format: per image (H+4) x (W+4) rows of 32 channels, the pixel
 * (y, x) at row (y+2)(W+4) + x+2, zeros on the 2-pixel border (buffers the caller
 * zero-fills once).
 * to/from: NCHW FP32 [nimg, 32, H, W] <-> padded-HWC BF16 (interior only).
 */
int squint_op_to_phwc(int nimg, int H, int W, const float* src, void* dst, void* stream);
int squint_op_from_phwc(int nimg, int H, int W, const void* src, float* dst, void* stream);
/* FP32 filter [32, 32, 3, 3] -> BF16 forward and data-gradient layouts (18432 bytes each). */
int squint_op_conv32_layouts(const float* w, void* fwd_layout, void* dgrad_layout, void* stream);
/*
 * mode 0 (forward): x padded [nimg, H, W] -> y (H-2 x W-2): bias, ReLU if relu;
 * writes padded y (out_phwc, may be NULL) and/or NCHW FP32 y (out_nchw, may be NULL).
 * mode 1 (data gradient): `in` = padded dy [nimg, H, W] -> dx (H+2 x W+2), zeroed where
 * mask (padded activation of size H+2 x W+2) <= 0 when mask is given.
 */
int squint_op_conv32(int mode, int nimg, int H, int W, const void* in, const void* w_layout, const float* bias,
                     int relu, const void* mask, void* out_phwc, float* out_nchw, void* stream);
/*
 * The encoder's first layer on tensor cores (Sec. IV encoder: 3x3 convolution, stride s,
 * no padding, ReLU): x NCHW FP32 [nimg, Cin, H, W] (1 <= Cin <= 16), w FP32
 * [32, Cin, 3, 3], bias [32] -> y = ReLU(conv(x, w) + bias) as padded-HWC BF16 with
 * OH = (H-3)/s + 1, OW = (W-3)/s + 1 (the input format of squint_op_conv32; only the
 * interior is written).  x and w are rounded to BF16, products accumulated in FP32 over
 * k = (ci, ky, kx).  out_phwc 16-byte aligned.
 */
int squint_op_conv0_bf16(int nimg, int Cin, int H, int W, int stride, const float* x, const float* w,
                         const float* bias, void* out_phwc, void* stream);
/* Weight gradient: x padded [nimg, H, W], dy padded [nimg, H-2, W-2] -> dw [32,32,3,3], db [32]. */
size_t squint_op_wgrad32_workspace(int nimg);
int squint_op_wgrad32(int nimg, int H, int W, const void* x, const void* dy, float* dw, float* db, void* work,
                      size_t work_bytes, void* stream);

/*
 * Weight and bias gradient of the FP32 3x3 convolution (dw, db of
 * squint_op_conv3x3_bwd) without any device allocation and without a caller
 * workspace.  This entry point has no counterpart in the paper: it exists for
 * callers that cannot allocate device memory when they need the gradient (a
 * frozen or fully reserved memory pool, a real-time loop that forbids allocator
 * calls and their synchronisation, a host with its own allocator).  Its split
 * partial sums live in one fixed device array of squint_op_conv3x3_wgrad_noalloc_max()
 * floats (4 MiB) that every device loading the library keeps until exit; shapes
 * needing more return SQUINT_EINVAL with a message in squint_last_error().  The
 * first call in each CUDA context of a device (the device's primary context, and
 * again after a cudaDeviceReset) looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make that first call before
 * any stream capture.  A CUDA error left pending by an earlier call is reported as
 * SQUINT_ECUDA before anything is launched.  All calls share the array: two calls
 * whose kernels overlap on the GPU (different streams, or concurrent host threads)
 * race and give wrong results; serialise them.  Each call writes every partial it
 * reads, so nothing carries over between calls.
 */
int64_t squint_op_conv3x3_wgrad_noalloc_max(void);
int squint_op_conv3x3_wgrad_noalloc(int nimg, int cin, int h, int w, int cout, int stride, const float* x,
                                    const float* dy, float* dw, float* db, void* stream);

/*
 * ReLU backward given the ReLU's output: dx[i] = dy[i] if y[i] > 0 else 0 (the
 * nonlinearity after every encoder and hidden layer, Sec. IV).  F32 or F64;
 * dx may alias dy.
 */
int squint_op_relu_bwd(int dtype, int64_t n, const void* dy, const void* y, void* dx, void* stream);

/* LayerNorm over rows of n (Sec. IV "Normalization"), FP32: y = g (x - mean) rstd + b, ReLU if relu. */
int squint_op_layernorm_fwd(int rows, int n, const float* x, const float* g, const float* b, float eps, int relu,
                            float* y, float* mean, float* rstd, void* stream);
/* Backward: dy w.r.t. the output (masked by y > 0 when y is given, i.e. after ReLU). */
int squint_op_layernorm_bwd(int rows, int n, const float* dy, const float* y, const float* x, const float* mean,
                            const float* rstd, const float* g, float* dx, float* dg, float* db, void* stream);

/*
 * Categorical cross entropy against a target distribution m (C51 critic loss,
 * Sec. IV "Critic Design Choices"): row_loss[r] = -sum_j m[r,j] log softmax(l[r])_j,
 * dlogits = (softmax(l) - m) * scale, row_q[r] = sum_j softmax(l[r])_j z_j with
 * z_j = v_min + j (v_max - v_min)/(K-1).
 */
int squint_op_categorical_ce(int rows, int K, const float* logits, const float* m, float v_min, float v_max,
                             float scale, float* dlogits, float* row_loss, float* row_q, void* stream);

/*
 * C51 target (Alg. 1 "Compute target Q-value", distributional form): the E target
 * critics' softmax distributions averaged, the support shifted to
 * clip(r + gamma (1-d)(z_j - alpha logp), v_min, v_max) and projected linearly
 * onto the atoms.  logits [E, rows, K]; r, d, logp [rows]; m [rows, K].
 */
int squint_op_c51_project(int rows, int K, int E, const float* logits, const float* r, const float* d,
                          const float* logp, float alpha, float gamma, float v_min, float v_max, float* m,
                          void* stream);

/*
 * Tanh-Gaussian policy head (SAC, Sec. III) with given noise eps [rows, A]:
 * out [rows, 2A] = (mu, raw); log_std = lo + (hi-lo)(tanh(raw)+1)/2;
 * a = tanh(mu + exp(log_std) eps); logp = log density of a.
 */
int squint_op_tanh_gaussian_fwd(int rows, int A, const float* out, const float* eps, float lo, float hi, float* a,
                                float* logp, void* stream);
/* Backward with eps held fixed: dout from da [rows, A] and dlogp [rows]. */
int squint_op_tanh_gaussian_bwd(int rows, int A, const float* out, const float* eps, const float* da,
                                const float* dlogp, float lo, float hi, float* dout, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SQUINT_OPS_H */
