// Layer operations (include/squint_ops.h): the update's kernels on caller buffers.
#include "squint.h"
#include "squint_ops.h"
#include "sq_kernels.cuh"
#include "sq_tc.cuh"
#include "sq_mlp_tc.cuh"

#include <cstring>
#include <mutex>
#include <string>

using namespace sq;

namespace sq {
extern thread_local std::string g_last_error;
}

namespace {

int launch_status() { return cudaGetLastError() == cudaSuccess ? SQUINT_OK : SQUINT_ECUDA; }

int* tc_error_flag() {
    static int* flag = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        if (cudaMalloc(&flag, sizeof(int)) == cudaSuccess) cudaMemset(flag, 0, sizeof(int));
        tc_prepare();
        conv_tc_prepare();
        mlp_tc_prepare();
        mlp_bwd_tc_prepare();
    });
    return flag;
}

ConvShape conv_shape(int nimg, int cin, int h, int w, int cout, int stride) {
    ConvShape sh{};
    sh.nimg = nimg; sh.Cin = cin; sh.H = h; sh.W = w; sh.Cout = cout; sh.stride = stride;
    sh.OH = (h - 3) / stride + 1;
    sh.OW = (w - 3) / stride + 1;
    sh.x_img_stride = (int64_t)cin * h * w;
    sh.y_img_stride = (int64_t)cout * sh.OH * sh.OW;
    return sh;
}

bool conv_ok(int nimg, int cin, int h, int w, int cout, int stride) {
    return nimg >= 0 && cin > 0 && cout > 0 && h >= 3 && w >= 3 && stride >= 1;
}

// BF16 problem of the op entry points: majorness from the unit stride of each operand.
bool bf16_problem(int M, int N, int K, const void* A, int64_t sa_m, int64_t sa_k, const void* B, int64_t sb_n,
                  int64_t sb_k, void* C, int64_t ldc, const void* bias, int accumulate, TcGemm* g) {
    g->M = M; g->N = N; g->K = K; g->n_pairs = 1;
    if (sa_k == 1) g->a[0] = TcOperand{(const __nv_bfloat16*)A, sa_m, false};
    else if (sa_m == 1) g->a[0] = TcOperand{(const __nv_bfloat16*)A, sa_k, true};
    else return false;
    if (sb_k == 1) g->b[0] = TcOperand{(const __nv_bfloat16*)B, sb_n, false};
    else if (sb_n == 1) g->b[0] = TcOperand{(const __nv_bfloat16*)B, sb_k, true};
    else return false;
    g->bias = (const float*)bias;
    g->c = (float*)C; g->ldc = ldc;
    g->accumulate = accumulate;
    return true;
}

}  // namespace

extern "C" {

int squint_op_gemm(int dtype, int M, int N, int K, const void* A, int64_t sa_m, int64_t sa_k, const void* B,
                   int64_t sb_n, int64_t sb_k, void* C, int64_t ldc, const void* bias, int accumulate,
                   void* stream) {
    if (M < 0 || N < 0 || K < 1 || !A || !B || !C) return SQUINT_EINVAL;
    if (M == 0 || N == 0) return SQUINT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SQUINT_DT_F32 || dtype == SQUINT_DT_F64) {
        GemmProblem p{};
        p.M = M; p.N = N; p.K = K;
        p.A = A; p.sa_m = sa_m; p.sa_k = sa_k;
        p.B = B; p.sb_n = sb_n; p.sb_k = sb_k;
        p.C = C; p.sc_m = ldc; p.sc_n = 1;
        p.bias = bias; p.accumulate = accumulate; p.n_sum = 1;
        GemmLayout lay = kKK;
        if (sa_k == 1 && sb_k != 1) lay = kKN;
        else if (sa_k != 1 && sb_k != 1) lay = kMN;
        if (dtype == SQUINT_DT_F32) launch_gemm<float>(&p, 1, lay, s);
        else launch_gemm<double>(&p, 1, lay, s);
        return launch_status();
    }
    if (dtype != SQUINT_DT_BF16) return SQUINT_EINVAL;
    TcGemm g{};
    if (!bf16_problem(M, N, K, A, sa_m, sa_k, B, sb_n, sb_k, C, ldc, bias, accumulate, &g)) return SQUINT_EINVAL;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    if (launch_tc_gemm(&g, 1, err, s) != 0) return SQUINT_EINVAL;
    return launch_status();
}

int squint_op_gemm_layernorm(int M, int N, int K, const void* A, int64_t lda, const void* B, int64_t ldb,
                             const float* bias, const float* g, const float* beta, float eps, int relu, float* pre,
                             float* post, void* post_bf, float* mean, float* rstd, void* stream) {
    if (M < 0 || N < 1 || K < 1 || !A || !B || !g || !beta || !pre || !post || !mean || !rstd) return SQUINT_EINVAL;
    if (M == 0) return SQUINT_OK;
    tc_prepare();
    if (N > 128 * tc_max_cluster()) {
        g_last_error = "GEMM + LayerNorm: N above 128 x the largest GEMM cluster";
        return SQUINT_EINVAL;
    }
    TcGemm gm{};
    if (!bf16_problem(M, N, K, A, lda, 1, B, ldb, 1, pre, N, bias, 0, &gm)) return SQUINT_EINVAL;
    gm.ln_g = g; gm.ln_beta = beta; gm.ln_post = post; gm.ln_posth = (__nv_bfloat16*)post_bf;
    gm.ln_mean = mean; gm.ln_rstd = rstd; gm.ln_eps = eps; gm.ln_relu = relu;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    if (launch_tc_gemm(&gm, 1, err, (cudaStream_t)stream) != 0) return SQUINT_EINVAL;
    return launch_status();
}

int squint_op_mlp_bf16(int M, int kin, int nh, int H, int nout, const void* x, int64_t ldx, const void* const* w,
                       const int64_t* ldw, const float* const* bias, const float* const* g,
                       const float* const* beta, float eps, float* out, int64_t ldo, float* const* pre,
                       float* const* post, void* const* post_bf, float* const* mean, float* const* rstd, int cluster,
                       void* stream) {
    if (M < 0 || kin < 1 || nh < 1 || nh > kMlpMaxHidden || H < 1 || nout < 1 || !x || !w || !ldw || !bias || !g ||
        !beta || !out || ldo < nout || ldx < kin || (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8))
        return SQUINT_EINVAL;
    if (!mlp_tc_supported(nh, H, nout, kin) || (cluster && !mlp_tc_cluster(H, nout, cluster))) {
        g_last_error = "fused MLP: shape outside the kernel's range (or cluster size not possible for it)";
        return SQUINT_EINVAL;
    }
    if (M == 0) return SQUINT_OK;
    MlpTcProblem p;
    std::memset(&p, 0, sizeof(p));
    p.M = M; p.x = (const __nv_bfloat16*)x; p.ldx = ldx; p.kin = kin;
    for (int l = 0; l <= nh; ++l) {
        if (!w[l] || !bias[l]) return SQUINT_EINVAL;
        p.w[l] = (const __nv_bfloat16*)w[l]; p.ldw[l] = ldw[l]; p.bias[l] = bias[l];
        if (l == nh) break;
        if (!g[l] || !beta[l]) return SQUINT_EINVAL;
        p.g[l] = g[l]; p.beta[l] = beta[l];
        p.save[l] = MlpTcSave{pre ? pre[l] : nullptr, post ? post[l] : nullptr,
                              post_bf ? (__nv_bfloat16*)post_bf[l] : nullptr, mean ? mean[l] : nullptr,
                              rstd ? rstd[l] : nullptr};
    }
    p.out = out; p.ldo = ldo;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    const int rc = launch_mlp_tc(&p, 1, nh, H, nout, eps, err, nullptr, (cudaStream_t)stream, cluster);
    if (rc != 0) {
        g_last_error = "fused MLP: an operand cannot be described by a tensor map (alignment, extents)";
        return SQUINT_EINVAL;
    }
    return launch_status();
}

int squint_op_mlp_bwd_bf16(int M, int kin, int nh, int H, int nout, const void* dout, int64_t ld_dout,
                           const void* const* w, const int64_t* ldw, const float* const* g,
                           const float* const* beta, const float* const* pre, const float* const* post,
                           const float* const* mean, const float* const* rstd, void* const* dpre_bf,
                           float* const* colpart, int c0, int ncols, float* dx, int64_t lddx, void* stream) {
    if (M < 0 || nh < 1 || nh > kMlpMaxHidden || !dout || !w || !ldw || !g || !pre || (!post && !beta) || !mean || !rstd ||
        (ncols > 0 && !dx) || lddx < ncols || (ncols == 0 && (!dpre_bf || !dpre_bf[0])))
        return SQUINT_EINVAL;
    if (!mlp_bwd_tc_supported(nh, H, nout, kin, c0, ncols)) {
        g_last_error = "fused MLP backward: shape outside the kernel's range";
        return SQUINT_EINVAL;
    }
    if (M == 0) return SQUINT_OK;
    MlpTcBwdProblem p;
    std::memset(&p, 0, sizeof(p));
    p.M = M; p.dout = (const __nv_bfloat16*)dout; p.ld_dout = ld_dout;
    for (int l = 0; l <= nh; ++l) {
        p.w[l] = (const __nv_bfloat16*)w[l]; p.ldw[l] = ldw[l];
        if (l == nh) break;
        p.g[l] = g[l]; p.beta[l] = beta ? beta[l] : nullptr; p.pre[l] = pre[l]; p.post[l] = post ? post[l] : nullptr;
        p.mean[l] = mean[l]; p.rstd[l] = rstd[l];
        p.dpre_bf[l] = dpre_bf ? (__nv_bfloat16*)dpre_bf[l] : nullptr;
        p.colpart[l] = colpart ? colpart[l] : nullptr;
    }
    p.dx = dx; p.lddx = lddx;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    if (launch_mlp_bwd_tc(&p, 1, nh, H, nout, kin, c0, ncols, err, nullptr, (cudaStream_t)stream) != 0) {
        g_last_error = "fused MLP backward: an operand cannot be described by a tensor map (alignment, extents)";
        return SQUINT_EINVAL;
    }
    return launch_status();
}

int squint_op_cast_bf16(int rows, int cols, const float* src, int64_t ld_src, void* dst, int64_t ld_dst,
                        void* stream) {
    if (rows < 0 || cols < 1 || !src || !dst || ld_src < cols || ld_dst < cols) return SQUINT_EINVAL;
    if (rows == 0) return SQUINT_OK;
    CastItem it{src, ld_src, rows, cols, (__nv_bfloat16*)dst, ld_dst};
    launch_cast_rows(&it, 1, (cudaStream_t)stream);
    return launch_status();
}

static int64_t pad16(int64_t n) { return (n + 15) / 16 * 16; }

size_t squint_op_gemm_fp8_workspace(int M, int N, int K) {
    if (M < 0 || N < 0 || K < 1) return 0;
    return (size_t)quant_workspace() * 4 + 64 + (size_t)(M + N) * pad16(K) + 64;
}

int squint_op_gemm_fp8(int M, int N, int K, const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                       int64_t ldc, const float* bias, void* work, size_t work_bytes, void* stream) {
    if (M < 0 || N < 0 || K < 1 || !A || !B || !C || !work || lda < K || ldb < K) return SQUINT_EINVAL;
    if (work_bytes < squint_op_gemm_fp8_workspace(M, N, K) || (reinterpret_cast<uintptr_t>(work) & 15)) {
        g_last_error = "FP8 GEMM: workspace smaller than squint_op_gemm_fp8_workspace() or not 16-byte aligned";
        return SQUINT_EINVAL;
    }
    if (M == 0 || N == 0) return SQUINT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = static_cast<char*>(work);
    float* part = reinterpret_cast<float*>(w);
    float* scales = reinterpret_cast<float*>(w + quant_workspace() * 4);
    uint8_t* a8 = reinterpret_cast<uint8_t*>(w + quant_workspace() * 4 + 64);
    uint8_t* b8 = a8 + (size_t)M * pad16(K);
    QuantItem q[2];
    q[0] = QuantItem{(const __nv_bfloat16*)A, lda, M, K, a8, pad16(K), scales};
    q[1] = QuantItem{(const __nv_bfloat16*)B, ldb, N, K, b8, pad16(K), scales + 1};
    launch_quantize_e4m3(q, 2, part, s);
    TcGemm g{};
    g.M = M; g.N = N; g.K = K; g.n_pairs = 1;
    g.a[0] = TcOperand{a8, pad16(K), false};
    g.b[0] = TcOperand{b8, pad16(K), false};
    g.bias = bias; g.c = C; g.ldc = ldc;
    g.fp8 = 1; g.scale_a = scales; g.scale_b = scales + 1;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    if (launch_tc_gemm(&g, 1, err, s) != 0) return SQUINT_EINVAL;
    return launch_status();
}

int64_t squint_op_mx_scale_bytes(int rows, int cols) {
    if (rows < 0 || cols < 0) return -1;
    return mx_scale_bytes(rows, cols);
}

int squint_op_quantize_mxfp8(int rows, int cols, const void* src, int64_t ld, void* dst, int64_t dst_ld, void* sf,
                             void* stream) {
    if (rows < 0 || cols < 1 || ld < cols || dst_ld < cols || (dst_ld % 16) || (rows > 0 && (!src || !dst || !sf)))
        return SQUINT_EINVAL;
    if (rows == 0) return SQUINT_OK;
    QuantItem q{(const __nv_bfloat16*)src, ld, rows, cols, (uint8_t*)dst, dst_ld, nullptr, (uint8_t*)sf};
    launch_quantize_mx(&q, 1, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_gemm_mxfp8(int M, int N, int K, const void* A, int64_t lda, const void* sfa, const void* B, int64_t ldb,
                         const void* sfb, float* C, int64_t ldc, const float* bias, void* stream) {
    if (M < 0 || N < 0 || K < 1 || !A || !B || !C || !sfa || !sfb || lda < K || ldb < K || ldc < N || (lda % 16) ||
        (ldb % 16) || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        return SQUINT_EINVAL;
    if (M == 0 || N == 0) return SQUINT_OK;
    TcGemm g{};
    g.M = M; g.N = N; g.K = K; g.n_pairs = 1;
    g.a[0] = TcOperand{A, lda, false};
    g.b[0] = TcOperand{B, ldb, false};
    g.bias = bias; g.c = C; g.ldc = ldc;
    g.fp8 = 2; g.sf_a = (const uint8_t*)sfa; g.sf_b = (const uint8_t*)sfb;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    if (launch_tc_gemm(&g, 1, err, (cudaStream_t)stream) != 0) return SQUINT_EINVAL;
    return launch_status();
}

int squint_op_squint_store(int n, int C, int H, int W, int f, const void* src, void* ring, int64_t slot0,
                           int64_t n_slots, void* stream) {
    if (n < 0 || C < 1 || f < 1 || H < f || W < f || (H % f) || (W % f) || n_slots < 1 || slot0 < 0 ||
        (n > 0 && (!src || !ring)))
        return SQUINT_EINVAL;
    launch_squint_store((const uint8_t*)src, n, C, H, W, f, (uint8_t*)ring, slot0 % n_slots, n_slots,
                        (cudaStream_t)stream);
    return launch_status();
}

int squint_op_conv3x3_fwd(int dtype, int nimg, int cin, int h, int w, int cout, int stride, const void* x,
                          const void* wt, const void* b, void* y, int relu, void* stream) {
    if (!conv_ok(nimg, cin, h, w, cout, stride) || !x || !wt || !b || !y) return SQUINT_EINVAL;
    ConvShape sh = conv_shape(nimg, cin, h, w, cout, stride);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SQUINT_DT_F32)
        launch_conv_fwd<float>(sh, (const float*)x, (const float*)wt, (const float*)b, (float*)y, relu != 0, s);
    else if (dtype == SQUINT_DT_F64)
        launch_conv_fwd<double>(sh, (const double*)x, (const double*)wt, (const double*)b, (double*)y, relu != 0, s);
    else
        return SQUINT_EINVAL;
    return launch_status();
}

size_t squint_op_conv3x3_workspace(int dtype, int nimg, int cin, int h, int w, int cout, int stride) {
    if (!conv_ok(nimg, cin, h, w, cout, stride)) return 0;
    const size_t el = dtype == SQUINT_DT_F64 ? 8 : 4;
    return el * (size_t)conv_wgrad_workspace(conv_shape(nimg, cin, h, w, cout, stride));
}

int squint_op_conv3x3_bwd(int dtype, int nimg, int cin, int h, int w, int cout, int stride, const void* x,
                          const void* wt, const void* dy, void* dx, const void* dx_mask, void* dw, void* db,
                          void* workspace, size_t workspace_bytes, void* stream) {
    if (!conv_ok(nimg, cin, h, w, cout, stride) || !x || !wt || !dy || !dw || !db) return SQUINT_EINVAL;
    if (workspace_bytes < squint_op_conv3x3_workspace(dtype, nimg, cin, h, w, cout, stride) || !workspace)
        return SQUINT_EINVAL;
    ConvShape sh = conv_shape(nimg, cin, h, w, cout, stride);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SQUINT_DT_F32) {
        launch_conv_wgrad<float>(sh, (const float*)dy, (const float*)x, (float*)dw, (float*)db, (float*)workspace, s);
        if (dx) launch_conv_dgrad<float>(sh, (const float*)dy, (const float*)wt, (float*)dx, (const float*)dx_mask, s);
    } else if (dtype == SQUINT_DT_F64) {
        launch_conv_wgrad<double>(sh, (const double*)dy, (const double*)x, (double*)dw, (double*)db,
                                  (double*)workspace, s);
        if (dx)
            launch_conv_dgrad<double>(sh, (const double*)dy, (const double*)wt, (double*)dx, (const double*)dx_mask, s);
    } else {
        return SQUINT_EINVAL;
    }
    return launch_status();
}

int squint_op_to_phwc(int nimg, int H, int W, const float* src, void* dst, void* stream) {
    if (nimg < 0 || H < 1 || W < 1 || !src || !dst) return SQUINT_EINVAL;
    launch_to_phwc(src, (int64_t)32 * H * W, nimg, H, W, (__nv_bfloat16*)dst, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_from_phwc(int nimg, int H, int W, const void* src, float* dst, void* stream) {
    if (nimg < 0 || H < 1 || W < 1 || !src || !dst) return SQUINT_EINVAL;
    launch_from_phwc((const __nv_bfloat16*)src, nimg, H, W, dst, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_conv32_layouts(const float* w, void* fwd_layout, void* dgrad_layout, void* stream) {
    if (!w || !fwd_layout || !dgrad_layout) return SQUINT_EINVAL;
    launch_conv_weight_cast(w, (__nv_bfloat16*)fwd_layout, (__nv_bfloat16*)dgrad_layout, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_conv32(int mode, int nimg, int H, int W, const void* in, const void* w_layout, const float* bias,
                     int relu, const void* mask, void* out_phwc, float* out_nchw, void* stream) {
    if ((mode != 0 && mode != 1) || nimg < 0 || !in || !w_layout || (!out_phwc && !out_nchw)) return SQUINT_EINVAL;
    if (mode == 0 && (H < 3 || W < 3 || !bias)) return SQUINT_EINVAL;
    if (mode == 1 && (H < 1 || W < 1)) return SQUINT_EINVAL;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    ConvTc c{};
    c.in = (const __nv_bfloat16*)in;
    c.nimg = nimg;
    c.Wp = W + 4;
    c.in_rows = (H + 4) * (W + 4);
    c.out_h = mode == 0 ? H - 2 : H + 2;
    c.out_w = mode == 0 ? W - 2 : W + 2;
    c.off0 = mode == 0 ? 2 * c.Wp + 2 : 0;
    c.w = (const __nv_bfloat16*)w_layout;
    c.bias = mode == 0 ? bias : nullptr;
    c.relu = mode == 0 ? relu : 0;
    c.mask = (const __nv_bfloat16*)mask;
    c.out_phwc = (__nv_bfloat16*)out_phwc;
    c.out_chw = out_nchw;
    if (launch_conv32_tc(c, err, (cudaStream_t)stream) != 0) return SQUINT_EINVAL;
    return launch_status();
}

int squint_op_conv0_bf16(int nimg, int Cin, int H, int W, int stride, const float* x, const float* w,
                         const float* bias, void* out_phwc, void* stream) {
    if (nimg < 0 || Cin < 1 || Cin > 16 || stride < 1 || H < 3 || W < 3 || !x || !w || !bias || !out_phwc)
        return SQUINT_EINVAL;
    if (reinterpret_cast<uintptr_t>(out_phwc) & 15) return SQUINT_EINVAL;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    const int OH = (H - 3) / stride + 1, OW = (W - 3) / stride + 1;
    ConvShape sh{nimg, Cin, H, W, 32, stride, OH, OW, (int64_t)Cin * H * W, (int64_t)32 * OH * OW};
    if (launch_conv0_tc(sh, x, w, bias, (__nv_bfloat16*)out_phwc, err, (cudaStream_t)stream) != 0) return SQUINT_EINVAL;
    return launch_status();
}

size_t squint_op_wgrad32_workspace(int nimg) { return nimg > 0 ? 4 * (size_t)wgrad32_tc_workspace(nimg) : 0; }

int squint_op_wgrad32(int nimg, int H, int W, const void* x, const void* dy, float* dw, float* db, void* work,
                      size_t work_bytes, void* stream) {
    if (nimg < 1 || H < 3 || W < 3 || !x || !dy || !dw || !db || !work) return SQUINT_EINVAL;
    if (work_bytes < squint_op_wgrad32_workspace(nimg)) return SQUINT_EINVAL;
    int* err = tc_error_flag();
    if (!err) return SQUINT_ECUDA;
    WgradTc c{};
    c.x = (const __nv_bfloat16*)x;
    c.dy = (const __nv_bfloat16*)dy;
    c.nimg = nimg;
    c.Wp = W + 4;
    c.in_rows = (H + 4) * (W + 4);
    c.out_h = H - 2;
    c.out_w = W - 2;
    if (launch_wgrad32_tc(c, (float*)work, dw, db, err, (cudaStream_t)stream) != 0) return SQUINT_EINVAL;
    return launch_status();
}

int squint_op_relu_bwd(int dtype, int64_t n, const void* dy, const void* y, void* dx, void* stream) {
    if (n < 0 || (n > 0 && (!dy || !y || !dx))) return SQUINT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SQUINT_DT_F32) launch_relu_bwd<float>(n, (const float*)dy, (const float*)y, (float*)dx, s);
    else if (dtype == SQUINT_DT_F64) launch_relu_bwd<double>(n, (const double*)dy, (const double*)y, (double*)dx, s);
    else return SQUINT_EINVAL;
    return launch_status();
}

int squint_op_layernorm_fwd(int rows, int n, const float* x, const float* g, const float* b, float eps, int relu,
                            float* y, float* mean, float* rstd, void* stream) {
    if (rows < 0 || n < 1 || !x || !g || !b || !y || !mean || !rstd) return SQUINT_EINVAL;
    LnProblem p{};
    p.rows = rows; p.n = n; p.pre = x; p.ld_pre = n; p.g = g; p.beta = b;
    p.out = y; p.ld_out = n; p.mean = mean; p.rstd = rstd;
    launch_ln_fwd(&p, 1, relu != 0, eps, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_layernorm_bwd(int rows, int n, const float* dy, const float* y, const float* x, const float* mean,
                            const float* rstd, const float* g, float* dx, float* dg, float* db, void* stream) {
    if (rows < 0 || n < 1 || !dy || !x || !mean || !rstd || !g || !dx) return SQUINT_EINVAL;
    LnBwdProblem p{};
    p.rows = rows; p.n = n;
    p.dout = dy; p.ld_dout = n; p.out = y; p.ld_out = n; p.pre = x; p.ld_pre = n;
    p.mean = mean; p.rstd = rstd; p.g = g; p.dpre = dx; p.ld_dpre = n;
    p.dg = dg; p.dbeta = db;
    cudaStream_t s = (cudaStream_t)stream;
    float* work = nullptr;
    const int64_t wn = ln_bwd_workspace(&p, 1);
    if ((dg || db) && cudaMallocAsync((void**)&work, (size_t)wn * sizeof(float), s) != cudaSuccess) return SQUINT_ECUDA;
    if (work) cudaMemsetAsync(work, 0, kLnTickets * sizeof(float), s);
    ln_prepare();
    launch_ln_bwd(&p, 1, work, s);
    if (work) cudaFreeAsync(work, s);
    return launch_status();
}

int squint_op_categorical_ce(int rows, int K, const float* logits, const float* m, float v_min, float v_max,
                             float scale, float* dlogits, float* row_loss, float* row_q, void* stream) {
    if (rows < 0 || K < 2 || K > 256 || !logits || !m || !dlogits || !row_loss || !row_q) return SQUINT_EINVAL;
    if (rows == 0) return SQUINT_OK;
    CeArgs a{};
    a.B = rows; a.K = K; a.E = 1; a.logits = logits; a.m = m; a.v_min = v_min; a.v_max = v_max;
    a.scale = scale; a.dlogits = dlogits; a.row_loss = row_loss; a.row_q = row_q;
    launch_ce(a, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_c51_project(int rows, int K, int E, const float* logits, const float* r, const float* d,
                          const float* logp, float alpha, float gamma, float v_min, float v_max, float* m,
                          void* stream) {
    if (rows < 0 || K < 2 || K > 256 || E < 1 || !logits || !r || !d || !logp || !m || !(v_max > v_min))
        return SQUINT_EINVAL;
    if (rows == 0) return SQUINT_OK;
    C51TargetArgs a{};
    a.B = rows; a.K = K; a.E = E; a.logits_bar = logits; a.r = r; a.d = d; a.logp_next = logp;
    a.log_alpha = nullptr; a.alpha_value = alpha; a.gamma = gamma; a.v_min = v_min; a.v_max = v_max; a.m = m;
    launch_c51_target(a, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_tanh_gaussian_fwd(int rows, int A, const float* out, const float* eps, float lo, float hi, float* a,
                                float* logp, void* stream) {
    if (rows < 0 || A < 1 || !out || !eps || !a || !logp) return SQUINT_EINVAL;
    if (rows == 0) return SQUINT_OK;
    // rows are treated as the "actor" half (rows >= B), so actions land in a_dst1 with ld A
    ActorHeadArgs h{};
    h.rows = rows; h.B = 0; h.A = A; h.out = out; h.ld_out = 2 * A; h.lo = lo; h.hi = hi;
    h.a_dst1 = a; h.ld1 = A; h.a_dst0 = a; h.ld0 = A;
    h.logp = logp;
    h.eps = nullptr;
    h.eps_in = eps;
    launch_actor_head(h, (cudaStream_t)stream);
    return launch_status();
}

int squint_op_tanh_gaussian_bwd(int rows, int A, const float* out, const float* eps, const float* da,
                                const float* dlogp, float lo, float hi, float* dout, void* stream) {
    if (rows < 0 || A < 1 || !out || !eps || !da || !dlogp || !dout) return SQUINT_EINVAL;
    if (rows == 0) return SQUINT_OK;
    ActorHeadBwdArgs h{};
    h.B = rows; h.A = A; h.out = out; h.ld_out = 2 * A; h.eps = eps; h.da = da;
    h.lo = lo; h.hi = hi; h.dout = dout; h.dlogp_rows = dlogp;
    launch_actor_head_bwd(h, (cudaStream_t)stream);
    return launch_status();
}

}  // extern "C"
