"""torch.autograd.Function wrappers over the library's hand-written layer kernels.

Each forward and each backward is one or more calls into include/squint_ops.h;
the wrappers only allocate outputs and pass pointers:

  Linear        y = x W^T + b                 (Sec. III: critic and actor MLP layers)
  Conv3x3       y = [ReLU](conv3x3(x) + b)    (Sec. III: the shared CNN encoder)
  LayerNorm     y = [ReLU](LN(x) g + beta)    (Sec. IV "Normalization")
  CategoricalCE mean_r -sum_j m[r,j] log softmax(l[r])_j   (C51 critic loss, Sec. IV)
  TanhGaussian  (a, log pi) of the squashed Gaussian policy, noise fixed (Eq. 1)

Linear and Conv3x3 take FP32 or FP64 CUDA tensors and run the CUDA-core kernels of
the FP32 learner; the others are FP32.  The BF16 learner's tensor-core kernels have
their own wrappers, with FP32 tensors in and out and every operand rounded to BF16
by the library's cast kernel (FP32 accumulation):

  LinearBF16    forward, data and weight gradient on the tcgen05 GEMM
  Conv32BF16    32 -> 32 channel, stride-1 convolution: forward and data gradient on
                the tcgen05 convolution kernel, weight gradient on its tcgen05
                weight-gradient kernel (padded-HWC BF16 activations)
  MlpHeadBF16   a LayerNorm MLP head: forward by the fused head kernel, backward by
                the hand-written LayerNorm backward and tcgen05 GEMM kernels

The C51 target is not differentiated (the target is held fixed), so it has no
wrapper: call ops.c51_project.
"""
import torch

from . import ops


def _ones_row(n, like):
    return torch.ones(1, n, dtype=like.dtype, device=like.device)


def _col_sum(t):
    """Sum over rows of a 2-D tensor, as a 1 x rows by rows x cols product on the GEMM kernel."""
    rows, cols = t.shape
    return ops.gemm(_ones_row(rows, t), t.t(), M=1, N=cols, K=rows).reshape(cols)


class Linear(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b):
        ctx.save_for_backward(x, w)
        return ops.gemm(x, w, bias=b)

    @staticmethod
    def backward(ctx, dy):
        x, w = ctx.saved_tensors
        dy = dy.contiguous()
        rows, n_out = dy.shape
        n_in = x.shape[1]
        dx = ops.gemm(dy, w.t(), M=rows, N=n_in, K=n_out) if ctx.needs_input_grad[0] else None
        dw = ops.gemm(dy.t(), x.t(), M=n_out, N=n_in, K=rows) if ctx.needs_input_grad[1] else None
        db = _col_sum(dy) if ctx.needs_input_grad[2] else None
        return dx, dw, db


class Conv3x3(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, w, b, stride, relu):
        x = x.contiguous()
        y = ops.conv3x3_fwd(x, w.contiguous(), b, stride, relu)
        ctx.stride, ctx.relu = stride, relu
        ctx.save_for_backward(x, w, y)
        return y

    @staticmethod
    def backward(ctx, dy):
        x, w, y = ctx.saved_tensors
        dy = dy.contiguous()
        if ctx.relu:
            dy = ops.relu_bwd(dy, y)
        dx, dw, db = ops.conv3x3_bwd(x, w.contiguous(), dy, ctx.stride, need_dx=ctx.needs_input_grad[0])
        return dx, dw, db, None, None


class LayerNorm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, g, beta, relu, eps=1e-5):
        x = x.contiguous()
        y, mean, rstd = ops.layernorm_fwd(x, g, beta, eps, relu)
        ctx.relu = relu
        ctx.save_for_backward(x, g, y, mean, rstd)
        return y

    @staticmethod
    def backward(ctx, dy):
        x, g, y, mean, rstd = ctx.saved_tensors
        dx, dg, db = ops.layernorm_bwd(dy.contiguous(), y, x, mean, rstd, g, ctx.relu)
        return dx, dg, db, None, None


class CategoricalCE(torch.autograd.Function):
    """Mean over rows of the cross entropy of softmax(logits) against the fixed target m."""

    @staticmethod
    def forward(ctx, logits, m, v_min, v_max):
        logits, m = logits.contiguous(), m.contiguous()
        rows = logits.shape[0]
        loss_rows, _, _ = ops.categorical_ce(logits, m, v_min, v_max, 1.0 / rows)
        ctx.v = (v_min, v_max)
        ctx.save_for_backward(logits, m)
        inv = torch.full((1, rows), 1.0 / rows, dtype=loss_rows.dtype, device=loss_rows.device)
        return ops.gemm(inv, loss_rows.reshape(1, rows), M=1, N=1, K=rows).reshape(())

    @staticmethod
    def backward(ctx, dloss):
        logits, m = ctx.saved_tensors
        scale = float(dloss) / logits.shape[0]
        _, dlogits, _ = ops.categorical_ce(logits, m, ctx.v[0], ctx.v[1], scale)
        return dlogits, None, None, None


class TanhGaussian(torch.autograd.Function):
    """out = [mu | raw log-std] rows -> (a, log pi) with the noise eps held fixed."""

    @staticmethod
    def forward(ctx, out, eps, lo=-5.0, hi=2.0):
        out, eps = out.contiguous(), eps.contiguous()
        a, logp = ops.tanh_gaussian_fwd(out, eps, lo, hi)
        ctx.lim = (lo, hi)
        ctx.save_for_backward(out, eps)
        return a, logp

    @staticmethod
    def backward(ctx, da, dlogp):
        out, eps = ctx.saved_tensors
        if da is None:
            da = torch.zeros_like(eps)
        if dlogp is None:
            dlogp = torch.zeros(eps.shape[0], dtype=eps.dtype, device=eps.device)
        dout = ops.tanh_gaussian_bwd(out, eps, da.contiguous(), dlogp.contiguous(), *ctx.lim)
        return dout, None, None, None


class LinearBF16(torch.autograd.Function):
    """y = bf16(x) bf16(W)^T + b on the tcgen05 GEMM; the backward rounds dy to BF16 and runs
    dx = dy W and dW = dy^T x on the same kernel (MN-major operands), db as a column sum."""

    @staticmethod
    def forward(ctx, x, w, b):
        xh, wh = ops.cast_bf16(x), ops.cast_bf16(w)
        ctx.save_for_backward(xh, wh)
        return ops.gemm(xh, wh, bias=b)

    @staticmethod
    def backward(ctx, dy):
        xh, wh = ctx.saved_tensors
        dy = dy.contiguous()
        dyh = ops.cast_bf16(dy)
        rows, n_out = dy.shape
        n_in = xh.shape[1]
        dx = ops.gemm(dyh, wh.t(), M=rows, N=n_in, K=n_out) if ctx.needs_input_grad[0] else None
        dw = ops.gemm(dyh.t(), xh.t(), M=n_out, N=n_in, K=rows) if ctx.needs_input_grad[1] else None
        db = _col_sum(dy) if ctx.needs_input_grad[2] else None
        return dx, dw, db


class Conv32BF16(torch.autograd.Function):
    """y = [ReLU](conv3x3(bf16(x), bf16(W)) + b), 32 -> 32 channels, stride 1, valid, on the
    tensor-core convolution; x FP32 [n, 32, H, W].  The backward masks dy by the ReLU (FP32),
    rounds it to BF16 and runs the data gradient and the weight gradient kernels."""

    @staticmethod
    def forward(ctx, x, w, b, relu=True):
        n, c, H, W = x.shape
        xp = ops.to_phwc(x.contiguous())
        wf, wb = ops.conv32_layouts(w)
        _, y = ops.conv32_fwd(xp, H, W, wf, b, relu)
        ctx.relu, ctx.hw = relu, (H, W)
        ctx.save_for_backward(xp, wb, y)
        return y

    @staticmethod
    def backward(ctx, dy):
        xp, wb, y = ctx.saved_tensors
        H, W = ctx.hw
        dy = dy.contiguous()
        if ctx.relu:
            dy = ops.relu_bwd(dy, y)
        dyp = ops.to_phwc(dy)
        dx = ops.conv32_dgrad(dyp, H - 2, W - 2, wb)[1] if ctx.needs_input_grad[0] else None
        dw, db = ops.wgrad32(xp, dyp, H, W)
        return dx, dw, db, None


class MlpHeadBF16(torch.autograd.Function):
    """A LayerNorm MLP head (hidden layers Linear -> LayerNorm -> ReLU, plain Linear output),
    params = (w_0, b_0, g_0, beta_0, ..., w_nh, b_nh) in FP32.  Forward: the fused head
    kernel on BF16 operands.  Backward: per layer, from the output down, the weight
    gradient bf16(dy)^T h and the data gradient bf16(dy) W on the tcgen05 GEMM, the
    LayerNorm (+ReLU) backward kernel, bias gradients as column sums: the kernels the BF16
    learner's backward runs."""

    @staticmethod
    def forward(ctx, x, eps, *params):
        nh = (len(params) - 2) // 4
        ws = [ops.cast_bf16(params[4 * l]) for l in range(nh)] + [ops.cast_bf16(params[4 * nh])]
        bs = [params[4 * l + 1] for l in range(nh)] + [params[4 * nh + 1]]
        gs = [params[4 * l + 2] for l in range(nh)]
        betas = [params[4 * l + 3] for l in range(nh)]
        xh = ops.cast_bf16(x)
        out, saved = ops.mlp_bf16(xh, ws, bs, gs, betas, eps=eps)
        ctx.nh = nh
        flat = [t for sv in saved for t in sv]
        ctx.save_for_backward(xh, *ws, *gs, *flat)
        return out

    @staticmethod
    def backward(ctx, dout):
        nh = ctx.nh
        st = ctx.saved_tensors
        xh, ws, gs = st[0], st[1:nh + 2], st[nh + 2:2 * nh + 2]
        saved = [st[2 * nh + 2 + 5 * l: 2 * nh + 7 + 5 * l] for l in range(nh)]   # pre, post, post_bf, mean, rstd
        grads = [None] * (4 * nh + 2)
        dy = dout.contiguous()
        for l in range(nh, -1, -1):
            h = xh if l == 0 else saved[l - 1][2]                       # the layer's BF16 input
            dyh = ops.cast_bf16(dy)
            rows, n_out = dy.shape
            n_in = h.shape[1]
            gi = 4 * l
            grads[gi] = ops.gemm(dyh.t(), h.t(), M=n_out, N=n_in, K=rows)
            grads[gi + 1] = _col_sum(dy)
            dh = ops.gemm(dyh, ws[l].t(), M=rows, N=n_in, K=n_out)
            if l == 0:
                dx = dh
                break
            pre, post, _, mean, rstd = saved[l - 1]
            dy, dg, dbeta = ops.layernorm_bwd(dh, post, pre, mean, rstd, gs[l - 1], relu=True)
            grads[4 * (l - 1) + 2], grads[4 * (l - 1) + 3] = dg, dbeta
        return (dx, None, *grads)


linear = Linear.apply
conv3x3 = Conv3x3.apply
layer_norm = LayerNorm.apply
categorical_ce = CategoricalCE.apply
tanh_gaussian = TanhGaussian.apply
linear_bf16 = LinearBF16.apply
conv32_bf16 = Conv32BF16.apply


def mlp_head_bf16(x, params, eps=1e-5):
    """MlpHeadBF16 over x FP32 [rows, kin] and the FP32 parameter list (w, b, g, beta per
    hidden layer, then w, b of the output layer)."""
    return MlpHeadBF16.apply(x, eps, *params)
