"""torch.autograd.Function wrappers over the library's hand-written layer kernels.

Each forward and each backward is one or more calls into include/squint_ops.h;
the wrappers only allocate outputs and pass pointers, so autograd (and
torch.autograd.gradcheck) exercises exactly the kernels the learner runs:

  Linear        y = x W^T + b                 (Sec. III: critic and actor MLP layers)
  Conv3x3       y = [ReLU](conv3x3(x) + b)    (Sec. III: the shared CNN encoder)
  LayerNorm     y = [ReLU](LN(x) g + beta)    (Sec. IV "Normalization")
  CategoricalCE mean_r -sum_j m[r,j] log softmax(l[r])_j   (C51 critic loss, Sec. IV)
  TanhGaussian  (a, log pi) of the squashed Gaussian policy, noise fixed (Eq. 1)

Linear and Conv3x3 take FP32 or FP64 CUDA tensors (CUDA-core kernels); the
others are FP32.  The C51 target is not differentiated (the target is held
fixed), so it has no wrapper: call ops.c51_project.
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


linear = Linear.apply
conv3x3 = Conv3x3.apply
layer_norm = LayerNorm.apply
categorical_ce = CategoricalCE.apply
tanh_gaussian = TanhGaussian.apply
