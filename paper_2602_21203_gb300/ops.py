"""Layer operations of include/squint_ops.h on torch CUDA tensors (marshalling only).

Each call launches the library's kernel on the current torch stream.  There is
no fallback: tensors must be CUDA tensors of the stated dtype and layout.
"""
import ctypes

import torch

from . import lib as _lib

DT_F32, DT_F64, DT_BF16 = 0, 1, 2
_DT = {torch.float32: DT_F32, torch.float64: DT_F64, torch.bfloat16: DT_BF16}


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(rc, what):
    if rc != 0:
        raise _lib.SquintError(rc, what)


def _need(t, dtype, name):
    if not t.is_cuda or t.dtype != dtype:
        raise TypeError(f"{name}: expected a CUDA {dtype} tensor, got {t.dtype} on {t.device}")


def gemm(A, B, bias=None, out=None, accumulate=False, M=None, N=None, K=None):
    """out[m, n] (+)= sum_k A(m, k) B(n, k) + bias; A, B 2-D views given as (rows = m|n, cols = k) with any strides.

    For BF16 operands each of A, B must have one unit stride; out and bias are FP32.
    """
    M = A.shape[0] if M is None else M
    K = A.shape[1] if K is None else K
    N = B.shape[0] if N is None else N
    dt = _DT[A.dtype]
    odt = torch.float32 if dt == DT_BF16 else A.dtype
    if out is None:
        out = torch.zeros(M, N, device=A.device, dtype=odt)
    _need(out, odt, "out")
    if bias is not None:
        _need(bias, odt, "bias")
    _chk(_lib.load().squint_op_gemm(dt, M, N, K, _p(A), A.stride(0), A.stride(1), _p(B), B.stride(0), B.stride(1),
                                    _p(out), out.stride(0), _p(bias), int(accumulate), _s()), "squint_op_gemm")
    return out


def squint_store(frames, ring_obs, slot0, f):
    """Squint at insert: uint8 frames [n, C, H, W] -> rounded f x f means into ring_obs
    [n_slots, C, H/f, W/f] at slots slot0, slot0 + 1, ... (mod n_slots)."""
    _need(frames, torch.uint8, "frames")
    _need(ring_obs, torch.uint8, "ring_obs")
    n, c, h, w = frames.shape
    frames = frames.contiguous()
    _chk(_lib.load().squint_op_squint_store(n, c, h, w, int(f), _p(frames), _p(ring_obs), int(slot0),
                                            ring_obs.shape[0], _s()), "squint_op_squint_store")


def gemm_layernorm(A, B, bias, g, beta, eps=1e-5, relu=True):
    """BF16 A [M, K] B [N, K]^T + bias, then LayerNorm (+ReLU) per row in the same kernel.
    Returns (pre, post, post_bf16, mean, rstd)."""
    _need(A, torch.bfloat16, "A")
    _need(B, torch.bfloat16, "B")
    M, K = A.shape
    N = B.shape[0]
    dev = A.device
    pre = torch.empty(M, N, device=dev)
    post = torch.empty(M, N, device=dev)
    post_bf = torch.empty(M, N, device=dev, dtype=torch.bfloat16)
    mean = torch.empty(M, device=dev)
    rstd = torch.empty(M, device=dev)
    _chk(_lib.load().squint_op_gemm_layernorm(M, N, K, _p(A), A.stride(0), _p(B), B.stride(0), _p(bias), _p(g),
                                              _p(beta), float(eps), int(relu), _p(pre), _p(post), _p(post_bf),
                                              _p(mean), _p(rstd), _s()), "squint_op_gemm_layernorm")
    return pre, post, post_bf, mean, rstd


def cast_bf16(x):
    """FP32 [rows, cols] -> BF16 (round to nearest even) in a buffer whose row stride is
    cols rounded up to 8 (the tensor-core operand alignment); returns the [rows, cols] view."""
    _need(x, torch.float32, "x")
    rows, cols = x.shape
    ld = (cols + 7) // 8 * 8
    buf = torch.empty(rows, ld, dtype=torch.bfloat16, device=x.device)
    if x.stride(1) != 1:
        x = x.contiguous()
    _chk(_lib.load().squint_op_cast_bf16(rows, cols, _p(x), x.stride(0), _p(buf), ld, _s()), "squint_op_cast_bf16")
    return buf[:, :cols]


def mlp_bf16(x, ws, biases, gs, betas, eps=1e-5, save=True, cluster=0):
    """A LayerNorm MLP head in one launch: hidden layers Linear -> LayerNorm -> ReLU
    (weights ws[l] BF16 [out, in], biases FP32), then a plain Linear output layer.
    x BF16 [M, kin].  Returns (out [M, nout], saved) with saved = per hidden layer
    (pre, post, post_bf16, mean, rstd) if save, else None."""
    _need(x, torch.bfloat16, "x")
    nh = len(ws) - 1
    M, kin = x.shape
    H, nout = ws[0].shape[0], ws[-1].shape[0]
    dev = x.device
    for w in ws:
        _need(w, torch.bfloat16, "w")
    out = torch.empty(M, nout, device=dev)

    def arr(ctype, vals):
        return (ctype * len(vals))(*vals)

    P = ctypes.c_void_p
    saved = None
    pre = post = pbf = mean = rstd = None
    if save:
        saved = [(torch.empty(M, H, device=dev), torch.empty(M, H, device=dev),
                  torch.empty(M, H, device=dev, dtype=torch.bfloat16), torch.empty(M, device=dev),
                  torch.empty(M, device=dev)) for _ in range(nh)]
        pre, post, pbf, mean, rstd = (arr(P, [t[i].data_ptr() for t in saved]) for i in range(5))
    _chk(_lib.load().squint_op_mlp_bf16(M, kin, nh, H, nout, _p(x), x.stride(0), arr(P, [w.data_ptr() for w in ws]),
                                        arr(ctypes.c_int64, [w.stride(0) for w in ws]),
                                        arr(P, [b.data_ptr() for b in biases]), arr(P, [g.data_ptr() for g in gs]),
                                        arr(P, [b.data_ptr() for b in betas]), float(eps), _p(out), out.stride(0),
                                        pre, post, pbf, mean, rstd, int(cluster), _s()), "squint_op_mlp_bf16")
    return out, saved


def mlp_bf16_bwd(dout, ws, gs, saved, kin, c0, ncols, want_dpre=True, want_cols=True, betas=None):
    """The input-gradient chain of a head evaluated by mlp_bf16 (saved = its per-layer
    (pre, post, post_bf16, mean, rstd)): dout BF16 [M, nout], weights as for mlp_bf16.
    With betas (the LayerNorm shifts) the ReLU mask is rebuilt from pre and post is not read.
    Returns (dx [M, ncols] = columns c0 .. c0 + ncols of the input gradient,
    dpre_bf16 per hidden layer or None, colpart per hidden layer [ceil(M/128), 3, H] or None)."""
    _need(dout, torch.bfloat16, "dout")
    nh = len(ws) - 1
    M, nout = dout.shape
    H = ws[0].shape[0]
    dev = dout.device
    dx = torch.empty(M, ncols, device=dev)

    def arr(ctype, vals):
        return (ctype * len(vals))(*vals)

    P = ctypes.c_void_p
    dp = [torch.empty(M, H, device=dev, dtype=torch.bfloat16) for _ in range(nh)] if want_dpre else None
    cp = [torch.empty((M + 127) // 128, 3, H, device=dev) for _ in range(nh)] if want_cols else None
    _chk(_lib.load().squint_op_mlp_bwd_bf16(
        M, kin, nh, H, nout, _p(dout), dout.stride(0), arr(P, [w.data_ptr() for w in ws]),
        arr(ctypes.c_int64, [w.stride(0) for w in ws]), arr(P, [t.data_ptr() for t in gs]),
        arr(P, [t.data_ptr() for t in betas]) if betas is not None else None,
        arr(P, [sv[0].data_ptr() for sv in saved]),
        arr(P, [sv[1].data_ptr() for sv in saved]) if betas is None else None,
        arr(P, [sv[3].data_ptr() for sv in saved]), arr(P, [sv[4].data_ptr() for sv in saved]),
        arr(P, [t.data_ptr() for t in dp]) if dp else None, arr(P, [t.data_ptr() for t in cp]) if cp else None,
        int(c0), int(ncols), _p(dx), dx.stride(0), _s()), "squint_op_mlp_bwd_bf16")
    return dx, dp, cp


def gemm_fp8(A, B, bias=None, out=None):
    """out = scale_A scale_B e4m3(A / scale_A) e4m3(B / scale_B)^T + bias for BF16 A [M, K], B [N, K]
    (row-major, unit column stride); per-tensor scales amax / 448.  Returns (out, (scale_A, scale_B))."""
    _need(A, torch.bfloat16, "A")
    _need(B, torch.bfloat16, "B")
    M, K = A.shape
    N = B.shape[0]
    L = _lib.load()
    work = torch.empty(max(L.squint_op_gemm_fp8_workspace(M, N, K), 16), dtype=torch.uint8, device=A.device)
    if out is None:
        out = torch.empty(M, N, device=A.device, dtype=torch.float32)
    if bias is not None:
        _need(bias, torch.float32, "bias")
    _chk(L.squint_op_gemm_fp8(M, N, K, _p(A), A.stride(0), _p(B), B.stride(0), _p(out), out.stride(0), _p(bias),
                              _p(work), work.numel(), _s()), "squint_op_gemm_fp8")
    scales = work[2048:2056].view(torch.float32)
    return out, (scales[0], scales[1])


def quantize_mxfp8(X):
    """MX-FP8 codes and scale bytes of BF16 X [rows, cols] (row-major): returns (codes uint8
    [rows, ceil16(cols)], sf uint8 [squint_op_mx_scale_bytes(rows, cols)])."""
    _need(X, torch.bfloat16, "X")
    rows, cols = X.shape
    L = _lib.load()
    ld8 = (cols + 15) // 16 * 16
    codes = torch.empty(rows, ld8, dtype=torch.uint8, device=X.device)
    sf = torch.empty(max(L.squint_op_mx_scale_bytes(rows, cols), 16), dtype=torch.uint8, device=X.device)
    _chk(L.squint_op_quantize_mxfp8(rows, cols, _p(X), X.stride(0), _p(codes), codes.stride(0), _p(sf), _s()),
         "squint_op_quantize_mxfp8")
    return codes, sf


def gemm_mxfp8(A8, sfa, B8, sfb, K, bias=None, out=None):
    """out = dequant(A) dequant(B)^T + bias for MX-FP8 operands (codes [M, >=K], [N, >=K] with
    their scale bytes from quantize_mxfp8)."""
    M, N = A8.shape[0], B8.shape[0]
    if out is None:
        out = torch.empty(M, N, device=A8.device, dtype=torch.float32)
    if bias is not None:
        _need(bias, torch.float32, "bias")
    _chk(_lib.load().squint_op_gemm_mxfp8(M, N, K, _p(A8), A8.stride(0), _p(sfa), _p(B8), B8.stride(0), _p(sfb),
                                          _p(out), out.stride(0), _p(bias), _s()), "squint_op_gemm_mxfp8")
    return out


def conv3x3_fwd(x, w, b, stride, relu):
    n, cin, h, wd = x.shape
    cout = w.shape[0]
    oh, ow = (h - 3) // stride + 1, (wd - 3) // stride + 1
    y = torch.empty(n, cout, oh, ow, device=x.device, dtype=x.dtype)
    _chk(_lib.load().squint_op_conv3x3_fwd(_DT[x.dtype], n, cin, h, wd, cout, stride, _p(x), _p(w), _p(b), _p(y),
                                           int(relu), _s()), "squint_op_conv3x3_fwd")
    return y


def conv3x3_bwd(x, w, dy, stride, need_dx=True, dx_mask=None):
    n, cin, h, wd = x.shape
    cout = w.shape[0]
    L = _lib.load()
    dt = _DT[x.dtype]
    ws = L.squint_op_conv3x3_workspace(dt, n, cin, h, wd, cout, stride)
    work = torch.empty(max(ws, 16), dtype=torch.uint8, device=x.device)
    dw = torch.empty_like(w)
    db = torch.empty(cout, device=x.device, dtype=x.dtype)
    dx = torch.empty_like(x) if need_dx else None
    _chk(L.squint_op_conv3x3_bwd(dt, n, cin, h, wd, cout, stride, _p(x), _p(w), _p(dy), _p(dx), _p(dx_mask), _p(dw),
                                 _p(db), _p(work), work.numel(), _s()), "squint_op_conv3x3_bwd")
    return dx, dw, db


def relu_bwd(dy, y, out=None):
    """dy * (y > 0) for F32/F64 tensors of the same shape (out may be dy itself)."""
    _need(y, dy.dtype, "y")
    dy, y = dy.contiguous(), y.contiguous()
    out = torch.empty_like(dy) if out is None else out
    _chk(_lib.load().squint_op_relu_bwd(_DT[dy.dtype], dy.numel(), _p(dy), _p(y), _p(out), _s()), "squint_op_relu_bwd")
    return out


def layernorm_fwd(x, g, b, eps=1e-5, relu=False):
    rows, n = x.shape
    y = torch.empty_like(x)
    mean = torch.empty(rows, device=x.device, dtype=torch.float32)
    rstd = torch.empty_like(mean)
    _chk(_lib.load().squint_op_layernorm_fwd(rows, n, _p(x), _p(g), _p(b), float(eps), int(relu), _p(y), _p(mean),
                                             _p(rstd), _s()), "squint_op_layernorm_fwd")
    return y, mean, rstd


def layernorm_bwd(dy, y, x, mean, rstd, g, relu=False):
    rows, n = x.shape
    dx = torch.empty_like(x)
    dg = torch.empty_like(g)
    db = torch.empty_like(g)
    _chk(_lib.load().squint_op_layernorm_bwd(rows, n, _p(dy), _p(y) if relu else None, _p(x), _p(mean), _p(rstd),
                                             _p(g), _p(dx), _p(dg), _p(db), _s()), "squint_op_layernorm_bwd")
    return dx, dg, db


def categorical_ce(logits, m, v_min, v_max, scale):
    rows, K = logits.shape
    d = torch.empty_like(logits)
    loss = torch.empty(rows, device=logits.device, dtype=torch.float32)
    q = torch.empty_like(loss)
    _chk(_lib.load().squint_op_categorical_ce(rows, K, _p(logits), _p(m), float(v_min), float(v_max), float(scale),
                                              _p(d), _p(loss), _p(q), _s()), "squint_op_categorical_ce")
    return loss, d, q


def c51_project(logits, r, d, logp, alpha, gamma, v_min, v_max):
    E, rows, K = logits.shape
    m = torch.empty(rows, K, device=logits.device, dtype=torch.float32)
    _chk(_lib.load().squint_op_c51_project(rows, K, E, _p(logits), _p(r), _p(d), _p(logp), float(alpha), float(gamma),
                                           float(v_min), float(v_max), _p(m), _s()), "squint_op_c51_project")
    return m


def tanh_gaussian_fwd(out, eps, lo=-5.0, hi=2.0):
    rows, A = eps.shape
    a = torch.empty_like(eps)
    logp = torch.empty(rows, device=out.device, dtype=torch.float32)
    _chk(_lib.load().squint_op_tanh_gaussian_fwd(rows, A, _p(out), _p(eps), float(lo), float(hi), _p(a), _p(logp),
                                                 _s()), "squint_op_tanh_gaussian_fwd")
    return a, logp


def tanh_gaussian_bwd(out, eps, da, dlogp, lo=-5.0, hi=2.0):
    rows, A = eps.shape
    dout = torch.empty_like(out)
    _chk(_lib.load().squint_op_tanh_gaussian_bwd(rows, A, _p(out), _p(eps), _p(da), _p(dlogp), float(lo), float(hi),
                                                 _p(dout), _s()), "squint_op_tanh_gaussian_bwd")
    return dout


# ---------------------------------------------------------------- tensor-core convolutions (32 -> 32, stride 1)
def phwc_empty(nimg, H, W, device="cuda"):
    """A zero-filled padded-HWC BF16 buffer for nimg images of H x W x 32."""
    return torch.zeros(nimg, (H + 4) * (W + 4), 32, dtype=torch.bfloat16, device=device)


def to_phwc(x):
    n, c, H, W = x.shape
    assert c == 32 and x.dtype == torch.float32
    out = phwc_empty(n, H, W, x.device)
    _chk(_lib.load().squint_op_to_phwc(n, H, W, _p(x.contiguous()), _p(out), _s()), "squint_op_to_phwc")
    return out


def from_phwc(t, H, W):
    n = t.shape[0]
    out = torch.empty(n, 32, H, W, device=t.device, dtype=torch.float32)
    _chk(_lib.load().squint_op_from_phwc(n, H, W, _p(t), _p(out), _s()), "squint_op_from_phwc")
    return out


def conv0_bf16(x, w, bias, stride, out=None):
    """The encoder's first layer on tensor cores: x NCHW FP32 [n, Cin, H, W], w [32, Cin, 3, 3],
    bias [32] -> ReLU(conv + bias) as padded-HWC BF16 (interior written; `out` defaults to a
    zero-filled buffer)."""
    n, cin, H, W = x.shape
    OH, OW = (H - 3) // stride + 1, (W - 3) // stride + 1
    if out is None:
        out = phwc_empty(n, OH, OW, x.device)
    _chk(_lib.load().squint_op_conv0_bf16(n, cin, H, W, int(stride), _p(x.contiguous()), _p(w.contiguous()),
                                          _p(bias.contiguous()), _p(out), _s()), "squint_op_conv0_bf16")
    return out


def conv32_layouts(w):
    fwd = torch.empty(9 * 32 * 32, dtype=torch.bfloat16, device=w.device)
    bwd = torch.empty_like(fwd)
    _chk(_lib.load().squint_op_conv32_layouts(_p(w.contiguous()), _p(fwd), _p(bwd), _s()), "squint_op_conv32_layouts")
    return fwd, bwd


def conv32_fwd(x_phwc, H, W, w_fwd, bias, relu=True):
    n = x_phwc.shape[0]
    y = phwc_empty(n, H - 2, W - 2, x_phwc.device)
    y_nchw = torch.empty(n, 32, H - 2, W - 2, device=x_phwc.device)
    _chk(_lib.load().squint_op_conv32(0, n, H, W, _p(x_phwc), _p(w_fwd), _p(bias), int(relu), None, _p(y), _p(y_nchw),
                                      _s()), "squint_op_conv32")
    return y, y_nchw


def conv32_dgrad(dy_phwc, H, W, w_bwd, mask_phwc=None):
    n = dy_phwc.shape[0]
    dx = phwc_empty(n, H + 2, W + 2, dy_phwc.device)
    dx_nchw = torch.empty(n, 32, H + 2, W + 2, device=dy_phwc.device)
    _chk(_lib.load().squint_op_conv32(1, n, H, W, _p(dy_phwc), _p(w_bwd), None, 0, _p(mask_phwc), _p(dx),
                                      _p(dx_nchw), _s()), "squint_op_conv32")
    return dx, dx_nchw


def wgrad32(x_phwc, dy_phwc, H, W):
    n = x_phwc.shape[0]
    L = _lib.load()
    work = torch.empty(max(L.squint_op_wgrad32_workspace(n), 16), dtype=torch.uint8, device=x_phwc.device)
    dw = torch.empty(32, 32, 3, 3, device=x_phwc.device)
    db = torch.empty(32, device=x_phwc.device)
    _chk(L.squint_op_wgrad32(n, H, W, _p(x_phwc), _p(dy_phwc), _p(dw), _p(db), _p(work), work.numel(), _s()),
         "squint_op_wgrad32")
    return dw, db
