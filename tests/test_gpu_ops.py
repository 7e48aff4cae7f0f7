"""Layer operations (include/squint_ops.h) vs the FP64 oracle's layers (needs a GB300).

The BF16 tensor-core GEMM is checked against the FP64 product of the same
BF16-rounded operands (only the FP32 accumulation order differs): relative
error in norm <= 1e-5.  FP64 layer kernels match the oracle to 1e-12, FP32 ones
to 1e-5.
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    from paper_2602_21203_gb300 import ops
    return ops


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _operand(rows, cols, mn_major, g):
    """A (rows x cols) BF16 operand; mn_major stores it transposed (rows contiguous) with a padded stride."""
    x = torch.randn(rows, cols, generator=g).to(torch.bfloat16)
    if not mn_major:
        ld = (cols + 7) // 8 * 8
        buf = torch.zeros(rows, ld, dtype=torch.bfloat16)
        buf[:, :cols] = x
        return x, buf.cuda()[:, :cols]
    ld = (rows + 7) // 8 * 8
    buf = torch.zeros(cols, ld, dtype=torch.bfloat16)
    buf[:, :rows] = x.t()
    return x, buf.cuda()[:, :rows].t()


SHAPES = [(512, 512, 512), (300, 101, 274), (128, 12, 512), (1024, 256, 2592), (7, 16, 64), (256, 200, 512),
          (1, 1, 8)]


@pytest.mark.parametrize("a_mn", [False, True])
@pytest.mark.parametrize("b_mn", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_bf16_tensor_core_gemm(ops, a_mn, b_mn, shape):
    M, N, K = shape
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    a, A = _operand(M, K, a_mn, g)
    b, B = _operand(N, K, b_mn, g)
    bias = torch.randn(N, generator=g)
    out = ops.gemm(A, B, bias=bias.cuda(), M=M, N=N, K=K)
    torch.cuda.synchronize()
    ref = a.double().numpy() @ b.double().numpy().T + bias.double().numpy()
    assert _rel(out.cpu().numpy(), ref) < 1e-5, (shape, a_mn, b_mn)


def test_bf16_gemm_accumulates(ops):
    g = torch.Generator().manual_seed(3)
    a, A = _operand(256, 128, False, g)
    b, B = _operand(128, 128, True, g)
    base = torch.randn(256, 128, generator=g)
    out = base.clone().cuda()
    ops.gemm(A, B, out=out, accumulate=True)
    torch.cuda.synchronize()
    ref = base.double().numpy() + a.double().numpy() @ b.double().numpy().T
    assert _rel(out.cpu().numpy(), ref) < 1e-5


SPLIT_SHAPES = [(512, 256, 2592), (512, 512, 512), (300, 101, 2740), (128, 12, 4096), (1, 1, 800),
                (256, 2592, 512), (130, 130, 1536)]


@pytest.mark.parametrize("a_mn,b_mn", [(False, False), (False, True), (True, True)])
@pytest.mark.parametrize("shape", SPLIT_SHAPES)
def test_bf16_gemm_k_split_over_cluster(ops, a_mn, b_mn, shape):
    """Few output tiles and a long K split K over a CTA cluster: same product (FP64 of
    the BF16 operands), identical bits on a repeat call, accumulate adds onto the output."""
    M, N, K = shape
    g = torch.Generator().manual_seed(M + 5 * N + 11 * K)
    a, A = _operand(M, K, a_mn, g)
    b, B = _operand(N, K, b_mn, g)
    bias = torch.randn(N, generator=g)
    out = ops.gemm(A, B, bias=bias.cuda(), M=M, N=N, K=K)
    again = ops.gemm(A, B, bias=bias.cuda(), M=M, N=N, K=K)
    torch.cuda.synchronize()
    ref = a.double().numpy() @ b.double().numpy().T + bias.double().numpy()
    assert _rel(out.cpu().numpy(), ref) < 1e-5, (shape, a_mn, b_mn)
    assert torch.equal(out, again)
    base = torch.randn(M, N, generator=g)
    acc = base.clone().cuda()
    ops.gemm(A, B, out=acc, accumulate=True, M=M, N=N, K=K)
    torch.cuda.synchronize()
    ref2 = base.double().numpy() + a.double().numpy() @ b.double().numpy().T
    assert _rel(acc.cpu().numpy(), ref2) < 1e-5


LN_SHAPES = [(512, 512, 512), (300, 256, 274), (37, 300, 64), (1, 16, 8), (1030, 1024, 128)]


@pytest.mark.parametrize("shape", LN_SHAPES)
@pytest.mark.parametrize("relu", [True, False])
def test_gemm_with_fused_layernorm(ops, shape, relu):
    """GEMM + LayerNorm (+ReLU) in one kernel vs the FP64 GEMM of the same BF16 operands
    followed by the oracle's LayerNorm."""
    M, N, K = shape
    g = torch.Generator().manual_seed(M + N + K)
    a, A = _operand(M, K, False, g)             # row strides padded to multiples of 8
    b = (torch.randn(N, K, generator=g) * 0.1).bfloat16()
    buf = torch.zeros(N, (K + 7) // 8 * 8, dtype=torch.bfloat16)
    buf[:, :K] = b
    B = buf.cuda()[:, :K]
    bias = torch.randn(N, generator=g)
    gam = torch.rand(N, generator=g) + 0.5
    bet = torch.randn(N, generator=g) * 0.2
    pre, post, post_bf, mean, rstd = ops.gemm_layernorm(A, B, bias.cuda(), gam.cuda(), bet.cuda(), 1e-5, relu)
    torch.cuda.synchronize()
    ref_pre = a.double().numpy() @ b.double().numpy().T + bias.double().numpy()
    ref, (xhat, rs) = o.layernorm_fwd(ref_pre, gam.double().numpy(), bet.double().numpy(), 1e-5)
    if relu:
        ref = np.maximum(ref, 0)
    assert _rel(pre.cpu().numpy(), ref_pre) < 1e-5
    assert _rel(post.cpu().numpy(), ref) < 1e-4
    assert _rel(rstd.cpu().numpy(), rs.ravel()) < 1e-4
    assert _rel(mean.cpu().numpy(), ref_pre.mean(1)) < 1e-4 or np.abs(mean.cpu().numpy() - ref_pre.mean(1)).max() < 1e-4
    assert torch.equal(post_bf.cpu(), post.cpu().bfloat16())


FP8_SHAPES = [(512, 512, 512), (512, 256, 2592), (300, 101, 274), (7, 16, 64), (1, 1, 8), (1024, 12, 272)]


@pytest.mark.parametrize("shape", FP8_SHAPES)
def test_fp8_gemm_matches_quantised_product(ops, shape):
    """e4m3 GEMM with per-tensor scales vs the FP64 product of the same quantised operands
    (quantised here with PyTorch's float8_e4m3fn conversion: x / (amax / 448), nearest)."""
    M, N, K = shape
    g = torch.Generator().manual_seed(M + 3 * N + 7 * K)
    a = (torch.randn(M, K, generator=g) * 3).bfloat16()
    b = (torch.randn(N, K, generator=g) * 0.05).bfloat16()
    bias = torch.randn(N, generator=g)
    out, (sa, sb) = ops.gemm_fp8(a.cuda(), b.cuda(), bias=bias.cuda())
    torch.cuda.synchronize()

    def quant(x):
        x = x.float()
        s = x.abs().max() / 448.0
        return (x / s).to(torch.float8_e4m3fn).double(), s

    aq, ra = quant(a)
    bq, rb = quant(b)
    assert float(sa) == float(ra) and float(sb) == float(rb)
    ref = (aq @ bq.T) * (ra.double() * rb.double()) + bias.double()
    assert _rel(out.cpu().numpy(), ref.numpy()) < 1e-5, shape
    # and the quantisation error itself is what e4m3 allows (3 mantissa bits)
    full = a.double() @ b.double().T + bias.double()
    assert _rel(out.cpu().numpy(), full.numpy()) < 0.1


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_cuda_core_gemm_layouts(ops, dtype):
    g = torch.Generator().manual_seed(4)
    for M, N, K in [(70, 33, 129), (512, 512, 512)]:
        a = torch.randn(M, K, generator=g, dtype=torch.float64)
        b = torch.randn(N, K, generator=g, dtype=torch.float64)
        ref = a.numpy() @ b.numpy().T
        for at in (False, True):
            for bt in (False, True):
                A = (a.t().contiguous().t() if at else a).to(dtype).cuda()
                B = (b.t().contiguous().t() if bt else b).to(dtype).cuda()
                out = ops.gemm(A, B)
                torch.cuda.synchronize()
                tol = 1e-12 if dtype == torch.float64 else 1e-5
                assert _rel(out.cpu().numpy(), ref) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-6)])
@pytest.mark.parametrize("stride", [1, 2])
@pytest.mark.parametrize("cout", [8, 32])
def test_conv3x3_matches_oracle(ops, dtype, tol, stride, cout):
    g = torch.Generator().manual_seed(5 + stride + cout)
    x = torch.randn(5, 3, 17, 15, generator=g, dtype=torch.float64)
    w = torch.randn(cout, 3, 3, 3, generator=g, dtype=torch.float64) * 0.3
    b = torch.randn(cout, generator=g, dtype=torch.float64)
    y = ops.conv3x3_fwd(x.to(dtype).cuda(), w.to(dtype).cuda(), b.to(dtype).cuda(), stride, relu=False)
    ref = o.conv3x3_fwd(x.numpy(), w.numpy(), b.numpy(), stride)
    assert _rel(y.cpu().numpy(), ref) < tol
    dy = torch.randn(*ref.shape, generator=g, dtype=torch.float64)
    dx, dw, db = ops.conv3x3_bwd(x.to(dtype).cuda(), w.to(dtype).cuda(), dy.to(dtype).cuda(), stride)
    rdx, rdw, rdb = o.conv3x3_bwd(x.numpy(), w.numpy(), dy.numpy(), stride)
    assert _rel(dx.cpu().numpy(), rdx) < tol
    assert _rel(dw.cpu().numpy(), rdw) < tol
    assert _rel(db.cpu().numpy(), rdb) < tol


def test_first_layer_weight_gradient_at_training_shape(ops):
    """The 3 -> 32 stride-2 layer's weight gradient over 512 images of 32x32 (the split
    over pixels and its fixed-order reduction) vs the FP64 oracle."""
    g = torch.Generator().manual_seed(77)
    x = torch.rand(512, 3, 32, 32, generator=g, dtype=torch.float64) - 0.5
    w = torch.randn(32, 3, 3, 3, generator=g, dtype=torch.float64) * 0.2
    dy = torch.randn(512, 32, 15, 15, generator=g, dtype=torch.float64) * 1e-3
    dx, dw, db = ops.conv3x3_bwd(x.float().cuda(), w.float().cuda(), dy.float().cuda(), 2)
    _, rdw, rdb = o.conv3x3_bwd(x.float().double().numpy(), w.float().double().numpy(), dy.float().double().numpy(), 2)
    assert _rel(dw.cpu().numpy(), rdw) < 1e-5
    assert _rel(db.cpu().numpy(), rdb) < 1e-5


@pytest.mark.parametrize("relu", [False, True])
def test_layernorm_matches_oracle(ops, relu):
    g = torch.Generator().manual_seed(6)
    x = torch.randn(37, 300, generator=g, dtype=torch.float64) * 2 + 0.5
    gam = torch.rand(300, generator=g, dtype=torch.float64) + 0.5
    bet = torch.randn(300, generator=g, dtype=torch.float64)
    y, mean, rstd = ops.layernorm_fwd(x.float().cuda(), gam.float().cuda(), bet.float().cuda(), 1e-5, relu)
    ry, cache = o.layernorm_fwd(x.numpy(), gam.numpy(), bet.numpy(), 1e-5)
    if relu:
        ry = np.maximum(ry, 0)
    assert _rel(y.cpu().numpy(), ry) < 1e-5
    dy = torch.randn(37, 300, generator=g, dtype=torch.float64)
    dx, dg, db = ops.layernorm_bwd(dy.float().cuda(), y, x.float().cuda(), mean, rstd, gam.float().cuda(), relu)
    dyn = dy.numpy() * (ry > 0) if relu else dy.numpy()
    rdx, rdg, rdb = o.layernorm_bwd(dyn, gam.numpy(), cache)
    assert _rel(dx.cpu().numpy(), rdx) < 1e-4
    assert _rel(dg.cpu().numpy(), rdg) < 1e-5
    assert _rel(db.cpu().numpy(), rdb) < 1e-5


def test_categorical_ce_matches_oracle(ops):
    cfg = synth.make_config("train_b512")
    g = torch.Generator().manual_seed(7)
    logits = torch.randn(64, 101, generator=g, dtype=torch.float64) * 3
    m = torch.rand(64, 101, generator=g, dtype=torch.float64)
    m /= m.sum(1, keepdim=True)
    loss, d, q = ops.categorical_ce(logits.float().cuda(), m.float().cuda(), -20, 20, 1 / 64)
    lsm = o.log_softmax(logits.numpy())
    assert _rel(loss.cpu().numpy(), -(m.numpy() * lsm).sum(1)) < 1e-5
    assert _rel(d.cpu().numpy(), (np.exp(lsm) - m.numpy()) / 64) < 1e-5
    assert _rel(q.cpu().numpy(), o.q_values(logits.numpy(), cfg)) < 1e-5


@pytest.mark.parametrize("name", ["tiny_b8", "small_b32", "train_b512"])
def test_c51_projection_matches_oracle(ops, name):
    cfg = synth.make_config(name)
    K = cfg["atoms"]
    g = torch.Generator().manual_seed(8)
    rows = 40
    logits = torch.randn(2, rows, K, generator=g, dtype=torch.float64) * 2
    r = torch.randn(rows, generator=g, dtype=torch.float64) * 5
    d = (torch.rand(rows, generator=g) < 0.3).double()
    logp = torch.randn(rows, generator=g, dtype=torch.float64) * 3
    m = ops.c51_project(logits.float().cuda(), r.float().cuda(), d.float().cuda(), logp.float().cuda(), 0.17,
                        cfg["gamma"], cfg["v_min"], cfg["v_max"])
    pbar = o.softmax(logits.numpy()).mean(0)
    ref = o.project_c51(pbar, r.numpy(), d.numpy(), logp.numpy(), 0.17, cfg)
    mm = m.cpu().numpy()
    assert np.abs(mm - ref).max() < 2e-5
    assert np.allclose(mm.sum(1), 1, atol=1e-5)


def test_tanh_gaussian_matches_oracle(ops):
    cfg = synth.make_config("train_b512")
    g = torch.Generator().manual_seed(9)
    out = torch.randn(50, 12, generator=g, dtype=torch.float64)
    eps = torch.randn(50, 6, generator=g, dtype=torch.float64)
    a, logp = ops.tanh_gaussian_fwd(out.float().cuda(), eps.float().cuda())
    ra, rl, cache = o.tanh_gaussian(out.numpy(), eps.numpy(), cfg)
    assert _rel(a.cpu().numpy(), ra) < 1e-5
    assert np.abs(logp.cpu().numpy() - rl).max() < 1e-4
    da = torch.randn(50, 6, generator=g, dtype=torch.float64)
    dl = torch.randn(50, generator=g, dtype=torch.float64)
    dout = ops.tanh_gaussian_bwd(out.float().cuda(), eps.float().cuda(), da.float().cuda(), dl.float().cuda())
    ref = o.tanh_gaussian_bwd(da.numpy(), dl.numpy(), cache, cfg)
    assert _rel(dout.cpu().numpy(), ref) < 1e-5


# ---------------------------------------------------------------- tensor-core convolutions
@pytest.mark.parametrize("n,H", [(6, 15), (300, 13), (37, 11)])
def test_conv32_tensor_core_matches_oracle(ops, n, H):
    """32->32 stride-1 conv on tcgen05: forward (bias, ReLU), data gradient (ReLU mask of the
    layer below), weight and bias gradient, each vs the FP64 oracle on BF16-exact inputs."""
    g = torch.Generator().manual_seed(20 + H)
    W = H
    x = torch.randn(n, 32, H, W, generator=g).bfloat16().float()
    w = (torch.randn(32, 32, 3, 3, generator=g) * 0.1).bfloat16().float()
    b = torch.randn(32, generator=g)
    dy = torch.randn(n, 32, H - 2, W - 2, generator=g).bfloat16().float()
    xp = ops.to_phwc(x.cuda())
    assert torch.equal(ops.from_phwc(xp, H, W).cpu(), x)
    wf, wb = ops.conv32_layouts(w.cuda())
    y_p, y = ops.conv32_fwd(xp, H, W, wf, b.cuda(), relu=True)
    torch.cuda.synchronize()
    xn, wn = x.double().numpy(), w.double().numpy()
    ref = np.maximum(o.conv3x3_fwd(xn, wn, b.double().numpy(), 1), 0)
    assert _rel(y.cpu().numpy(), ref) < 1e-5
    assert torch.equal(ops.from_phwc(y_p, H - 2, W - 2).cpu(), y.cpu().bfloat16().float())
    dyp = ops.to_phwc(dy.cuda())
    dx_p, dx = ops.conv32_dgrad(dyp, H - 2, W - 2, wb, mask_phwc=xp)
    torch.cuda.synchronize()
    rdx, rdw, rdb = o.conv3x3_bwd(xn, wn, dy.double().numpy(), 1)
    assert _rel(dx.cpu().numpy(), rdx * (xn > 0)) < 1e-5
    dw, db = ops.wgrad32(xp, dyp, H, W)
    torch.cuda.synchronize()
    assert _rel(dw.cpu().numpy(), rdw) < 1e-5
    assert _rel(db.cpu().numpy(), rdb) < 1e-5


# (images, input channels, height = width, stride): the training encoder's first layer
# (3 x 32 x 32, stride 2) over several 128-pixel tiles with a ragged last one, a single
# image, one channel at stride 1, and the wider filters (K = 63, K = 108) of the other
# tile widths, stride 3
@pytest.mark.parametrize("n,cin,H,s", [(300, 3, 32, 2), (1, 3, 32, 2), (5, 1, 11, 1), (7, 7, 20, 2), (3, 12, 17, 3)])
def test_conv0_tensor_core_matches_oracle(ops, n, cin, H, s):
    """The first layer on tcgen05 (BF16 operands, FP32 accumulation) against the FP64
    oracle on the same BF16-rounded inputs: each output is the BF16 rounding of the
    oracle's value, or (an FP32 sum that lands on the other side of a rounding boundary)
    within one BF16 step of it; the 2-pixel border of the padded output is not touched."""
    g = torch.Generator().manual_seed(40 + cin + H)
    W = H
    x = torch.rand(n, cin, H, W, generator=g).bfloat16().float()
    w = (torch.randn(32, cin, 3, 3, generator=g) * 0.3).bfloat16().float()
    b = torch.randn(32, generator=g) * 0.1
    OH = (H - 3) // s + 1
    out = torch.full((n, OH + 4, OH + 4, 32), float("nan"), dtype=torch.bfloat16, device="cuda")
    ops.conv0_bf16(x.cuda(), w.cuda(), b.cuda(), s, out=out)
    torch.cuda.synchronize()
    got = out.float().cpu()
    border = torch.ones(OH + 4, OH + 4, dtype=torch.bool)
    border[2:OH + 2, 2:OH + 2] = False
    assert torch.isnan(got[:, border]).all()
    y = got[:, 2:OH + 2, 2:OH + 2, :].permute(0, 3, 1, 2).double().numpy()
    ref = np.maximum(o.conv3x3_fwd(x.double().numpy(), w.double().numpy(), b.double().numpy(), s), 0)
    ref_bf = torch.from_numpy(ref).to(torch.bfloat16).double().numpy()
    off = y != ref_bf
    assert np.all(np.abs(y - ref)[off] <= 2.0 ** -8 * np.abs(ref)[off] + 1e-6)
    assert off.mean() < 1e-2, off.mean()
