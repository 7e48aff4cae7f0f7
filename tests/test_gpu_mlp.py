"""The fused LayerNorm-MLP head (one tensor-core launch per chain) against the FP64
oracle on the same BF16 operands (needs a GB300).

Each layer of the chain (Sec. IV "Normalization": Linear -> LayerNorm -> ReLU per
hidden layer, plain Linear output) is checked on the kernel's own inputs: layer l's
pre-activation against FP64 of (the kernel's BF16 output of layer l - 1) W_l^T + b_l,
its LayerNorm + ReLU output and row statistics against the oracle's LayerNorm of the
kernel's own pre-activation, the output layer likewise, all within 1e-5 relative in
norm (FP32 accumulation and statistics); the BF16 hidden outputs equal the rounding of
the kernel's own FP32 outputs bit for bit.  The whole chain is also compared with an
FP64 evaluation that rounds each hidden output to BF16 itself, within 1e-3: an element
whose FP32 and FP64 values straddle a BF16 rounding boundary rounds one way on each
side (2^-8 relative), which the next layers carry.  A row's result is the same bits
whichever rows share its launch.
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o

pytestmark = pytest.mark.gpu

EPS = 1e-5


def _bf16_round(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()


def _make(M, kin, H, nout, nh, seed):
    g = torch.Generator().manual_seed(seed)
    ldx = (kin + 7) // 8 * 8
    xs = torch.zeros(M, ldx)
    xs[:, :kin] = torch.randn(M, kin, generator=g)
    x = xs.to(torch.bfloat16).cuda()
    ws, bs, gs, betas = [], [], [], []
    ins = [kin] + [H] * nh
    outs = [H] * nh + [nout]
    for l in range(nh + 1):
        ld = (ins[l] + 7) // 8 * 8
        w = torch.zeros(outs[l], ld)
        w[:, :ins[l]] = (torch.rand(outs[l], ins[l], generator=g) * 2 - 1) / ins[l] ** 0.5
        ws.append(w.to(torch.bfloat16).cuda())
        bs.append((0.1 * torch.randn(outs[l], generator=g)).cuda())
        if l < nh:
            gs.append((1 + 0.1 * torch.randn(H, generator=g)).cuda())
            betas.append((0.1 * torch.randn(H, generator=g)).cuda())
    return x, ws, bs, gs, betas


def _reference(x, ws, bs, gs, betas, kin):
    """FP64 chain; each hidden output rounded to BF16 before the next layer reads it."""
    nh = len(gs)
    h = x.float().cpu().double().numpy()[:, :kin]
    saved = []
    for l in range(nh):
        w = ws[l].float().cpu().double().numpy()[:, :h.shape[1]]
        pre = h @ w.T + bs[l].cpu().double().numpy()
        y, (_, rstd) = o.layernorm_fwd(pre, gs[l].cpu().double().numpy(), betas[l].cpu().double().numpy(), EPS)
        post = np.maximum(y, 0.0)
        saved.append((pre, post, pre.mean(-1), rstd[:, 0]))
        h = _bf16_round(post)
    w = ws[nh].float().cpu().double().numpy()[:, :h.shape[1]]
    return h @ w.T + bs[nh].cpu().double().numpy(), saved


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


# (M, kin, H, nout, hidden layers, cluster): the training-shape critic pair's and actor's
# heads (274 / 268 inputs, 512-512, 101 atoms / 12 outputs), the small and tiny heads,
# ragged row counts, one and three hidden layers, a scalar (MSE) output
CASES = [
    (512, 274, 512, 101, 2, 0), (512, 274, 512, 101, 2, 2), (37, 274, 512, 101, 2, 4), (1024, 268, 512, 12, 2, 0),
    (300, 274, 512, 101, 2, 8), (1024, 268, 512, 12, 2, 8),
    (300, 418, 256, 51, 2, 0), (300, 418, 256, 51, 2, 1), (33, 418, 256, 51, 2, 2), (8, 218, 32, 11, 2, 0),
    (1, 218, 32, 11, 2, 0), (200, 64, 256, 16, 1, 0), (130, 96, 128, 1, 3, 0),
]


@pytest.mark.parametrize("M,kin,H,nout,nh,cl", CASES)
def test_fused_mlp_matches_oracle_chain(M, kin, H, nout, nh, cl):
    from paper_2602_21203_gb300 import ops
    x, ws, bs, gs, betas = _make(M, kin, H, nout, nh, seed=M + 7 * kin + H)
    xin = x[:, :kin]
    out, saved = ops.mlp_bf16(xin, [w[:, :(kin if l == 0 else H)] for l, w in enumerate(ws)], bs, gs, betas,
                              eps=EPS, cluster=cl)
    torch.cuda.synchronize()
    d = lambda t: t.float().cpu().double().numpy()
    h = d(xin)
    for l, (pre, post, pbf, mean, rstd) in enumerate(saved):
        # layer l on the kernel's own input
        rpre = h @ d(ws[l])[:, :h.shape[1]].T + d(bs[l])
        assert _rel(d(pre), rpre) < 1e-5, (l, "pre", _rel(d(pre), rpre))
        y, (_, rr) = o.layernorm_fwd(d(pre), d(gs[l]), d(betas[l]), EPS)
        assert _rel(d(post), np.maximum(y, 0.0)) < 1e-5, (l, "post", _rel(d(post), np.maximum(y, 0.0)))
        assert np.abs(d(mean) - d(pre).mean(-1)).max() < 1e-5 * max(1.0, float(np.abs(d(pre)).max())), (l, "mean")
        assert _rel(d(rstd), rr[:, 0]) < 1e-5, (l, "rstd")
        assert torch.equal(pbf, post.to(torch.bfloat16)), (l, "post_bf")
        h = d(pbf)
    rout = h @ d(ws[nh])[:, :H].T + d(bs[nh])
    assert _rel(d(out), rout) < 1e-5, ("out", _rel(d(out), rout))
    # the whole chain against an FP64 evaluation that rounds to BF16 on its own
    ref_out, _ = _reference(x, ws, bs, gs, betas, kin)
    assert _rel(d(out), ref_out) < 1e-3, _rel(d(out), ref_out)


def test_fused_mlp_rows_are_independent_of_their_batch():
    """A row's outputs are the same bits alone, in a sub-batch at another offset, and in the whole batch."""
    from paper_2602_21203_gb300 import ops
    M, kin, H, nout = 300, 274, 512, 101
    x, ws, bs, gs, betas = _make(M, kin, H, nout, 2, seed=11)
    wv = [w[:, :(kin if l == 0 else H)] for l, w in enumerate(ws)]
    full, _ = ops.mlp_bf16(x[:, :kin], wv, bs, gs, betas, eps=EPS, save=False)
    part, _ = ops.mlp_bf16(x[70:201, :kin], wv, bs, gs, betas, eps=EPS, save=False)
    one, _ = ops.mlp_bf16(x[155:156, :kin], wv, bs, gs, betas, eps=EPS, save=False)
    torch.cuda.synchronize()
    assert torch.equal(full[70:201], part)
    assert torch.equal(full[155:156], one)


def test_fused_mlp_rejects_shapes_outside_its_range():
    from paper_2602_21203_gb300 import lib, ops
    x, ws, bs, gs, betas = _make(16, 64, 48, 8, 2, seed=3)     # H = 48 is no multiple of 32
    with pytest.raises(lib.SquintError) as e:
        ops.mlp_bf16(x[:, :64], [ws[0][:, :64], ws[1][:, :48], ws[2][:, :48]], bs, gs, betas)
    assert e.value.code == lib.EINVAL


# ---------------------------------------------------------------- the backward chain
# (M, kin, H, nout, hidden layers, c0, ncols): the critics' backward to the projected
# features (columns 0..255 of 274, split over the output columns), the actor step's
# backward to the action columns (264..273, split over K), the actor's backward (268
# inputs, 12 outputs), ragged rows, the small head and a 64-wide one, one and three hidden
# layers (hidden widths below 64 are outside the kernel's range)
BWD_CASES = [
    (512, 274, 512, 101, 2, 0, 256), (512, 274, 512, 101, 2, 264, 10), (512, 268, 512, 12, 2, 0, 256),
    (37, 274, 512, 101, 2, 0, 256), (300, 274, 512, 101, 2, 264, 10), (300, 418, 256, 51, 2, 400, 18),
    (8, 218, 64, 11, 2, 200, 18), (200, 64, 256, 16, 1, 0, 64), (130, 96, 128, 1, 3, 0, 64),
]


@pytest.mark.parametrize("rebuild", [False, True], ids=["post", "rebuild"])
@pytest.mark.parametrize("M,kin,H,nout,nh,c0,ncols", BWD_CASES)
def test_fused_mlp_backward_matches_oracle_layer_by_layer(M, kin, H, nout, nh, c0, ncols, rebuild):
    """Each hidden layer's dpre against the oracle's LayerNorm backward (FP64) of dout or
    the kernel's own BF16 dpre of the layer above times the weight (5e-3 relative in norm:
    the BF16 rounding of dpre, 2^-9 per element); the input gradient 1e-5 of FP64 of the
    kernel's own dpre_0; the per-row-block column sums 1e-4 of FP64 column sums.  The ReLU
    mask read from the saved post, or rebuilt from pre, g and beta."""
    from paper_2602_21203_gb300 import ops
    x, ws, bs, gs, betas = _make(M, kin, H, nout, nh, seed=5 * M + kin + H)
    wv = [w[:, :(kin if l == 0 else H)] for l, w in enumerate(ws)]
    _, saved = ops.mlp_bf16(x[:, :kin], wv, bs, gs, betas, eps=EPS)
    g = torch.Generator().manual_seed(M + nout)
    ld = (nout + 7) // 8 * 8
    dbuf = torch.zeros(M, ld)
    dbuf[:, :nout] = torch.randn(M, nout, generator=g) * 0.1
    dout = dbuf.to(torch.bfloat16).cuda()[:, :nout]
    dx, dps, cps = ops.mlp_bf16_bwd(dout, wv, gs, saved, kin, c0, ncols, betas=betas if rebuild else None)
    torch.cuda.synchronize()
    d = lambda t: t.float().cpu().double().numpy()
    dy = d(dout)
    for lh in range(nh - 1, -1, -1):
        w_above = d(ws[lh + 1])[:, :H]
        dpost = dy @ w_above
        pre, post, _, mean, rstd = (d(t) for t in saved[lh])
        xhat = (pre - mean[:, None]) * rstd[:, None]
        dn = dpost * (post > 0)
        dpre, dg, db = o.layernorm_bwd(dn, d(gs[lh]), (xhat, rstd[:, None]))
        got = d(dps[lh])
        assert _rel(got, dpre) < 5e-3, (lh, "dpre", _rel(got, dpre))
        cols = d(cps[lh]).sum(0)                       # the row blocks added
        assert _rel(cols[0], dg) < 1e-4, (lh, "dg", _rel(cols[0], dg))
        assert _rel(cols[1], db) < 1e-4, (lh, "dbeta", _rel(cols[1], db))
        assert _rel(cols[2], dpre.sum(0)) < 1e-4, (lh, "dbias", _rel(cols[2], dpre.sum(0)))
        dy = got                                       # the next product reads the BF16 dpre
    ref_dx = dy @ d(ws[0])[:, c0:c0 + ncols]
    assert _rel(d(dx), ref_dx) < 1e-5, ("dx", _rel(d(dx), ref_dx))


def test_fused_mlp_backward_rejects_shapes_outside_its_range():
    from paper_2602_21203_gb300 import lib, ops
    x, ws, bs, gs, betas = _make(8, 218, 32, 11, 2, seed=9)     # 32-wide hidden layers
    wv = [w[:, :(218 if l == 0 else 32)] for l, w in enumerate(ws)]
    _, saved = ops.mlp_bf16(x[:, :218], wv, bs, gs, betas, eps=EPS)
    dout = torch.zeros(8, 16, dtype=torch.bfloat16, device="cuda")[:, :11]
    with pytest.raises(lib.SquintError) as e:
        ops.mlp_bf16_bwd(dout, wv, gs, saved, 218, 200, 18)
    assert e.value.code == lib.EINVAL


def test_fused_mlp_backward_rows_are_independent_of_their_batch():
    """The input gradient of a row is the same bits in the whole batch and in a sub-batch."""
    from paper_2602_21203_gb300 import ops
    M, kin, H, nout = 300, 274, 512, 101
    x, ws, bs, gs, betas = _make(M, kin, H, nout, 2, seed=17)
    wv = [w[:, :(kin if l == 0 else H)] for l, w in enumerate(ws)]
    _, saved = ops.mlp_bf16(x[:, :kin], wv, bs, gs, betas, eps=EPS)
    g = torch.Generator().manual_seed(3)
    dbuf = torch.zeros(M, 104)
    dbuf[:, :nout] = torch.randn(M, nout, generator=g) * 0.1
    dout = dbuf.to(torch.bfloat16).cuda()
    for c0, ncols in ((0, 256), (264, 10)):
        full, _, _ = ops.mlp_bf16_bwd(dout[:, :nout], wv, gs, saved, kin, c0, ncols, False, False)
        sub = [tuple(t[128:300] for t in sv) for sv in saved]
        part, _, _ = ops.mlp_bf16_bwd(dout[128:300, :nout], wv, gs, sub, kin, c0, ncols, False, False)
        torch.cuda.synchronize()
        assert torch.equal(full[128:300], part)


@pytest.mark.parametrize("M,kin,H,nout,nh,c0,ncols", [BWD_CASES[0], BWD_CASES[1], BWD_CASES[5], BWD_CASES[8]])
def test_fused_mlp_backward_rebuilt_mask_is_the_forward_mask(M, kin, H, nout, nh, c0, ncols):
    """The forward rounds post = max(fma(g, xhat, beta), 0) once; the backward's mask
    rebuilt from pre by the same expression is the saved post's mask, so the two modes
    give the same bits."""
    from paper_2602_21203_gb300 import ops
    x, ws, bs, gs, betas = _make(M, kin, H, nout, nh, seed=7 * M + H)
    wv = [w[:, :(kin if l == 0 else H)] for l, w in enumerate(ws)]
    _, saved = ops.mlp_bf16(x[:, :kin], wv, bs, gs, betas, eps=EPS)
    g = torch.Generator().manual_seed(M)
    ld = (nout + 7) // 8 * 8
    dbuf = torch.zeros(M, ld)
    dbuf[:, :nout] = torch.randn(M, nout, generator=g) * 0.1
    dout = dbuf.to(torch.bfloat16).cuda()[:, :nout]
    a = ops.mlp_bf16_bwd(dout, wv, gs, saved, kin, c0, ncols)
    b = ops.mlp_bf16_bwd(dout, wv, gs, saved, kin, c0, ncols, betas=betas)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0])
    for l in range(nh):
        assert torch.equal(a[1][l], b[1][l])
        assert torch.equal(a[2][l], b[2][l])
