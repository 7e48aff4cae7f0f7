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
