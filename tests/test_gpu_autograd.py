"""autograd.Function wrappers over the layer kernels (needs a GB300).

FP64 layers (Linear, Conv3x3) are checked by torch.autograd.gradcheck: central
finite differences with h = 1e-6 in FP64 against the hand-written backward
kernels.  The FP32-only layers (LayerNorm, categorical CE, tanh-Gaussian) are
checked against the FP64 oracle's analytic gradients (relative error <= 1e-4 in
norm) and against FP32 central differences along random directions (h = 1e-2,
relative error <= 2e-2: rounding of an FP32 loss divided by h bounds it; the
ReLU variant of LayerNorm only against the oracle, since a finite step crosses
the kink).  A
small encoder + LayerNorm-MLP critic composed from the wrappers is compared
parameter by parameter with the oracle's chain of layer backwards.
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    from paper_2602_21203_gb300 import autograd
    return autograd


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _d(*shape, g, scale=1.0):
    return (torch.randn(*shape, generator=g, dtype=torch.float64) * scale).cuda().requires_grad_()


def test_linear_gradcheck_fp64(ag):
    g = torch.Generator().manual_seed(1)
    x, w, b = _d(5, 7, g=g), _d(3, 7, g=g), _d(3, g=g)
    assert torch.autograd.gradcheck(ag.linear, (x, w, b), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("stride", [1, 2])
@pytest.mark.parametrize("relu", [False, True])
def test_conv3x3_gradcheck_fp64(ag, stride, relu):
    g = torch.Generator().manual_seed(2 + stride + 2 * relu)
    x, w, b = _d(2, 3, 9, 8, g=g), _d(4, 3, 3, 3, g=g, scale=0.4), _d(4, g=g)
    f = lambda x, w, b: ag.conv3x3(x, w, b, stride, relu)
    assert torch.autograd.gradcheck(f, (x, w, b), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_encoder_then_linear_gradcheck_fp64(ag):
    """Two ReLU convolutions (stride 2, 1), flatten, a linear layer: the encoder path's
    kernels chained by autograd, against FP64 central differences."""
    g = torch.Generator().manual_seed(3)
    x = _d(2, 3, 16, 16, g=g)
    w1, b1 = _d(8, 3, 3, 3, g=g, scale=0.3), _d(8, g=g, scale=0.1)
    w2, b2 = _d(8, 8, 3, 3, g=g, scale=0.2), _d(8, g=g, scale=0.1)
    wl, bl = _d(5, 8 * 5 * 5, g=g, scale=0.1), _d(5, g=g)

    def f(x, w1, b1, w2, b2, wl, bl):
        h = ag.conv3x3(ag.conv3x3(x, w1, b1, 2, True), w2, b2, 1, True)
        return ag.linear(h.reshape(h.shape[0], -1), wl, bl)

    assert torch.autograd.gradcheck(f, (x, w1, b1, w2, b2, wl, bl), eps=1e-6, atol=1e-7, rtol=1e-5)


def _fd_dir(f, args, i, g, h=1e-2, n=3):
    """(FD, analytic) directional derivatives of scalar f w.r.t. args[i] along n random directions."""
    out = f(*args)
    grad, = torch.autograd.grad(out, args[i])
    res = []
    for _ in range(n):
        v = torch.randn(args[i].shape, generator=g).to(args[i])
        with torch.no_grad():
            p = [a.detach().clone() for a in args]
            p[i] = args[i].detach() + h * v
            fp = float(f(*p))
            p[i] = args[i].detach() - h * v
            fm = float(f(*p))
        res.append(((fp - fm) / (2 * h), float((grad * v).sum())))
    return res


def _check_fd(pairs, tol=2e-2):
    for fd, an in pairs:
        assert abs(fd - an) <= tol * max(abs(an), 1e-2), (fd, an)


@pytest.mark.parametrize("relu", [False, True])
def test_layernorm_fp32_vs_oracle_and_fd(ag, relu):
    g = torch.Generator().manual_seed(4 + relu)
    x = (torch.randn(9, 40, generator=g) * 2 + 0.3).cuda().requires_grad_()
    gam = (torch.rand(40, generator=g) + 0.5).cuda().requires_grad_()
    bet = torch.randn(40, generator=g).cuda().requires_grad_()
    wts = torch.randn(9, 40, generator=g).cuda()
    f = lambda x, gm, bt: (ag.layer_norm(x, gm, bt, relu) * wts).sum()
    out = f(x, gam, bet)
    gx, gg, gb = torch.autograd.grad(out, (x, gam, bet))
    y, cache = o.layernorm_fwd(x.detach().double().cpu().numpy(), gam.detach().double().cpu().numpy(),
                               bet.detach().double().cpu().numpy(), 1e-5)
    dy = wts.double().cpu().numpy() * ((y > 0) if relu else 1.0)
    rx, rg, rb = o.layernorm_bwd(dy, gam.detach().double().cpu().numpy(), cache)
    assert _rel(gx.cpu(), rx) < 1e-4
    assert _rel(gg.cpu(), rg) < 1e-4
    assert _rel(gb.cpu(), rb) < 1e-4
    if not relu:   # a step of h moves outputs near zero across the ReLU kink: no FD there
        for i in range(3):
            _check_fd(_fd_dir(f, (x, gam, bet), i, g))


def test_categorical_ce_fp32_vs_oracle_and_fd(ag):
    cfg = synth.make_config("train_b512")
    g = torch.Generator().manual_seed(6)
    logits = (torch.randn(12, cfg["atoms"], generator=g) * 2).cuda().requires_grad_()
    m = torch.rand(12, cfg["atoms"], generator=g)
    m = (m / m.sum(1, keepdim=True)).cuda()
    f = lambda l: ag.categorical_ce(l, m, cfg["v_min"], cfg["v_max"])
    loss = f(logits)
    gl, = torch.autograd.grad(loss, logits)
    lsm = o.log_softmax(logits.detach().double().cpu().numpy())
    mn = m.double().cpu().numpy()
    assert abs(float(loss.detach()) - float(-(mn * lsm).sum(1).mean())) < 1e-5
    assert _rel(gl.cpu(), (np.exp(lsm) - mn) / 12) < 1e-4
    _check_fd(_fd_dir(f, (logits,), 0, g))


def test_tanh_gaussian_fp32_vs_oracle_and_fd(ag):
    cfg = synth.make_config("train_b512")
    A = cfg["action_dim"]
    g = torch.Generator().manual_seed(7)
    out = torch.randn(10, 2 * A, generator=g).cuda().requires_grad_()
    eps = torch.randn(10, A, generator=g).cuda()
    wa = torch.randn(10, A, generator=g).cuda()
    wl = torch.randn(10, generator=g).cuda()

    def f(out):
        a, logp = ag.tanh_gaussian(out, eps, cfg["log_std_min"], cfg["log_std_max"])
        return (a * wa).sum() + (logp * wl).sum() * 0.1

    go, = torch.autograd.grad(f(out), out)
    _, _, cache = o.tanh_gaussian(out.detach().double().cpu().numpy(), eps.double().cpu().numpy(), cfg)
    ref = o.tanh_gaussian_bwd(wa.double().cpu().numpy(), 0.1 * wl.double().cpu().numpy(), cache, cfg)
    assert _rel(go.cpu(), ref) < 1e-4
    _check_fd(_fd_dir(f, (out,), 0, g, h=1e-3))


def test_small_critic_composition_matches_oracle_chain(ag):
    """conv(s2) -> conv -> flatten -> [Linear -> LN+ReLU] x 2 -> Linear -> CE, FP32 wrappers
    vs the same network through the oracle's FP64 layer functions and backwards."""
    cfg = synth.make_config("tiny_b8")
    K = cfg["atoms"]
    g = torch.Generator().manual_seed(8)
    B = 8
    x = torch.rand(B, 3, 16, 16, generator=g) - 0.5
    shapes = {"w1": (8, 3, 3, 3), "b1": (8,), "w2": (8, 8, 3, 3), "b2": (8,),
              "l1": (32, 200), "c1": (32,), "g1": (32,), "e1": (32,),
              "l2": (32, 32), "c2": (32,), "g2": (32,), "e2": (32,),
              "l3": (K, 32), "c3": (K,)}
    P = {}
    for k, s in shapes.items():
        t = torch.randn(*s, generator=g) * (0.3 if k[0] in "wl" else 0.1)
        if k[0] == "g":
            t = 1.0 + t
        P[k] = t
    m = torch.rand(B, K, generator=g)
    m = m / m.sum(1, keepdim=True)
    T = {k: v.cuda().requires_grad_() for k, v in P.items()}
    h = ag.conv3x3(ag.conv3x3(x.cuda(), T["w1"], T["b1"], 2, True), T["w2"], T["b2"], 1, True)
    h = h.reshape(B, -1)
    h = ag.layer_norm(ag.linear(h, T["l1"], T["c1"]), T["g1"], T["e1"], True)
    h = ag.layer_norm(ag.linear(h, T["l2"], T["c2"]), T["g2"], T["e2"], True)
    loss = ag.categorical_ce(ag.linear(h, T["l3"], T["c3"]), m.cuda(), cfg["v_min"], cfg["v_max"])
    grads = dict(zip(T, torch.autograd.grad(loss, list(T.values()))))

    # the same network on the oracle's FP64 layers, backward by hand
    N = {k: v.double().numpy() for k, v in P.items()}
    xn, mn = x.double().numpy(), m.double().numpy()
    a1 = np.maximum(o.conv3x3_fwd(xn, N["w1"], N["b1"], 2), 0)
    a2 = np.maximum(o.conv3x3_fwd(a1, N["w2"], N["b2"], 1), 0)
    z = a2.reshape(B, -1)
    p1 = z @ N["l1"].T + N["c1"]
    n1, c1 = o.layernorm_fwd(p1, N["g1"], N["e1"], 1e-5)
    r1 = np.maximum(n1, 0)
    p2 = r1 @ N["l2"].T + N["c2"]
    n2, c2 = o.layernorm_fwd(p2, N["g2"], N["e2"], 1e-5)
    r2 = np.maximum(n2, 0)
    lg = r2 @ N["l3"].T + N["c3"]
    lsm = o.log_softmax(lg)
    assert abs(float(loss) - float(-(mn * lsm).sum(1).mean())) < 1e-5
    R = {}
    dlg = (np.exp(lsm) - mn) / B
    R["l3"], R["c3"] = dlg.T @ r2, dlg.sum(0)
    dn2 = (dlg @ N["l3"]) * (n2 > 0)
    dp2, R["g2"], R["e2"] = o.layernorm_bwd(dn2, N["g2"], c2)
    R["l2"], R["c2"] = dp2.T @ r1, dp2.sum(0)
    dn1 = (dp2 @ N["l2"]) * (n1 > 0)
    dp1, R["g1"], R["e1"] = o.layernorm_bwd(dn1, N["g1"], c1)
    R["l1"], R["c1"] = dp1.T @ z, dp1.sum(0)
    dz = (dp1 @ N["l1"]).reshape(a2.shape) * (a2 > 0)
    da1, R["w2"], R["b2"] = o.conv3x3_bwd(a1, N["w2"], dz, 1)
    _, R["w1"], R["b1"] = o.conv3x3_bwd(xn, N["w1"], da1 * (a1 > 0), 2, need_dx=False)
    for k in shapes:
        assert _rel(grads[k].cpu(), R[k]) < 1e-4, k


# ---------------------------------------------------------------- BF16 tensor-core wrappers
def _bf(t):
    """FP64 numpy copy of t rounded to BF16 (the operand the tensor-core kernels read)."""
    return t.detach().to(torch.bfloat16).double().cpu().numpy()


def _fd_check(F, X, G, g, n=3, h=1e-6):
    """Central differences of the FP64 function F at X along n random directions against
    the analytic gradient G (FP64 numpy arrays): the largest discrepancy relative to the
    typical size of a directional derivative, ||G|| ||V|| / sqrt(size) (a single projection
    can pass near zero, where a plain relative error says nothing)."""
    worst = 0.0
    for _ in range(n):
        V = torch.randn(X.shape, generator=g, dtype=torch.float64).numpy()
        fd = (F(X + h * V) - F(X - h * V)) / (2 * h)
        an = float((G * V).sum())
        scale = float(np.linalg.norm(G) * np.linalg.norm(V)) / np.sqrt(V.size)
        worst = max(worst, abs(fd - an) / max(scale, 1e-30))
    return worst


def test_linear_bf16_gradients_vs_fp64_on_bf16_operands(ag):
    """Forward within 1e-5 of FP64 on the same BF16 operands; dx and dW within 1e-2 of the
    FP64 gradients and of FP64 central differences (dy is rounded to BF16: 2^-9 per element)."""
    g = torch.Generator().manual_seed(11)
    x = torch.randn(37, 70, generator=g).cuda().requires_grad_()
    w = (torch.randn(50, 70, generator=g) * 0.1).cuda().requires_grad_()
    b = torch.randn(50, generator=g).cuda().requires_grad_()
    r = torch.randn(37, 50, generator=g).cuda()
    y = ag.linear_bf16(x, w, b)
    (y * r).sum().backward()
    xh, wh, bn, rn = _bf(x), _bf(w), b.detach().double().cpu().numpy(), r.double().cpu().numpy()
    assert _rel(y.detach().cpu().numpy(), xh @ wh.T + bn) < 1e-5
    gx, gw, gb = x.grad.double().cpu().numpy(), w.grad.double().cpu().numpy(), b.grad.double().cpu().numpy()
    assert _rel(gx, rn @ wh) < 1e-2
    assert _rel(gw, rn.T @ xh) < 1e-2
    assert _rel(gb, rn.sum(0)) < 1e-5
    assert _fd_check(lambda X: float((rn * (X @ wh.T + bn)).sum()), xh, gx, g) < 1e-2
    assert _fd_check(lambda W: float((rn * (xh @ W.T + bn)).sum()), wh, gw, g) < 1e-2


@pytest.mark.parametrize("relu", [False, True])
def test_conv32_bf16_gradients_vs_oracle(ag, relu):
    """The tensor-core 32-channel convolution (forward, data gradient, weight gradient) against
    the oracle's conv3x3 on the same BF16 operands: forward 1e-5, gradients 1e-2 of the
    oracle's conv3x3_bwd and of FP64 central differences."""
    g = torch.Generator().manual_seed(12 + relu)
    x = torch.randn(6, 32, 13, 11, generator=g).cuda().requires_grad_()
    w = (torch.randn(32, 32, 3, 3, generator=g) * 0.06).cuda().requires_grad_()
    b = (0.1 * torch.randn(32, generator=g)).cuda().requires_grad_()
    y = ag.conv32_bf16(x, w, b, relu)
    r = torch.randn(y.shape, generator=g).cuda()
    (y * r).sum().backward()
    xh, wh, bn, rn = _bf(x), _bf(w), b.detach().double().cpu().numpy(), r.double().cpu().numpy()
    pre = o.conv3x3_fwd(xh, wh, bn, 1)
    act = (lambda v: np.maximum(v, 0.0)) if relu else (lambda v: v)
    assert _rel(y.detach().cpu().numpy(), act(pre)) < 1e-5
    rdx, rdw, rdb = o.conv3x3_bwd(xh, wh, rn * (pre > 0) if relu else rn, 1)
    gx, gw, gb = x.grad.double().cpu().numpy(), w.grad.double().cpu().numpy(), b.grad.double().cpu().numpy()
    assert _rel(gx, rdx) < 1e-2 and _rel(gw, rdw) < 1e-2 and _rel(gb, rdb) < 1e-2
    assert _fd_check(lambda X: float((rn * act(o.conv3x3_fwd(X, wh, bn, 1))).sum()), xh, gx, g) < 1e-2
    assert _fd_check(lambda W: float((rn * act(o.conv3x3_fwd(xh, W, bn, 1))).sum()), wh, gw, g) < 1e-2


def test_mlp_head_bf16_gradients_vs_oracle(ag):
    """A LayerNorm MLP head through MlpHeadBF16 (fused forward, hand-written backward
    kernels) against the oracle's mlp_fwd / mlp_bwd on the same BF16 weights and input:
    output and every gradient within the BF16 bounds (5e-2 relative in norm, cosine > 0.99)."""
    g = torch.Generator().manual_seed(13)
    rows, kin, H, nout = 50, 40, 64, 11
    cfg = dict(hidden=[H, H], ln_eps=1e-5)
    params, P = [], {}
    ins = [kin, H, H]
    for l in range(3):
        n_out = H if l < 2 else nout
        w = (torch.rand(n_out, ins[l], generator=g) * 2 - 1) / ins[l] ** 0.5
        bb = 0.1 * torch.randn(n_out, generator=g)
        params += [w.cuda().requires_grad_(), bb.cuda().requires_grad_()]
        P[f"c.fc{l}.w"], P[f"c.fc{l}.b"] = _bf(w), bb.double().numpy()
        if l < 2:
            gg, be = 1 + 0.1 * torch.randn(H, generator=g), 0.1 * torch.randn(H, generator=g)
            params += [gg.cuda().requires_grad_(), be.cuda().requires_grad_()]
            P[f"c.ln{l}.g"], P[f"c.ln{l}.b"] = gg.double().numpy(), be.double().numpy()
    x = torch.randn(rows, kin, generator=g).cuda().requires_grad_()
    out = ag.mlp_head_bf16(x, params)
    r = torch.randn(rows, nout, generator=g).cuda()
    (out * r).sum().backward()
    ref, cache = o.mlp_fwd(P, "c", _bf(x), cfg)
    assert _rel(out.detach().cpu().numpy(), ref) < 1e-2
    rdx, rg = o.mlp_bwd(P, "c", cache, r.double().cpu().numpy(), cfg)
    names = []
    for l in range(3):
        names += [f"c.fc{l}.w", f"c.fc{l}.b"] + ([f"c.ln{l}.g", f"c.ln{l}.b"] if l < 2 else [])
    for name, p in zip(names, params):
        got, want = p.grad.double().cpu().numpy(), rg[name]
        cos = float((got.ravel() @ want.ravel()) / max(np.linalg.norm(got) * np.linalg.norm(want), 1e-30))
        assert _rel(got, want) < 5e-2 and cos > 0.99, (name, _rel(got, want), cos)
    gx = x.grad.double().cpu().numpy()
    assert _rel(gx, rdx) < 5e-2
