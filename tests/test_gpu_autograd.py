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
