"""Squint visual SAC update and actor inference: plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.  This module is the independent definition the CUDA
path is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import or run it; the product path never does.

What it computes (one update = Algorithm 1, body of the inner loop):
  1. sample a minibatch from the replay ring                      (Alg. 1, "Sample mini-batch")
  2. random shift (replicate pad + crop) and squint: area
     downsampling by an integer factor f                          (Sec. IV "Resolution Squinting")
  3. shared conv encoder on o_t and o_{t+1}                       (Sec. III, Sec. IV "Encoder Design Choices")
  4. per-head one-layer projections + LayerNorm                   (Sec. IV "Encoder Design Choices", "Normalization")
  5. distributional (C51) target from the average of the two
     target critics, with the soft entropy term                   (Eq. 1, Alg. 1 "Compute target Q-value", Sec. IV "Critic Design Choices")
  6. critic + encoder step: cross-entropy against the projected
     target, summed over both critics                             (Eq. 2 in its distributional form, Alg. 1 "Update critic and encoder")
  7. entropy-temperature step                                     (Sec. III, Alg. 1 "Update entropy temperature")
  8. actor step on stop-gradient features, average of the two
     critics                                                      (Eq. 3, Alg. 1 "Update actor")
  9. polyak update of the target critics                          (Sec. III, Alg. 1 "Update target critic")
Optimiser: Adam (the paper says only "stochastic gradient descent", Sec. III).

Readings of what the paper leaves open are listed where they are used; every
one is stated once more, with its reason, in the design notes.

Parity pins: tests/test_oracle_*.py check this file against closed forms,
invariants, brute force and central finite differences, never against itself.
"""
import math

import numpy as np

from . import philox as px

LOG2 = math.log(2.0)
HALF_LOG_2PI = 0.5 * math.log(2.0 * math.pi)


# --------------------------------------------------------------------------
# configuration and parameter layout
# --------------------------------------------------------------------------

def dims(cfg):
    """Derived sizes: training resolution, conv output sizes, feature widths."""
    f = cfg["squint_f"]
    hs, ws = cfg["obs_h"] // f, cfg["obs_w"] // f
    n_conv = cfg["conv_layers"]
    strides = (cfg.get("conv_strides") or [2] + [1] * (n_conv - 1)) if n_conv > 0 else []
    conv = []
    cin, h, w = cfg["obs_c"], hs, ws
    for s in strides:
        oh, ow = (h - 3) // s + 1, (w - 3) // s + 1
        conv.append(dict(cin=cin, cout=cfg["conv_ch"], h=h, w=w, oh=oh, ow=ow, s=s))
        cin, h, w = cfg["conv_ch"], oh, ow
    # state-based SAC (Fig. 6 left: the encoder removed): no image features at all
    feat = cin * h * w if n_conv > 0 else 0
    d = cfg["proj_dim"]
    zdim = d if d > 0 else feat
    return dict(hs=hs, ws=ws, conv=conv, feat=feat, zdim=zdim,
                critic_in=zdim + cfg["proprio_dim"] + cfg["action_dim"],
                actor_in=zdim + cfg["proprio_dim"])


def param_spec(cfg):
    """Canonical parameter list: (name, shape, init kind, fan_in).

    Order = flat layout of the state: encoder, critic projection, critics,
    actor projection, actor, log_alpha.  Weights are [out, in] row-major.
    """
    dm = dims(cfg)
    spec = []
    for l, c in enumerate(dm["conv"]):
        fan = c["cin"] * 9
        spec.append((f"enc.conv{l}.w", (c["cout"], c["cin"], 3, 3), "U", fan))
        spec.append((f"enc.conv{l}.b", (c["cout"],), "U", fan))
    d = cfg["proj_dim"]

    def proj(prefix):
        out = []
        if d > 0:
            out.append((f"{prefix}.proj.w", (d, dm["feat"]), "U", dm["feat"]))
            out.append((f"{prefix}.proj.b", (d,), "U", dm["feat"]))
            out.append((f"{prefix}.proj.ln.g", (d,), "ONE", 0))
            out.append((f"{prefix}.proj.ln.b", (d,), "ZERO", 0))
        return out

    def mlp(prefix, din, dout):
        out = []
        for l, h in enumerate(cfg["hidden"]):
            out.append((f"{prefix}.fc{l}.w", (h, din), "U", din))
            out.append((f"{prefix}.fc{l}.b", (h,), "U", din))
            out.append((f"{prefix}.ln{l}.g", (h,), "ONE", 0))
            out.append((f"{prefix}.ln{l}.b", (h,), "ZERO", 0))
            din = h
        n = len(cfg["hidden"])
        out.append((f"{prefix}.fc{n}.w", (dout, din), "U", din))
        out.append((f"{prefix}.fc{n}.b", (dout,), "U", din))
        return out

    spec += proj("critic")
    for i in range(cfg["n_critics"]):
        spec += mlp(f"critic{i}", dm["critic_in"], critic_out(cfg))
    spec += proj("actor")
    spec += mlp("actor", dm["actor_in"], 2 * cfg["action_dim"])
    spec.append(("log_alpha", (1,), "LOGALPHA", 0))
    return spec


def critic_kind(cfg):
    """'c51' (categorical critic, Sec. IV "Critic Design Choices") or 'mse' (scalar Q, Eq. 2)."""
    return cfg.get("critic", "c51")


def critic_out(cfg):
    """Width of a critic's output layer: the atoms, or one value for the MSE critic."""
    return 1 if critic_kind(cfg) == "mse" else cfg["atoms"]


def group_of(name):
    """Optimiser group: the encoder trains with the critic (Sec. III: encoder trained by critic gradients)."""
    if name.startswith("enc.") or name.startswith("critic"):
        return "critic"
    if name.startswith("actor"):
        return "actor"
    return "alpha"


def is_target(name):
    """Target copies exist for the critic projection and the critics; the encoder has none (Alg. 1 encodes o_{t+1} with f_psi)."""
    return name.startswith("critic")


def init_params(cfg):
    """Uniform(+-1/sqrt(fan_in)) weights and biases, LayerNorm gain 1 / bias 0, log(alpha0).

    Element e of tensor t draws block (e, STREAM_INIT, t); the value is formed in
    FP64 and rounded once to FP32, the precision the state is stored in.
    """
    params = {}
    for t, (name, shape, kind, fan) in enumerate(param_spec(cfg)):
        n = int(np.prod(shape))
        if kind == "U":
            w = px.block(cfg["seed"], np.arange(n), px.STREAM_INIT, t)[0]
            val = (2.0 * px.uniform01(w) - 1.0) * (1.0 / math.sqrt(fan))
        elif kind == "ONE":
            val = np.ones(n)
        elif kind == "ZERO":
            val = np.zeros(n)
        else:
            val = np.full(n, math.log(cfg["init_alpha"]))
        params[name] = val.astype(np.float32).astype(np.float64).reshape(shape)
    return params


def init_state(cfg, params=None):
    """Learner state: parameters, Adam moments, target critics, step counters."""
    p = init_params(cfg) if params is None else {k: np.array(v, dtype=np.float64) for k, v in params.items()}
    return dict(
        params=p,
        m={k: np.zeros_like(v) for k, v in p.items()},
        v={k: np.zeros_like(v) for k, v in p.items()},
        target={k: v.copy() for k, v in p.items() if is_target(k)},
        steps=dict(critic=0, actor=0, alpha=0),
        update_idx=0,
    )


# --------------------------------------------------------------------------
# front end: sampling, random shift, squint
# --------------------------------------------------------------------------

def sample_indices(cfg, u, n_slots):
    """Uniform minibatch slots (Alg. 1 "Sample mini-batch"); next slot is (idx+1) mod N."""
    b = np.arange(cfg["batch"])
    idx = px.mulhi_range(px.block(cfg["seed"], b, px.STREAM_INDEX, u)[0], n_slots)
    return idx, (idx + 1) % n_slots


def sample_shifts(cfg, u, stream):
    """Crop offsets (dx, dy) in [0, 2p] for the replicate-padded image."""
    b = np.arange(cfg["batch"])
    w = px.block(cfg["seed"], b, stream, u)
    n = 2 * cfg["shift_pad"] + 1
    return px.mulhi_range(w[0], n), px.mulhi_range(w[1], n)


def shift_squint_sums(img, dx, dy, pad, f):
    """Integer box sums S[b,c,i,j] = sum_{u,v<f} I[b,c,clip(i*f+u+dy-p), clip(j*f+v+dx-p)].

    Random shift = replicate pad by p then crop at (dx, dy) (DrQ-style augmentation,
    by citation in Sec. III), then squint = area downsampling by f (Sec. IV).
    """
    bsz, c, h, w = img.shape
    hs, ws = h // f, w // f
    rows = np.clip(np.arange(hs * f)[None, :] + dy[:, None] - pad, 0, h - 1)   # [B, hs*f]
    cols = np.clip(np.arange(ws * f)[None, :] + dx[:, None] - pad, 0, w - 1)
    bi = np.arange(bsz)[:, None, None, None]
    ci = np.arange(c)[None, :, None, None]
    shifted = img[bi, ci, rows[:, None, :, None], cols[:, None, None, :]].astype(np.int64)
    return shifted.reshape(bsz, c, hs, f, ws, f).sum(axis=(3, 5))


def squint_store(img, f):
    """Squint at insert (Alg. 1: the transition is stored with Downsample(o); Sec. IV
    "Resolution Squinting", area downsampling): the f x f area mean of a uint8 frame,
    rounded half up to uint8, q = floor((S + floor(f^2 / 2)) / f^2), S the integer box sum.
    The update then reads q with f = 1: x = q / 255 - 0.5."""
    n, c, h, w = img.shape
    hs, ws = h // f, w // f
    s = img[:, :, :hs * f, :ws * f].astype(np.int64).reshape(n, c, hs, f, ws, f).sum(axis=(3, 5))
    return ((s + (f * f) // 2) // (f * f)).astype(np.uint8)


def squint_values(sums, f):
    """Pixel values from box sums: mean intensity in [0,1], centred: S/(255 f^2) - 0.5."""
    return sums.astype(np.float64) / (255.0 * f * f) - 0.5


def frontend(cfg, ring, u):
    """Steps a1-a4: indices, gathers, shifts, squint for o_t and o_{t+1} (state-based
    SAC, conv_layers = 0: no images, only the proprioceptive state and the transition)."""
    n_slots = ring["proprio"].shape[0]
    idx, nxt = sample_indices(cfg, u, n_slots)
    if cfg["conv_layers"] == 0:
        B = len(idx)
        empty = np.zeros((B, 0))
        return dict(
            idx=idx, nxt=nxt, x_t=empty, x_t1=empty,
            p_t=ring["proprio"][idx].astype(np.float64), a_t=ring["action"][idx].astype(np.float64),
            r=ring["reward"][idx].astype(np.float64), d=ring["done"][idx].astype(np.float64),
            p_t1=ring["proprio"][nxt].astype(np.float64),
        )
    dx0, dy0 = sample_shifts(cfg, u, px.STREAM_SHIFT_T)
    dx1, dy1 = sample_shifts(cfg, u, px.STREAM_SHIFT_T1)
    p, f = cfg["shift_pad"], cfg["squint_f"]
    s_t = shift_squint_sums(ring["obs"][idx], dx0, dy0, p, f)
    s_t1 = shift_squint_sums(ring["obs"][nxt], dx1, dy1, p, f)
    return dict(
        idx=idx, nxt=nxt, shift_t=np.stack([dx0, dy0], 1), shift_t1=np.stack([dx1, dy1], 1),
        sums_t=s_t, sums_t1=s_t1, x_t=squint_values(s_t, f), x_t1=squint_values(s_t1, f),
        p_t=ring["proprio"][idx].astype(np.float64), a_t=ring["action"][idx].astype(np.float64),
        r=ring["reward"][idx].astype(np.float64), d=ring["done"][idx].astype(np.float64),
        p_t1=ring["proprio"][nxt].astype(np.float64),
    )


# --------------------------------------------------------------------------
# layers with hand-written backward
# --------------------------------------------------------------------------

def conv3x3_fwd(x, w, b, s):
    """Valid 3x3 convolution with stride s: y[b,o,i,j] = bias[o] + sum_{c,ky,kx} w[o,c,ky,kx] x[b,c,s*i+ky,s*j+kx]."""
    _, _, h, wd = x.shape
    oh, ow = (h - 3) // s + 1, (wd - 3) // s + 1
    y = np.broadcast_to(b[None, :, None, None], (x.shape[0], w.shape[0], oh, ow)).copy()
    for ky in range(3):
        for kx in range(3):
            xs = x[:, :, ky:ky + s * (oh - 1) + 1:s, kx:kx + s * (ow - 1) + 1:s]
            y += np.einsum("bchw,oc->bohw", xs, w[:, :, ky, kx], optimize=True)
    return y


def conv3x3_bwd(x, w, dy, s, need_dx=True):
    """Gradients of conv3x3_fwd: (dx, dw, db)."""
    oh, ow = dy.shape[2], dy.shape[3]
    dw = np.zeros_like(w)
    dx = np.zeros_like(x) if need_dx else None
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(None), slice(ky, ky + s * (oh - 1) + 1, s), slice(kx, kx + s * (ow - 1) + 1, s))
            dw[:, :, ky, kx] = np.einsum("bohw,bchw->oc", dy, x[sl], optimize=True)
            if need_dx:
                dx[sl] += np.einsum("bohw,oc->bchw", dy, w[:, :, ky, kx], optimize=True)
    return dx, dw, dy.sum(axis=(0, 2, 3))


def layernorm_fwd(x, g, b, eps):
    """LayerNorm over the last axis (Ba et al., by citation in Sec. IV "Normalization")."""
    mu = x.mean(axis=-1, keepdims=True)
    var = ((x - mu) ** 2).mean(axis=-1, keepdims=True)
    rstd = 1.0 / np.sqrt(var + eps)
    xhat = (x - mu) * rstd
    return xhat * g + b, (xhat, rstd)


def layernorm_bwd(dy, g, cache):
    xhat, rstd = cache
    dxhat = dy * g
    dx = rstd * (dxhat - dxhat.mean(-1, keepdims=True) - xhat * (dxhat * xhat).mean(-1, keepdims=True))
    return dx, (dy * xhat).reshape(-1, dy.shape[-1]).sum(0), dy.reshape(-1, dy.shape[-1]).sum(0)


def encoder_fwd(P, x, cfg):
    """Conv stack with ReLU after every layer, flattened in (C, H, W) order (no layers:
    state-based SAC, an empty feature vector)."""
    if cfg["conv_layers"] == 0:
        return np.zeros((x.shape[0], 0)), []
    cache = []
    h = x
    for l, c in enumerate(dims(cfg)["conv"]):
        y = np.maximum(conv3x3_fwd(h, P[f"enc.conv{l}.w"], P[f"enc.conv{l}.b"], c["s"]), 0.0)
        cache.append((h, y))
        h = y
    return h.reshape(h.shape[0], -1), cache


def encoder_bwd(P, cache, dz, cfg):
    grads = {}
    conv = dims(cfg)["conv"]
    if not conv:
        return grads
    dh = dz.reshape(cache[-1][1].shape)
    for l in reversed(range(len(conv))):
        xin, y = cache[l]
        dpre = dh * (y > 0)
        dx, dw, db = conv3x3_bwd(xin, P[f"enc.conv{l}.w"], dpre, conv[l]["s"], need_dx=l > 0)
        grads[f"enc.conv{l}.w"], grads[f"enc.conv{l}.b"] = dw, db
        dh = dx
    return grads


def proj_fwd(P, prefix, z, cfg):
    """Per-head one-layer projection: Linear then LayerNorm, no activation (reading R7)."""
    if cfg["proj_dim"] == 0:
        return z, None
    pre = z @ P[f"{prefix}.proj.w"].T + P[f"{prefix}.proj.b"]
    y, ln = layernorm_fwd(pre, P[f"{prefix}.proj.ln.g"], P[f"{prefix}.proj.ln.b"], cfg["ln_eps"])
    return y, (z, ln)


def proj_bwd(P, prefix, cache, dy, need_dz=True):
    z, ln = cache
    dpre, dg, db = layernorm_bwd(dy, P[f"{prefix}.proj.ln.g"], ln)
    grads = {f"{prefix}.proj.w": dpre.T @ z, f"{prefix}.proj.b": dpre.sum(0),
             f"{prefix}.proj.ln.g": dg, f"{prefix}.proj.ln.b": db}
    dz = dpre @ P[f"{prefix}.proj.w"] if need_dz else None
    return dz, grads


def mlp_fwd(P, prefix, x, cfg):
    """Hidden layers Linear -> LayerNorm -> ReLU (Sec. IV "Normalization"), output layer plain Linear."""
    cache = []
    h = x
    nh = len(cfg["hidden"])
    for l in range(nh):
        pre = h @ P[f"{prefix}.fc{l}.w"].T + P[f"{prefix}.fc{l}.b"]
        n, ln = layernorm_fwd(pre, P[f"{prefix}.ln{l}.g"], P[f"{prefix}.ln{l}.b"], cfg["ln_eps"])
        y = np.maximum(n, 0.0)
        cache.append((h, ln, y))
        h = y
    out = h @ P[f"{prefix}.fc{nh}.w"].T + P[f"{prefix}.fc{nh}.b"]
    cache.append((h,))
    return out, cache


def mlp_bwd(P, prefix, cache, dout, cfg, need_param_grads=True):
    """Backward of mlp_fwd: (d input, parameter grads or {})."""
    nh = len(cfg["hidden"])
    grads = {}
    h = cache[nh][0]
    if need_param_grads:
        grads[f"{prefix}.fc{nh}.w"] = dout.T @ h
        grads[f"{prefix}.fc{nh}.b"] = dout.sum(0)
    dh = dout @ P[f"{prefix}.fc{nh}.w"]
    for l in reversed(range(nh)):
        xin, ln, y = cache[l]
        dn = dh * (y > 0)
        dpre, dg, db = layernorm_bwd(dn, P[f"{prefix}.ln{l}.g"], ln)
        if need_param_grads:
            grads[f"{prefix}.ln{l}.g"], grads[f"{prefix}.ln{l}.b"] = dg, db
            grads[f"{prefix}.fc{l}.w"] = dpre.T @ xin
            grads[f"{prefix}.fc{l}.b"] = dpre.sum(0)
        dh = dpre @ P[f"{prefix}.fc{l}.w"]
    return dh, grads


def log_softmax(x):
    mx = x.max(-1, keepdims=True)
    s = x - mx
    return s - np.log(np.exp(s).sum(-1, keepdims=True))


def softmax(x):
    return np.exp(log_softmax(x))


def softplus(x):
    return np.logaddexp(0.0, x)


def tanh_gaussian(out, eps, cfg):
    """Tanh-squashed Gaussian policy head (SAC, Sec. III; reading R8).

    out = [mu, raw]; log_std = lo + (hi-lo)/2 * (tanh(raw)+1); u = mu + std*eps; a = tanh(u);
    log pi = sum_k [ -eps_k^2/2 - log_std_k - log(2 pi)/2 - 2 (log 2 - u_k - softplus(-2 u_k)) ].
    """
    A = cfg["action_dim"]
    mu, raw = out[:, :A], out[:, A:]
    lo, hi = cfg["log_std_min"], cfg["log_std_max"]
    th = np.tanh(raw)
    log_std = lo + 0.5 * (hi - lo) * (th + 1.0)
    std = np.exp(log_std)
    u = mu + std * eps
    a = np.tanh(u)
    logp = (-0.5 * eps ** 2 - log_std - HALF_LOG_2PI - 2.0 * (LOG2 - u - softplus(-2.0 * u))).sum(-1)
    return a, logp, (eps, th, std, a)


def tanh_gaussian_bwd(da, dlogp, cache, cfg):
    """d out from dL/da and dL/dlog pi (reparameterised: eps held fixed)."""
    eps, th, std, a = cache
    lo, hi = cfg["log_std_min"], cfg["log_std_max"]
    du = da * (1.0 - a ** 2) + dlogp[:, None] * 2.0 * a          # d log|det| / du = 2 tanh(u)
    dlog_std = du * std * eps - dlogp[:, None]
    draw = dlog_std * 0.5 * (hi - lo) * (1.0 - th ** 2)
    return np.concatenate([du, draw], axis=1)


# --------------------------------------------------------------------------
# networks
# --------------------------------------------------------------------------

def support(cfg):
    """Fixed atom support z_j = v_min + j * dz, j = 0..K-1 (C51, by citation in Sec. IV)."""
    K = cfg["atoms"]
    return cfg["v_min"] + np.arange(K) * ((cfg["v_max"] - cfg["v_min"]) / (K - 1))


def actor_fwd(P, z, prop, eps, cfg):
    """pi_phi(. | z, s^proprio): projection, MLP, tanh-Gaussian head."""
    h, pc = proj_fwd(P, "actor", z, cfg)
    out, mc = mlp_fwd(P, "actor", np.concatenate([h, prop], 1), cfg)
    a, logp, hc = tanh_gaussian(out, eps, cfg)
    return a, logp, (pc, mc, hc, out)


def critics_fwd(P, hc, prop, act, cfg):
    """Logits of every critic on [h_c, s^proprio, a]: [E, B, K]."""
    x = np.concatenate([hc, prop, act], 1)
    logits, caches = [], []
    for i in range(cfg["n_critics"]):
        lo, c = mlp_fwd(P, f"critic{i}", x, cfg)
        logits.append(lo)
        caches.append(c)
    return np.stack(logits), caches


def project_c51(pbar, r, d, logp, alpha, cfg):
    """Project the shifted, scaled support onto the fixed atoms (C51 distributional target).

    Tz_j = clip(r + gamma (1-d) (z_j - alpha log pi'), v_min, v_max)  (Eq. 1 on each atom),
    b = (Tz_j - v_min)/dz, l = floor b, u = ceil b; mass P_j goes (u-b) to l and (b-l) to u,
    all of it to l when l = u (reading R6: no mass lost on exact atoms).
    """
    K = cfg["atoms"]
    zj = support(cfg)
    dz = (cfg["v_max"] - cfg["v_min"]) / (K - 1)
    tz = np.clip(r[:, None] + cfg["gamma"] * (1.0 - d[:, None]) * (zj[None, :] - alpha * logp[:, None]),
                 cfg["v_min"], cfg["v_max"])
    b = np.clip((tz - cfg["v_min"]) / dz, 0.0, K - 1)
    lo = np.floor(b).astype(np.int64)
    up = np.ceil(b).astype(np.int64)
    m = np.zeros_like(pbar)
    rows = np.repeat(np.arange(pbar.shape[0])[:, None], K, 1)
    np.add.at(m, (rows, lo), pbar * (up - b))
    np.add.at(m, (rows, up), pbar * (b - lo))
    np.add.at(m, (rows, lo), pbar * (lo == up))
    return m


def q_values(logits, cfg):
    """Q_i = sum_j softmax(logits_i)_j z_j: mean of the categorical return distribution
    (the MSE critic's output is Q itself)."""
    if critic_kind(cfg) == "mse":
        return logits[..., 0]
    return (softmax(logits) * support(cfg)).sum(-1)


def combine_critics(q, cfg):
    """How the two critics' values combine (Sec. IV "Critic Design Choices"): their average
    (Squint's choice), or with clipped double Q (cfg "cdq") the smaller per sample, ties to
    critic 0.  Returns the combined value [B] and the index of the critic used [B] (or None
    for the average)."""
    if cfg.get("cdq", False):
        pick = np.argmin(q, axis=0)
        return q[pick, np.arange(q.shape[1])], pick
    return q.mean(0), None


# --------------------------------------------------------------------------
# losses with their gradients
# --------------------------------------------------------------------------

def target_distribution(P, T, z_t1, fe, alpha, eps, cfg):
    """Alg. 1 "Compute target Q-value" in distributional form (no gradient).

    a' ~ pi(.|z_{t+1}, s'), target critics on [h_bar(z_{t+1}), s', a'], the two
    categorical distributions averaged (Squint: average, not clipped double Q, Sec. IV),
    then projected with the soft term alpha log pi'.  Variants: with "cdq" the
    distribution of the target critic with the smaller mean is used per sample; the MSE
    critic (Eq. 1-2) returns the scalar TD target y as m[:, 0].
    """
    a1, logp1, _ = actor_fwd(P, z_t1, fe["p_t1"], eps, cfg)
    hbar, _ = proj_fwd(T, "critic", z_t1, cfg)
    logits_bar, _ = critics_fwd(T, hbar, fe["p_t1"], a1, cfg)
    if critic_kind(cfg) == "mse":
        # Eq. 1: y = r + gamma (1 - d) (Q_bar(s', a') - alpha log pi'), Q_bar combined over critics
        qbar, _ = combine_critics(logits_bar[..., 0], cfg)
        y = fe["r"] + cfg["gamma"] * (1.0 - fe["d"]) * (qbar - alpha * logp1)
        return dict(a_next=a1, logp_next=logp1, logits_target=logits_bar, m=y[:, None])
    probs = softmax(logits_bar)
    if cfg.get("cdq", False):
        # clipped double Q on distributions: per sample, the distribution of the target critic
        # whose mean is smaller
        _, pick = combine_critics(q_values(logits_bar, cfg), cfg)
        pbar = probs[pick, np.arange(probs.shape[1])]
    else:
        pbar = probs.mean(0)
    m = project_c51(pbar, fe["r"], fe["d"], logp1, alpha, cfg)
    return dict(a_next=a1, logp_next=logp1, logits_target=logits_bar, pbar=pbar, m=m)


def critic_loss(P, x_t, fe, m, cfg, with_grads=True):
    """L_c = sum_i mean_b [ -sum_j m_bj log softmax(logits_i,b)_j ], gradient to critics, projection, encoder."""
    B = x_t.shape[0]
    z, enc_cache = encoder_fwd(P, x_t, cfg)
    hc, pcache = proj_fwd(P, "critic", z, cfg)
    logits, caches = critics_fwd(P, hc, fe["p_t"], fe["a_t"], cfg)
    if critic_kind(cfg) == "mse":
        # Eq. 2: sum over critics of mean_b (Q_i - y)^2, y = m[:, 0] held fixed
        err = logits[..., 0] - m[None, :, 0]
        loss = float((err ** 2).mean(1).sum())
        out = dict(loss=loss, logits=logits, z=z, q=q_values(logits, cfg))
        if not with_grads:
            return out
        dlogits = (2.0 * err / B)[..., None]
    else:
        lsm = log_softmax(logits)
        loss = float(-(m[None] * lsm).sum(-1).mean(1).sum())
        out = dict(loss=loss, logits=logits, z=z, q=q_values(logits, cfg))
        if not with_grads:
            return out
        dlogits = (np.exp(lsm) - m[None]) / B            # d CE / d logits = softmax - m (sum_j m_j = 1)
    grads = {}
    zdim = hc.shape[1]
    dhc = np.zeros_like(hc)
    for i in range(cfg["n_critics"]):
        dx, g = mlp_bwd(P, f"critic{i}", caches[i], dlogits[i], cfg)
        grads.update(g)
        dhc += dx[:, :zdim]
    if cfg["proj_dim"] > 0:
        dz, g = proj_bwd(P, "critic", pcache, dhc)
        grads.update(g)
    else:
        dz = dhc
    grads.update(encoder_bwd(P, enc_cache, dz, cfg))
    out["grads"] = grads
    out["dlogits"] = dlogits
    return out


def actor_loss(P, z_sg, prop, eps, alpha, cfg, with_grads=True):
    """L_pi = mean_b [ alpha log pi(a~|z_sg,s) - (1/2) sum_i Q_i(z_sg, s, a~) ]  (Eq. 3, Alg. 1 "Update actor");
    with "cdq" the smaller of the two Q_i per sample instead of their average.

    z_sg is the stop-gradient encoder output; the critics (incl. their projection)
    are held fixed; gradients reach the actor projection and actor MLP only.
    """
    B = z_sg.shape[0]
    E = cfg["n_critics"]
    a, logp, acache = actor_fwd(P, z_sg, prop, eps, cfg)
    hc, _ = proj_fwd(P, "critic", z_sg, cfg)
    logits, caches = critics_fwd(P, hc, prop, a, cfg)
    q = q_values(logits, cfg)                             # [E, B]
    qc, pick = combine_critics(q, cfg)
    loss = float((alpha * logp - qc).mean())
    out = dict(loss=loss, a=a, logp=logp, q=q)
    if not with_grads:
        return out
    A = cfg["action_dim"]
    da = np.zeros_like(a)
    for i in range(E):
        # d(-mean_b Qc)/dQ_i: -1/(E B) for the average, -1/B where critic i is the minimum
        dq = np.full(B, -1.0 / (E * B)) if pick is None else np.where(pick == i, -1.0 / B, 0.0)
        if critic_kind(cfg) == "mse":
            dlogit = dq[:, None]
        else:
            prob = softmax(logits[i])
            zj = support(cfg)
            dlogit = dq[:, None] * prob * (zj[None, :] - q[i][:, None])   # dQ/dlogit_j = p_j (z_j - Q)
        dx, _ = mlp_bwd(P, f"critic{i}", caches[i], dlogit, cfg, need_param_grads=False)
        da += dx[:, -A:]
    pc, mc, hcache, _ = acache
    dout = tanh_gaussian_bwd(da, np.full(B, alpha / B), hcache, cfg)
    dx, grads = mlp_bwd(P, "actor", mc, dout, cfg)
    if cfg["proj_dim"] > 0:
        zdim = cfg["proj_dim"]
        _, g = proj_bwd(P, "actor", pc, dx[:, :zdim], need_dz=False)
        grads.update(g)
    out["grads"] = grads
    return out


def alpha_loss(log_alpha, logp, cfg):
    """L_alpha = -alpha * mean_b(log pi_b + H_target); d/d log_alpha = L_alpha (reading R9: standard SAC sign)."""
    alpha = math.exp(log_alpha)
    val = -alpha * float(np.mean(logp + target_entropy(cfg)))
    return val, val


def target_entropy(cfg):
    te = cfg.get("target_entropy")
    return -float(cfg["action_dim"]) if te is None else float(te)


# --------------------------------------------------------------------------
# optimiser and target update
# --------------------------------------------------------------------------

def adam_step(state, names, grads, group, cfg):
    """Adam (Kingma & Ba): bias-corrected moments, no weight decay (reading R15)."""
    state["steps"][group] += 1
    t = state["steps"][group]
    b1, b2, e, lr = cfg["adam_b1"], cfg["adam_b2"], cfg["adam_eps"], cfg["lr"]
    for k in names:
        g = grads[k]
        state["m"][k] = b1 * state["m"][k] + (1.0 - b1) * g
        state["v"][k] = b2 * state["v"][k] + (1.0 - b2) * g * g
        mhat = state["m"][k] / (1.0 - b1 ** t)
        vhat = state["v"][k] / (1.0 - b2 ** t)
        state["params"][k] = state["params"][k] - lr * mhat / (np.sqrt(vhat) + e)


def polyak(state, cfg):
    """theta_bar <- (1 - tau) theta_bar + tau theta; tau = 1 - rho of Alg. 1 (reading R12)."""
    tau = cfg["tau"]
    for k in state["target"]:
        state["target"][k] = (1.0 - tau) * state["target"][k] + tau * state["params"][k]


# --------------------------------------------------------------------------
# one update (Algorithm 1, inner loop body)
# --------------------------------------------------------------------------

def update(state, ring, cfg):
    """Run one SAC update in place; returns (stats, trace)."""
    u = state["update_idx"]
    P = state["params"]
    fe = frontend(cfg, ring, u)
    B = cfg["batch"]
    A = cfg["action_dim"]
    alpha = math.exp(float(P["log_alpha"][0]))

    # encode o_{t+1} (no gradient) and the target distribution
    z_t1, _ = encoder_fwd(P, fe["x_t1"], cfg)
    eps_tgt = px.normal_pairs(cfg["seed"], px.STREAM_EPS_TARGET, u, B, A)
    tgt = target_distribution(P, state["target"], z_t1, fe, alpha, eps_tgt, cfg)

    # critic + encoder step
    crit = critic_loss(P, fe["x_t"], fe, tgt["m"], cfg)
    z_sg = crit["z"]                                   # pre-update encoder features, detached
    names = [n for n, *_ in param_spec(cfg) if group_of(n) == "critic"]
    adam_step(state, names, crit["grads"], "critic", cfg)

    # entropy temperature step: log pi from the (not yet updated) actor at s_t
    eps_act = px.normal_pairs(cfg["seed"], px.STREAM_EPS_ACTOR, u, B, A)
    _, logp_t, _ = actor_fwd(P, z_sg, fe["p_t"], eps_act, cfg)
    la_loss, la_grad = alpha_loss(float(P["log_alpha"][0]), logp_t, cfg)
    adam_step(state, ["log_alpha"], {"log_alpha": np.array([la_grad])}, "alpha", cfg)
    alpha_new = math.exp(float(P["log_alpha"][0]))

    # actor step every policy_freq updates (counted from 1, Alg. 1)
    act = None
    if (u + 1) % cfg["policy_freq"] == 0:
        act = actor_loss(P, z_sg, fe["p_t"], eps_act, alpha_new, cfg)
        names = [n for n, *_ in param_spec(cfg) if group_of(n) == "actor"]
        adam_step(state, names, act["grads"], "actor", cfg)

    polyak(state, cfg)
    state["update_idx"] = u + 1

    stats = dict(
        critic_loss=crit["loss"],
        actor_loss=act["loss"] if act else float("nan"),
        alpha_loss=la_loss,
        alpha=alpha_new,
        q_mean=float(crit["q"].mean()),
        entropy=float(-logp_t.mean()),
    )
    trace = dict(frontend=fe, z_t1=z_t1, eps_target=eps_tgt, eps_actor=eps_act, target=tgt,
                 critic=crit, logp_t=logp_t, actor=act, alpha_before=alpha)
    return stats, trace


# --------------------------------------------------------------------------
# actor inference (Alg. 1, "downsample" and "sample a_t")
# --------------------------------------------------------------------------

def act(P, obs, prop, key, sample, cfg):
    """Actions for one request of n environments: squint without shift, encode, actor.

    Row b of a request with 64-bit key k draws its noise from blocks
    (b, STREAM_ACT | q << 16, k), so a row's action does not depend on which
    other requests share its batch.  `sample` False returns tanh(mu).
    """
    n = np.asarray(prop).shape[0]
    if cfg["conv_layers"] == 0:                       # state-based: no observation image
        z = np.zeros((n, 0))
    else:
        p, f = cfg["shift_pad"], cfg["squint_f"]
        centre = np.full(n, p)
        x = squint_values(shift_squint_sums(obs, centre, centre, p, f), f)
        z, _ = encoder_fwd(P, x, cfg)
    A = cfg["action_dim"]
    h, _ = proj_fwd(P, "actor", z, cfg)
    out, _ = mlp_fwd(P, "actor", np.concatenate([h, np.asarray(prop, dtype=np.float64)], 1), cfg)
    if not sample:
        return np.tanh(out[:, :A])
    eps = px.normal_pairs(cfg["seed"], px.STREAM_ACT, key, n, A)
    a, _, _ = tanh_gaussian(out, eps, cfg)
    return a
