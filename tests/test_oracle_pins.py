"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, brute force on tiny inputs, closed forms, invariants,
or a library routine in a special case where it computes the same thing.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import philox as px
from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- RNG

def test_philox_known_answers():
    """Philox4x32-10 reproduces the published known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = px.philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:]


def test_range_draw_is_floor_of_product():
    """idx = floor(w n / 2^32) checked with Python big integers, and lies in [0, n)."""
    rng = np.random.default_rng(1)
    w = rng.integers(0, 2 ** 32, size=1000, dtype=np.uint64)
    for n in (1, 17, 256, 100_000, 2 ** 31 + 7):
        got = px.mulhi_range(w, n)
        ref = np.array([(int(x) * n) >> 32 for x in w])
        assert np.array_equal(got, ref)
        assert got.min() >= 0 and got.max() < n


def test_uniform_and_normal_moments():
    """Uniforms lie strictly inside (0,1); Box-Muller normals have mean 0, variance 1, kurtosis 3."""
    w = px.block(7, np.arange(200_000), 3, 11)
    u = px.uniform01(w[0])
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 3e-3
    e = px.normal_pairs(7, px.STREAM_EPS_ACTOR, 5, 100_000, 6).ravel()
    assert abs(e.mean()) < 1e-2 and abs(e.var() - 1) < 1e-2
    assert abs(np.mean(e ** 4) - 3) < 5e-2


def test_streams_are_distinct():
    a = px.block(0, np.arange(64), px.STREAM_INDEX, 0)[0]
    b = px.block(0, np.arange(64), px.STREAM_SHIFT_T, 0)[0]
    c = px.block(0, np.arange(64), px.STREAM_INDEX, 1)[0]
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


# ---------------------------------------------------------------- squint

def _brute_sums(img, dx, dy, p, f):
    bsz, c, h, w = img.shape
    out = np.zeros((bsz, c, h // f, w // f), dtype=np.int64)
    for b in range(bsz):
        for ch in range(c):
            for i in range(h // f):
                for j in range(w // f):
                    s = 0
                    for uu in range(f):
                        for vv in range(f):
                            y = min(max(i * f + uu + dy[b] - p, 0), h - 1)
                            x = min(max(j * f + vv + dx[b] - p, 0), w - 1)
                            s += int(img[b, ch, y, x])
                    out[b, ch, i, j] = s
    return out


def test_minibatch_slots_and_crop_offsets_cover_their_ranges():
    """Alg. 1 "sample mini-batch": slots in [0, N) with the next slot (idx + 1) mod N;
    the crop offsets take every value of [0, 2p] and no other (p = 8, 512 samples, eight
    updates), x and y drawn separately, o_t and o_{t+1} separately."""
    cfg = synth.make_config("train_b512")
    p = cfg["shift_pad"]
    seen_x, seen_y = set(), set()
    for u in range(8):
        idx, nxt = o.sample_indices(cfg, u, 300)
        assert idx.min() >= 0 and idx.max() < 300 and np.array_equal(nxt, (idx + 1) % 300)
        dx, dy = o.sample_shifts(cfg, u, px.STREAM_SHIFT_T)
        dx1, dy1 = o.sample_shifts(cfg, u, px.STREAM_SHIFT_T1)
        seen_x |= set(dx.tolist()) | set(dx1.tolist())
        seen_y |= set(dy.tolist()) | set(dy1.tolist())
        assert not np.array_equal(dx, dy) and not np.array_equal(dx, dx1)
    assert seen_x == set(range(2 * p + 1)) and seen_y == set(range(2 * p + 1))
    idx, _ = o.sample_indices(cfg, 0, 2)                    # the smallest ring: both slots drawn
    assert set(idx.tolist()) == {0, 1}


def test_shift_squint_brute_force():
    rng = np.random.default_rng(2)
    img = rng.integers(0, 256, size=(3, 2, 12, 8), dtype=np.uint8)
    dx = np.array([0, 3, 6])
    dy = np.array([6, 0, 2])
    got = o.shift_squint_sums(img, dx, dy, 3, 4)
    assert np.array_equal(got, _brute_sums(img, dx, dy, 3, 4))


def test_squint_constant_image_is_constant():
    img = np.full((2, 3, 16, 16), 77, dtype=np.uint8)
    s = o.shift_squint_sums(img, np.array([0, 8]), np.array([5, 1]), 4, 4)
    assert np.all(s == 77 * 16)
    assert np.allclose(o.squint_values(s, 4), 77 / 255 - 0.5, rtol=0, atol=1e-15)


def test_centre_shift_and_unit_factor_is_identity():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(2, 3, 10, 10), dtype=np.uint8)
    s = o.shift_squint_sums(img, np.array([4, 4]), np.array([4, 4]), 4, 1)
    assert np.array_equal(s, img.astype(np.int64))


def test_squint_equals_area_pooling():
    """Unshifted squint equals average pooling / area interpolation (library special case)."""
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, size=(2, 3, 32, 32), dtype=np.uint8)
    s = o.shift_squint_sums(img, np.array([2, 2]), np.array([2, 2]), 2, 4)
    t = torch.from_numpy(img.astype(np.float64))
    pool = torch.nn.functional.avg_pool2d(t, 4).numpy()
    area = torch.nn.functional.interpolate(t, size=(8, 8), mode="area").numpy()
    assert np.allclose(s / 16.0, pool, atol=1e-12)
    assert np.allclose(s / 16.0, area, atol=1e-12)


def test_shift_is_a_translation():
    """Interior pixels move by (dx-p, dy-p): a shift of +1 reads the neighbouring column."""
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, size=(1, 1, 16, 16), dtype=np.uint8)
    a = o.shift_squint_sums(img, np.array([3]), np.array([2]), 2, 1)
    assert np.array_equal(a[0, 0, 2:12, 2:12], img[0, 0, 2:12, 3:13].astype(np.int64))


# ---------------------------------------------------------------- layers

def test_conv_matches_library_conv():
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, 3, 11, 9))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    for s in (1, 2):
        ref = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b), stride=s)
        assert np.allclose(o.conv3x3_fwd(x, w, b, s), ref.numpy(), atol=1e-12)


def test_conv_brute_force():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(1, 2, 7, 6))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    y = o.conv3x3_fwd(x, w, b, 2)
    for oc in range(3):
        for i in range(y.shape[2]):
            for j in range(y.shape[3]):
                ref = b[oc] + sum(w[oc, c, ky, kx] * x[0, c, 2 * i + ky, 2 * j + kx]
                                  for c in range(2) for ky in range(3) for kx in range(3))
                assert abs(y[0, oc, i, j] - ref) < 1e-12


def _fd(f, x, h=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = x[i]
        x[i] = old + h
        fp = f()
        x[i] = old - h
        fm = f()
        x[i] = old
        g[i] = (fp - fm) / (2 * h)
    return g


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(8)
    x = rng.normal(size=(2, 2, 7, 7))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    for s in (1, 2):
        proj = rng.normal(size=o.conv3x3_fwd(x, w, b, s).shape)
        f = lambda: float((o.conv3x3_fwd(x, w, b, s) * proj).sum())
        dx, dw, db = o.conv3x3_bwd(x, w, proj, s)
        assert np.allclose(dx, _fd(f, x), atol=1e-7)
        assert np.allclose(dw, _fd(f, w), atol=1e-7)
        assert np.allclose(db, _fd(f, b), atol=1e-7)


def test_layernorm_statistics_and_backward():
    rng = np.random.default_rng(9)
    x = rng.normal(size=(5, 16)) * 3 + 1
    y, cache = o.layernorm_fwd(x, np.ones(16), np.zeros(16), 1e-5)
    var = x.var(-1)
    assert np.allclose(y.mean(-1), 0, atol=1e-12)
    assert np.allclose(y.var(-1), var / (var + 1e-5), atol=1e-12)
    g = rng.normal(size=16)
    bb = rng.normal(size=16)
    proj = rng.normal(size=(5, 16))
    f = lambda: float((o.layernorm_fwd(x, g, bb, 1e-5)[0] * proj).sum())
    _, c2 = o.layernorm_fwd(x, g, bb, 1e-5)
    dx, dg, db = o.layernorm_bwd(proj, g, c2)
    assert np.allclose(dx, _fd(f, x), atol=1e-7)
    assert np.allclose(dg, _fd(f, g), atol=1e-7)
    assert np.allclose(db, _fd(f, bb), atol=1e-7)


def test_cross_entropy_gradient_closed_form():
    """d/dlogits of -sum m log softmax = softmax - m when sum m = 1; and CE >= H(m)."""
    rng = np.random.default_rng(10)
    logits = rng.normal(size=(4, 7))
    m = rng.random((4, 7))
    m /= m.sum(1, keepdims=True)
    f = lambda: float(-(m * o.log_softmax(logits)).sum())
    assert np.allclose(o.softmax(logits) - m, _fd(f, logits), atol=1e-8)
    ce = -(m * o.log_softmax(logits)).sum(1)
    ent = -(m * np.log(m)).sum(1)
    assert np.all(ce >= ent - 1e-12)


# ---------------------------------------------------------------- tanh-Gaussian

def _cfg_tiny(**kw):
    return synth.make_config("tiny_b8", **kw)


def test_tanh_gaussian_log_prob_change_of_variables():
    """log pi(a) = log N(u; mu, sigma) - sum log(1 - tanh(u)^2), evaluated directly."""
    from scipy.stats import norm
    cfg = _cfg_tiny()
    rng = np.random.default_rng(11)
    out = rng.normal(size=(16, 12))
    eps = rng.normal(size=(16, 6))
    a, logp, _ = o.tanh_gaussian(out, eps, cfg)
    mu = out[:, :6]
    log_std = -5 + 3.5 * (np.tanh(out[:, 6:]) + 1)
    u = mu + np.exp(log_std) * eps
    ref = (norm.logpdf(u, loc=mu, scale=np.exp(log_std)) - np.log(1 - np.tanh(u) ** 2)).sum(1)
    assert np.allclose(logp, ref, atol=1e-10)
    assert np.allclose(a, np.tanh(u))


def test_log_std_spans_its_bounds():
    """Reading R8: log sigma = lo + (hi - lo)(tanh(raw) + 1) / 2 covers [lo, hi], with the
    midpoint at raw = 0.  Read back from log pi at mu = 0, eps = 0 (u = 0, where the
    log-determinant term vanishes): log pi = -A (log sigma + log(2 pi) / 2)."""
    cfg = _cfg_tiny()
    A = cfg["action_dim"]
    lo, hi = cfg["log_std_min"], cfg["log_std_max"]
    for raw, want in ((-40.0, lo), (0.0, 0.5 * (lo + hi)), (40.0, hi)):
        out = np.concatenate([np.zeros((1, A)), np.full((1, A), raw)], axis=1)
        a, logp, _ = o.tanh_gaussian(out, np.zeros((1, A)), cfg)
        assert np.all(a == 0.0)
        log_std = -logp[0] / A - 0.5 * math.log(2 * math.pi)
        assert log_std == pytest.approx(want, abs=1e-12)


def test_tanh_gaussian_density_integrates_to_one():
    """For one action dimension the squashed density integrates to 1 over (-1, 1)."""
    from scipy.integrate import quad
    cfg = _cfg_tiny(action_dim=1)
    for mu, raw in ((0.3, -0.2), (-1.1, 0.4), (0.0, -1.5)):
        log_std = -5 + 3.5 * (math.tanh(raw) + 1)
        sd = math.exp(log_std)

        def dens(a):
            u = math.atanh(a)
            eps = (u - mu) / sd
            _, lp, _ = o.tanh_gaussian(np.array([[mu, raw]]), np.array([[eps]]), cfg)
            return math.exp(lp[0])

        tot, _ = quad(dens, -1 + 1e-12, 1 - 1e-12, limit=400, points=[math.tanh(mu)])
        assert abs(tot - 1) < 1e-6


def test_tanh_gaussian_backward_finite_differences():
    cfg = _cfg_tiny()
    rng = np.random.default_rng(12)
    out = rng.normal(size=(5, 12))
    eps = rng.normal(size=(5, 6))
    wa = rng.normal(size=(5, 6))
    wl = rng.normal(size=5)
    f = lambda: float((o.tanh_gaussian(out, eps, cfg)[0] * wa).sum() + (o.tanh_gaussian(out, eps, cfg)[1] * wl).sum())
    _, _, cache = o.tanh_gaussian(out, eps, cfg)
    assert np.allclose(o.tanh_gaussian_bwd(wa, wl, cache, cfg), _fd(f, out), atol=1e-7)


# ---------------------------------------------------------------- C51 projection

def _hat_projection(pbar, r, d, logp, alpha, cfg):
    """Brute force: m_j = sum_i P_i max(0, 1 - |b_i - j|) (linear interpolation onto atoms)."""
    K = cfg["atoms"]
    dz = (cfg["v_max"] - cfg["v_min"]) / (K - 1)
    m = np.zeros_like(pbar)
    for row in range(pbar.shape[0]):
        for i in range(K):
            zi = cfg["v_min"] + i * dz
            tz = min(max(r[row] + cfg["gamma"] * (1 - d[row]) * (zi - alpha * logp[row]), cfg["v_min"]), cfg["v_max"])
            b = (tz - cfg["v_min"]) / dz
            for j in range(K):
                m[row, j] += pbar[row, i] * max(0.0, 1.0 - abs(b - j))
    return m


def _rand_dist(rng, rows, K):
    p = rng.random((rows, K))
    return p / p.sum(1, keepdims=True)


@pytest.mark.parametrize("name", ["tiny_b8", "small_b32"])
def test_projection_matches_hat_kernel_and_keeps_mass(name):
    cfg = synth.make_config(name)
    rng = np.random.default_rng(13)
    rows = 12
    pbar = _rand_dist(rng, rows, cfg["atoms"])
    r = rng.normal(size=rows) * 3
    d = (rng.random(rows) < 0.3).astype(float)
    logp = rng.normal(size=rows) * 4
    m = o.project_c51(pbar, r, d, logp, 0.2, cfg)
    assert np.allclose(m, _hat_projection(pbar, r, d, logp, 0.2, cfg), atol=1e-12)
    assert np.allclose(m.sum(1), 1.0, atol=1e-12)
    assert np.all(m >= 0)


def test_projection_on_atom_is_one_hot():
    """Terminal transitions whose reward sits on an atom project to a one-hot on that atom."""
    cfg = _cfg_tiny()                      # 11 atoms on [-10, 10]: spacing exactly 2
    rng = np.random.default_rng(14)
    atoms = o.support(cfg)
    for j in (0, 3, 5, 10):
        pbar = _rand_dist(rng, 1, 11)
        m = o.project_c51(pbar, np.array([atoms[j]]), np.array([1.0]), np.array([0.7]), 0.3, cfg)
        ref = np.zeros(11)
        ref[j] = 1
        assert np.allclose(m[0], ref, atol=1e-15)
    big = synth.make_config("train_b512")
    for rv in (big["v_min"], 0.0, big["v_max"]):
        m = o.project_c51(_rand_dist(rng, 1, 101), np.array([rv]), np.array([1.0]), np.array([0.0]), 0.1, big)
        assert m[0].max() == pytest.approx(1.0, abs=1e-12)


def test_projection_preserves_clipped_mean():
    """sum_j m_j z_j = sum_i P_i clip(Tz_i) (linear splitting preserves the mean)."""
    cfg = synth.make_config("small_b32")
    rng = np.random.default_rng(15)
    pbar = _rand_dist(rng, 20, 51)
    r = rng.normal(size=20) * 4
    d = (rng.random(20) < 0.2).astype(float)
    logp = rng.normal(size=20)
    m = o.project_c51(pbar, r, d, logp, 0.5, cfg)
    z = o.support(cfg)
    tz = np.clip(r[:, None] + 0.99 * (1 - d[:, None]) * (z[None] - 0.5 * logp[:, None]), -10, 10)
    assert np.allclose((m * z).sum(1), (pbar * tz).sum(1), atol=1e-12)


def test_projection_is_linear_in_the_distribution():
    """Averaging two target critics then projecting = projecting each then averaging."""
    cfg = synth.make_config("small_b32")
    rng = np.random.default_rng(16)
    p1, p2 = _rand_dist(rng, 6, 51), _rand_dist(rng, 6, 51)
    r, d, lp = rng.normal(size=6), np.zeros(6), rng.normal(size=6)
    avg = o.project_c51(0.5 * (p1 + p2), r, d, lp, 0.1, cfg)
    sep = 0.5 * (o.project_c51(p1, r, d, lp, 0.1, cfg) + o.project_c51(p2, r, d, lp, 0.1, cfg))
    assert np.allclose(avg, sep, atol=1e-14)


def test_projection_gamma_zero_is_reward_alone():
    cfg = _cfg_tiny(gamma=0.0)
    rng = np.random.default_rng(17)
    pbar = _rand_dist(rng, 3, 11)
    m = o.project_c51(pbar, np.array([1.0, -3.0, 20.0]), np.zeros(3), np.ones(3), 0.5, cfg)
    assert np.allclose(m[0, 5], 0.5) and np.allclose(m[0, 6], 0.5)      # 1.0 halfway between 0 and 2
    assert np.allclose(m[1, 3], 0.5) and np.allclose(m[1, 4], 0.5)      # -3 between -4 and -2
    assert np.allclose(m[2, 10], 1.0)                                  # clipped to v_max


# ---------------------------------------------------------------- optimiser, polyak, init

def test_adam_first_step_closed_form():
    cfg = _cfg_tiny()
    g = np.array([1e-3, -2.0, 0.0, 5e-9])
    st = dict(params={"w": np.zeros(4)}, m={"w": np.zeros(4)}, v={"w": np.zeros(4)}, steps=dict(critic=0))
    o.adam_step(st, ["w"], {"w": g}, "critic", cfg)
    assert np.allclose(st["params"]["w"], -cfg["lr"] * g / (np.abs(g) + cfg["adam_eps"]), rtol=1e-12, atol=0)


def test_adam_constant_gradient_steps():
    """With a constant gradient every bias-corrected step is -lr g/(|g|+eps)."""
    cfg = _cfg_tiny()
    g = np.array([0.3, -0.7])
    st = dict(params={"w": np.zeros(2)}, m={"w": np.zeros(2)}, v={"w": np.zeros(2)}, steps=dict(critic=0))
    for _ in range(5):
        o.adam_step(st, ["w"], {"w": g}, "critic", cfg)
    assert np.allclose(st["params"]["w"], -5 * cfg["lr"] * g / (np.abs(g) + cfg["adam_eps"]), rtol=1e-10)


def test_polyak_closed_form():
    cfg = _cfg_tiny(tau=0.1)
    st = dict(params={"critic.w": np.array([2.0])}, target={"critic.w": np.array([-1.0])})
    for _ in range(7):
        o.polyak(st, cfg)
    rho = 0.9
    assert st["target"]["critic.w"][0] == pytest.approx(rho ** 7 * -1 + (1 - rho ** 7) * 2.0, abs=1e-14)


def test_init_bounds_and_layout():
    cfg = synth.make_config("small_b32")
    p = o.init_params(cfg)
    spec = o.param_spec(cfg)
    assert list(p) == [s[0] for s in spec]
    for name, shape, kind, fan in spec:
        v = p[name]
        assert v.shape == tuple(shape)
        assert np.array_equal(v, v.astype(np.float32).astype(np.float64))
        if kind == "U":
            bound = 1 / math.sqrt(fan)
            assert np.abs(v).max() <= bound
            if v.size > 2000:
                assert abs(v.var() - bound ** 2 / 3) < 0.1 * bound ** 2 / 3
    assert np.all(p["critic0.ln0.g"] == 1) and np.all(p["critic0.ln0.b"] == 0)
    assert p["log_alpha"][0] == pytest.approx(math.log(0.1), abs=1e-7)
    dm = o.dims(cfg)
    assert dm["feat"] == 16 * 5 * 5 and dm["critic_in"] == 418 and dm["actor_in"] == 412
    big = o.dims(synth.make_config("train_b512"))
    assert big["feat"] == 2592 and big["critic_in"] == 274 and big["actor_in"] == 268


# ---------------------------------------------------------------- whole-loss finite differences

def _tiny_setup(seed=0):
    cfg = _cfg_tiny()
    ring = synth.ring_numpy(synth.make_ring(cfg, seed))
    st = o.init_state(cfg)
    fe = o.frontend(cfg, ring, 0)
    return cfg, st, fe


def _check_tensor_fd(f, x, an, n_coords=6, h=1e-6, rng=None):
    """Central differences on a random subset of coordinates of x vs analytic `an`."""
    rng = rng or np.random.default_rng(0)
    flat = x.reshape(-1)
    anf = an.reshape(-1)
    picks = rng.choice(flat.size, size=min(n_coords, flat.size), replace=False)
    scale = max(np.abs(anf).max(), 1e-8)
    bad = []
    for i in picks:
        old = flat[i]
        flat[i] = old + h
        fp = f()
        flat[i] = old - h
        fm = f()
        flat[i] = old
        fd = (fp - fm) / (2 * h)
        if abs(fd - anf[i]) > 1e-6 * scale + 1e-9:
            bad.append((int(i), fd, anf[i]))
    return bad


def test_critic_loss_gradients_finite_differences():
    """Every gradient of the critic cross-entropy (critics, encoder) matches central differences."""
    cfg, st, fe = _tiny_setup()
    P = st["params"]
    z1, _ = o.encoder_fwd(P, fe["x_t1"], cfg)
    eps = px.normal_pairs(cfg["seed"], px.STREAM_EPS_TARGET, 0, cfg["batch"], 6)
    m = o.target_distribution(P, st["target"], z1, fe, 0.1, eps, cfg)["m"]      # stop-grad target
    res = o.critic_loss(P, fe["x_t"], fe, m, cfg)
    f = lambda: o.critic_loss(P, fe["x_t"], fe, m, cfg, with_grads=False)["loss"]
    rng = np.random.default_rng(1)
    for name, g in res["grads"].items():
        assert o.group_of(name) == "critic"
        assert not _check_tensor_fd(f, P[name], g, rng=rng), name
    assert set(res["grads"]) == {n for n, *_ in o.param_spec(cfg) if o.group_of(n) == "critic"}


def test_actor_loss_gradients_finite_differences():
    """Every gradient of the actor loss (through the frozen critics and log pi) matches central differences."""
    cfg, st, fe = _tiny_setup(1)
    P = st["params"]
    z, _ = o.encoder_fwd(P, fe["x_t"], cfg)
    eps = px.normal_pairs(cfg["seed"], px.STREAM_EPS_ACTOR, 0, cfg["batch"], 6)
    res = o.actor_loss(P, z, fe["p_t"], eps, 0.37, cfg)
    f = lambda: o.actor_loss(P, z, fe["p_t"], eps, 0.37, cfg, with_grads=False)["loss"]
    rng = np.random.default_rng(2)
    for name, g in res["grads"].items():
        assert o.group_of(name) == "actor"
        assert not _check_tensor_fd(f, P[name], g, rng=rng), name
    assert set(res["grads"]) == {n for n, *_ in o.param_spec(cfg) if o.group_of(n) == "actor"}


def _rows(d, lo, hi, B):
    """Rows lo:hi of every per-sample array of a front-end dict."""
    return {k: (v[lo:hi] if isinstance(v, np.ndarray) and v.ndim >= 1 and v.shape[0] == B else v)
            for k, v in d.items()}


@pytest.mark.parametrize("proj", [0, 16])
def test_losses_and_gradients_are_batch_means(proj):
    """Eq. 2 and Eq. 3 are expectations over the minibatch, estimated by the mean: on a
    split of the rows into parts of 3 and 5, the loss and every gradient of the whole
    batch are the size-weighted averages of the parts' (a sum in place of the mean, a
    wrong normaliser or rows mixed across samples all break this; finite differences
    alone would not see a normaliser shared by a loss and its gradient)."""
    cfg = synth.make_config("tiny_b8", proj_dim=proj)
    ring = synth.ring_numpy(synth.make_ring(cfg, 4))
    st = o.init_state(cfg)
    fe = o.frontend(cfg, ring, 0)
    P = st["params"]
    B = cfg["batch"]
    z1, _ = o.encoder_fwd(P, fe["x_t1"], cfg)
    eps_t = px.normal_pairs(cfg["seed"], px.STREAM_EPS_TARGET, 0, B, 6)
    m = o.target_distribution(P, st["target"], z1, fe, 0.1, eps_t, cfg)["m"]
    z, _ = o.encoder_fwd(P, fe["x_t"], cfg)
    eps_a = px.normal_pairs(cfg["seed"], px.STREAM_EPS_ACTOR, 0, B, 6)
    cut = 3

    def parts(loss_fn):
        whole = loss_fn(0, B)
        a, b = loss_fn(0, cut), loss_fn(cut, B)
        assert whole["loss"] == pytest.approx((cut * a["loss"] + (B - cut) * b["loss"]) / B, rel=1e-12, abs=1e-14)
        assert set(whole["grads"]) == set(a["grads"]) == set(b["grads"])
        for name, g in whole["grads"].items():
            avg = (cut * a["grads"][name] + (B - cut) * b["grads"][name]) / B
            assert np.allclose(g, avg, rtol=1e-10, atol=1e-14 * max(1.0, np.abs(g).max())), name

    parts(lambda lo, hi: o.critic_loss(P, fe["x_t"][lo:hi], _rows(fe, lo, hi, B), m[lo:hi], cfg))
    parts(lambda lo, hi: o.actor_loss(P, z[lo:hi], fe["p_t"][lo:hi], eps_a[lo:hi], 0.37, cfg))


@pytest.mark.parametrize("proj", [0, 16])
def test_target_reads_target_critics_and_the_online_actor(proj):
    """Alg. 1 "compute target": a' comes from the current actor and the distribution from
    the target critics (and target critic projection).  Perturbing the online critics
    leaves m unchanged; perturbing the target critics or the online actor changes it."""
    cfg = synth.make_config("tiny_b8", proj_dim=proj)
    ring = synth.ring_numpy(synth.make_ring(cfg, 5))
    st = o.init_state(cfg)
    fe = o.frontend(cfg, ring, 0)
    P, T = st["params"], st["target"]
    B = cfg["batch"]
    z1, _ = o.encoder_fwd(P, fe["x_t1"], cfg)
    eps = px.normal_pairs(cfg["seed"], px.STREAM_EPS_TARGET, 0, B, 6)
    m0 = o.target_distribution(P, T, z1, fe, 0.1, eps, cfg)["m"]
    rng = np.random.default_rng(6)

    def bumped(d, pred):
        out = dict(d)
        for k in d:
            if pred(k):
                out[k] = d[k] + 0.3 * rng.standard_normal(d[k].shape)
        return out

    crit = lambda k: k.startswith("critic")
    P_on = bumped(P, crit)                                   # online critics (and projection) moved
    assert np.array_equal(o.target_distribution(P_on, T, z1, fe, 0.1, eps, cfg)["m"], m0)
    T_moved = bumped(T, lambda k: True)                      # target critics moved
    assert np.abs(o.target_distribution(P, T_moved, z1, fe, 0.1, eps, cfg)["m"] - m0).max() > 1e-3
    P_act = bumped(P, lambda k: k.startswith("actor"))       # online actor moved: a', log pi' change
    assert np.abs(o.target_distribution(P_act, T, z1, fe, 0.1, eps, cfg)["m"] - m0).max() > 1e-3


def test_projection_heads_finite_differences():
    """With a projection layer (train-shape heads on a tiny body), projection grads match FD."""
    cfg = synth.make_config("tiny_b8", proj_dim=16)
    ring = synth.ring_numpy(synth.make_ring(cfg, 3))
    st = o.init_state(cfg)
    fe = o.frontend(cfg, ring, 0)
    P = st["params"]
    z1, _ = o.encoder_fwd(P, fe["x_t1"], cfg)
    eps = px.normal_pairs(0, px.STREAM_EPS_TARGET, 0, 8, 6)
    m = o.target_distribution(P, st["target"], z1, fe, 0.1, eps, cfg)["m"]
    res = o.critic_loss(P, fe["x_t"], fe, m, cfg)
    f = lambda: o.critic_loss(P, fe["x_t"], fe, m, cfg, with_grads=False)["loss"]
    rng = np.random.default_rng(3)
    for name in ("critic.proj.w", "critic.proj.b", "critic.proj.ln.g", "critic.proj.ln.b", "enc.conv0.w"):
        assert not _check_tensor_fd(f, P[name], res["grads"][name], rng=rng), name
    z, _ = o.encoder_fwd(P, fe["x_t"], cfg)
    ra = o.actor_loss(P, z, fe["p_t"], eps, 0.2, cfg)
    fa = lambda: o.actor_loss(P, z, fe["p_t"], eps, 0.2, cfg, with_grads=False)["loss"]
    for name in ("actor.proj.w", "actor.proj.ln.g", "actor.fc0.w"):
        assert not _check_tensor_fd(fa, P[name], ra["grads"][name], rng=rng), name


def test_alpha_gradient_finite_difference():
    cfg = _cfg_tiny()
    logp = np.array([-3.0, 1.0, 0.5])
    la = math.log(0.2)
    _, g = o.alpha_loss(la, logp, cfg)
    h = 1e-6
    fd = (o.alpha_loss(la + h, logp, cfg)[0] - o.alpha_loss(la - h, logp, cfg)[0]) / (2 * h)
    assert g == pytest.approx(fd, rel=1e-8)
    # entropy below target (log pi large) -> alpha must grow: gradient negative
    _, g_low = o.alpha_loss(la, np.array([10.0, 10.0]), cfg)
    assert g_low < 0


# ---------------------------------------------------------------- whole update structure

def test_update_zero_lr_keeps_parameters_and_moves_targets_only_by_polyak():
    cfg = _cfg_tiny(lr=0.0)
    ring = synth.ring_numpy(synth.make_ring(cfg, 0))
    st = o.init_state(cfg)
    p0 = {k: v.copy() for k, v in st["params"].items()}
    o.update(st, ring, cfg)
    for k in p0:
        assert np.array_equal(st["params"][k], p0[k])
    for k in st["target"]:
        assert np.allclose(st["target"][k], p0[k], atol=1e-15)


def test_update_targets_follow_polyak_of_updated_critics():
    cfg = _cfg_tiny()
    ring = synth.ring_numpy(synth.make_ring(cfg, 0))
    st = o.init_state(cfg)
    t0 = {k: v.copy() for k, v in st["target"].items()}
    o.update(st, ring, cfg)
    for k in t0:
        assert np.allclose(st["target"][k], 0.995 * t0[k] + 0.005 * st["params"][k], atol=1e-15)
    assert st["steps"] == dict(critic=1, actor=1, alpha=1) and st["update_idx"] == 1


def test_actor_step_reads_updated_critics_and_new_alpha():
    """Alg. 1 order: the critics take their step first, then the temperature, then the
    actor, whose objective reads the updated critics and the new alpha (and the
    pre-update encoder features, detached).  Its loss recomputed from the parameters
    in that state is the update's; with the pre-update critics or alpha it differs."""
    import copy
    cfg = _cfg_tiny()
    ring = synth.ring_numpy(synth.make_ring(cfg, 7))
    st = o.init_state(cfg)
    before = copy.deepcopy(st)
    stats, tr = o.update(st, ring, cfg)
    mixed = dict(before["params"])
    for name, *_ in o.param_spec(cfg):
        if o.group_of(name) == "critic":
            mixed[name] = st["params"][name]
    args = (tr["critic"]["z"], tr["frontend"]["p_t"], tr["eps_actor"])
    got = o.actor_loss(mixed, *args, stats["alpha"], cfg, with_grads=False)["loss"]
    assert got == stats["actor_loss"]
    stale_critics = o.actor_loss(before["params"], *args, stats["alpha"], cfg, with_grads=False)["loss"]
    stale_alpha = o.actor_loss(mixed, *args, tr["alpha_before"], cfg, with_grads=False)["loss"]
    assert abs(stale_critics - got) > 1e-9 and abs(stale_alpha - got) > 1e-9


def test_temperature_step_reads_the_pre_update_actor():
    """Alg. 1 "update entropy temperature": the temperature loss takes log pi of the actor
    before its step, at s_t with the actor's noise draws; the reported entropy is
    -mean(log pi); the first Adam step moves log alpha by lr against the sign of the
    gradient (|m_hat| / sqrt(v_hat) = 1 at t = 1)."""
    import copy
    cfg = _cfg_tiny()
    ring = synth.ring_numpy(synth.make_ring(cfg, 8))
    st = o.init_state(cfg)
    before = copy.deepcopy(st)
    stats, tr = o.update(st, ring, cfg)
    _, logp, _ = o.actor_fwd(before["params"], tr["critic"]["z"], tr["frontend"]["p_t"], tr["eps_actor"], cfg)
    la0 = float(before["params"]["log_alpha"][0])
    loss, grad = o.alpha_loss(la0, logp, cfg)
    assert stats["alpha_loss"] == loss
    assert stats["entropy"] == pytest.approx(-float(np.mean(logp)), rel=1e-15)
    la1 = float(st["params"]["log_alpha"][0])
    step = cfg["lr"] * abs(grad) / (abs(grad) + cfg["adam_eps"])
    assert la1 == pytest.approx(la0 - math.copysign(step, grad), rel=0, abs=1e-15)
    assert stats["alpha"] == pytest.approx(math.exp(la1), rel=1e-15)
    # the actor after its step gives another log pi (the temperature did not read it)
    _, logp_after, _ = o.actor_fwd(st["params"], tr["critic"]["z"], tr["frontend"]["p_t"], tr["eps_actor"], cfg)
    assert np.abs(logp_after - logp).max() > 1e-9


def test_policy_freq_delays_actor():
    cfg = _cfg_tiny(policy_freq=2)
    ring = synth.ring_numpy(synth.make_ring(cfg, 0))
    st = o.init_state(cfg)
    a0 = st["params"]["actor.fc0.w"].copy()
    s1, _ = o.update(st, ring, cfg)
    assert np.array_equal(st["params"]["actor.fc0.w"], a0) and math.isnan(s1["actor_loss"])
    s2, _ = o.update(st, ring, cfg)
    assert not np.array_equal(st["params"]["actor.fc0.w"], a0) and not math.isnan(s2["actor_loss"])
    assert st["steps"] == dict(critic=2, actor=1, alpha=2)


def test_act_is_row_independent_and_mean_mode_is_tanh_mu():
    cfg = _cfg_tiny()
    P = o.init_params(cfg)
    obs, prop = synth.make_obs_batch(5, cfg, 9)
    obs, prop = obs.numpy(), prop.numpy()
    full = o.act(P, obs, prop, 1234, True, cfg)
    part = o.act(P, obs[:3], prop[:3], 1234, True, cfg)
    assert np.allclose(full[:3], part, atol=1e-14)
    mean = o.act(P, obs, prop, 1234, False, cfg)
    assert np.all(np.abs(mean) < 1) and not np.allclose(mean, full)


# ---------------------------------------------------------------- squint at insert
def test_squint_store_brute_force_and_rounding():
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, size=(3, 2, 12, 8), dtype=np.uint8)
    f = 4
    q = o.squint_store(img, f)
    assert q.dtype == np.uint8 and q.shape == (3, 2, 3, 2)
    for n in range(3):
        for c in range(2):
            for i in range(3):
                for j in range(2):
                    s_ = int(img[n, c, i * f:(i + 1) * f, j * f:(j + 1) * f].astype(np.int64).sum())
                    mean = s_ / (f * f)
                    want = int(np.floor(mean + 0.5))          # round half up
                    assert q[n, c, i, j] == want
                    assert abs(q[n, c, i, j] / 255.0 - mean / 255.0) <= 0.5 / 255 + 1e-15


def test_squint_store_special_cases():
    # constant frames are unchanged; f = 1 is the identity; a half-way mean rounds up
    const = np.full((1, 3, 16, 16), 77, dtype=np.uint8)
    assert (o.squint_store(const, 4) == 77).all()
    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, size=(2, 3, 5, 7), dtype=np.uint8)
    assert np.array_equal(o.squint_store(img, 1), img)
    half = np.zeros((1, 1, 2, 2), dtype=np.uint8)
    half[0, 0, 0, :] = 1                        # sum 2 over 4 pixels: mean 0.5 -> 1
    assert o.squint_store(half, 2)[0, 0, 0, 0] == 1
    # the stored value is within half a level of the update's unrounded squint value
    img = rng.integers(0, 256, size=(4, 3, 32, 32), dtype=np.uint8)
    sums = o.shift_squint_sums(img, np.full(4, 0), np.full(4, 0), 0, 4)
    x_unrounded = o.squint_values(sums, 4)
    x_stored = o.squint_store(img, 4).astype(np.float64) / 255.0 - 0.5
    assert np.abs(x_unrounded - x_stored).max() <= 0.5 / 255 + 1e-12


# ---------------------------------------------------------------- critic variants (Sec. IV, Eq. 1-2)
VARIANTS = [dict(critic="mse"), dict(cdq=True), dict(critic="mse", cdq=True)]


def _variant_setup(seed, **kw):
    cfg = _cfg_tiny(**kw)
    ring = synth.ring_numpy(synth.make_ring(cfg, seed))
    st = o.init_state(cfg)
    return cfg, st, o.frontend(cfg, ring, 0)


@pytest.mark.parametrize("var", VARIANTS)
def test_variant_critic_and_actor_gradients_finite_differences(var):
    cfg, st, fe = _variant_setup(4, **var)
    P = st["params"]
    z1, _ = o.encoder_fwd(P, fe["x_t1"], cfg)
    eps = px.normal_pairs(cfg["seed"], px.STREAM_EPS_TARGET, 0, cfg["batch"], 6)
    m = o.target_distribution(P, st["target"], z1, fe, 0.1, eps, cfg)["m"]
    res = o.critic_loss(P, fe["x_t"], fe, m, cfg)
    f = lambda: o.critic_loss(P, fe["x_t"], fe, m, cfg, with_grads=False)["loss"]
    rng = np.random.default_rng(5)
    for name, g in res["grads"].items():
        assert not _check_tensor_fd(f, P[name], g, rng=rng), (var, name)
    z, _ = o.encoder_fwd(P, fe["x_t"], cfg)
    epa = px.normal_pairs(cfg["seed"], px.STREAM_EPS_ACTOR, 0, cfg["batch"], 6)
    ra = o.actor_loss(P, z, fe["p_t"], epa, 0.3, cfg)
    fa = lambda: o.actor_loss(P, z, fe["p_t"], epa, 0.3, cfg, with_grads=False)["loss"]
    for name, g in ra["grads"].items():
        assert not _check_tensor_fd(fa, P[name], g, rng=rng), (var, name)


def test_mse_critic_shapes_target_and_loss():
    cfg, st, fe = _variant_setup(6, critic="mse")
    P = st["params"]
    assert P["critic0.fc2.w"].shape == (1, 32)
    z1, _ = o.encoder_fwd(P, fe["x_t1"], cfg)
    eps = px.normal_pairs(cfg["seed"], px.STREAM_EPS_TARGET, 0, cfg["batch"], 6)
    tgt = o.target_distribution(P, st["target"], z1, fe, 0.25, eps, cfg)
    # Eq. 1 written out: average of the two target critics' Q, soft term on log pi'
    qbar = tgt["logits_target"][..., 0].mean(0)
    y = fe["r"] + cfg["gamma"] * (1 - fe["d"]) * (qbar - 0.25 * tgt["logp_next"])
    assert np.allclose(tgt["m"][:, 0], y, rtol=0, atol=1e-12)
    # gamma = 0: the target is the reward; a critic output equal to y has zero loss
    cfg0 = dict(cfg, gamma=0.0)
    y0 = o.target_distribution(P, st["target"], z1, fe, 0.25, eps, cfg0)["m"]
    assert np.array_equal(y0[:, 0], fe["r"])
    res = o.critic_loss(P, fe["x_t"], fe, y0, cfg0, with_grads=False)
    q = res["logits"][..., 0]
    assert res["loss"] == pytest.approx(float(((q - fe["r"][None]) ** 2).mean(1).sum()), rel=1e-12)


def test_clipped_double_q_selects_the_smaller_critic():
    cfg, st, fe = _variant_setup(7, cdq=True)
    P, T = st["params"], st["target"]
    z1, _ = o.encoder_fwd(P, fe["x_t1"], cfg)
    eps = px.normal_pairs(cfg["seed"], px.STREAM_EPS_TARGET, 0, cfg["batch"], 6)
    # identical target critics: clipped double Q equals the average exactly
    T2 = {k: v.copy() for k, v in T.items()}
    for k in list(T2):
        if k.startswith("critic1."):
            T2[k] = T2["critic0." + k[len("critic1."):]].copy()
    a = o.target_distribution(P, T2, z1, fe, 0.1, eps, cfg)["m"]
    b = o.target_distribution(P, T2, z1, fe, 0.1, eps, dict(cfg, cdq=False))["m"]
    assert np.allclose(a, b, rtol=0, atol=1e-15)
    # otherwise each sample takes the distribution of the critic with the smaller mean
    tgt = o.target_distribution(P, T, z1, fe, 0.1, eps, cfg)
    q = o.q_values(tgt["logits_target"], cfg)
    lo = np.argmin(q, axis=0)
    want = o.softmax(tgt["logits_target"])[lo, np.arange(q.shape[1])]
    assert np.allclose(tgt["pbar"], want, rtol=0, atol=1e-15)
    assert (q.min(0) <= q.mean(0) + 1e-15).all()


@pytest.mark.parametrize("name", ["tiny_b8", "train_b512"])
def test_q_value_is_the_mean_of_the_categorical_distribution(name):
    """Q = sum_j p_j z_j over the support of K atoms evenly spaced on [v_min, v_max]:
    equal logits give the midpoint, a dominant logit the value of its atom, a constant
    added to every logit changes nothing, and random logits match a plain loop."""
    cfg = synth.make_config(name)
    K, lo, hi = cfg["atoms"], cfg["v_min"], cfg["v_max"]
    z = o.support(cfg)
    assert z[0] == lo and z[-1] == hi and np.allclose(np.diff(z), (hi - lo) / (K - 1), rtol=0, atol=1e-12)
    assert o.q_values(np.zeros((1, 3, K)), cfg) == pytest.approx(0.5 * (lo + hi), abs=1e-12)
    for j in (0, K // 3, K - 1):
        lg = np.zeros((1, 1, K))
        lg[0, 0, j] = 60.0
        assert o.q_values(lg, cfg)[0, 0] == pytest.approx(lo + j * (hi - lo) / (K - 1), abs=1e-12)
    rng = np.random.default_rng(23)
    lg = rng.normal(size=(2, 5, K)) * 3
    q = o.q_values(lg, cfg)
    assert np.allclose(o.q_values(lg + 7.5, cfg), q, rtol=0, atol=1e-12)
    for e in range(2):
        for b in range(5):
            w = [math.exp(v) for v in lg[e, b]]
            tot = sum(w)
            ref = sum(wi / tot * (lo + i * (hi - lo) / (K - 1)) for i, wi in enumerate(w))
            assert q[e, b] == pytest.approx(ref, abs=1e-11)


# ---------------------------------------------------------------- state-based SAC (Fig. 6 left)

def _state_pair(seed=0):
    """A tiny visual config and its state-based twin (same heads, no encoder), on one ring."""
    vis = _cfg_tiny()
    st = _cfg_tiny(conv_layers=0, conv_ch=0, obs_c=0, obs_h=0, obs_w=0, squint_f=1, shift_pad=0)
    ring_v = synth.ring_numpy(synth.make_ring(vis, seed))
    ring_s = {k: v for k, v in ring_v.items() if k != "obs"}
    return vis, st, ring_v, ring_s


def _silent_encoder_params(P_state, vis, rng):
    """Visual parameters whose encoder outputs exactly zero features (zero conv weights and
    biases, so every ReLU sees 0), with the state parameters in the heads' state/action
    columns and arbitrary values in the feature columns of each head's first layer."""
    feat = o.dims(vis)["feat"]
    P = {}
    for name, shape, *_ in o.param_spec(vis):
        if name.startswith("enc."):
            P[name] = np.zeros(shape)
        elif name.endswith("fc0.w"):
            w = rng.standard_normal(shape)
            w[:, feat:] = P_state[name]
            P[name] = w
        else:
            P[name] = P_state[name].copy()
    return P


def test_state_based_layout_and_gather():
    vis, st, _, ring_s = _state_pair()
    dm = o.dims(st)
    assert dm["feat"] == 0 and dm["zdim"] == 0 and dm["conv"] == []
    assert dm["critic_in"] == st["proprio_dim"] + st["action_dim"] and dm["actor_in"] == st["proprio_dim"]
    names = [n for n, *_ in o.param_spec(st)]
    assert not any(n.startswith("enc.") for n in names)
    assert {n for n, *_ in o.param_spec(vis) if not n.startswith("enc.")} == set(names)
    fe = o.frontend(st, ring_s, 3)
    assert fe["x_t"].shape == (st["batch"], 0) and fe["x_t1"].shape == (st["batch"], 0)
    n = ring_s["proprio"].shape[0]
    for b in range(st["batch"]):                      # row b is slot idx[b]; its next state is slot idx[b] + 1
        i = int(fe["idx"][b])
        assert fe["nxt"][b] == (i + 1) % n
        assert np.array_equal(fe["p_t"][b], ring_s["proprio"][i])
        assert np.array_equal(fe["p_t1"][b], ring_s["proprio"][(i + 1) % n])
        assert np.array_equal(fe["a_t"][b], ring_s["action"][i])
        assert fe["r"][b] == ring_s["reward"][i] and fe["d"][b] == ring_s["done"][i]


def test_state_based_update_equals_visual_update_with_a_silent_encoder():
    """Removing the encoder is the same as an encoder whose features are identically zero:
    two updates of the state-based config and of the visual config with a silent encoder give
    the same losses and the same head parameters; the feature columns and the encoder get no
    gradient and do not move."""
    vis, st, ring_v, ring_s = _state_pair(2)
    Ps = o.init_params(st)
    Pv = _silent_encoder_params(Ps, vis, np.random.default_rng(3))
    feat = o.dims(vis)["feat"]
    Sv = o.init_state(vis, params={k: v.copy() for k, v in Pv.items()})
    Ss = o.init_state(st, params={k: v.copy() for k, v in Ps.items()})
    for _ in range(2):
        a, tv = o.update(Sv, ring_v, vis)
        b, ts = o.update(Ss, ring_s, st)
        for k in a:
            assert a[k] == pytest.approx(b[k], rel=1e-12, abs=1e-12), k
        for name, g in tv["critic"]["grads"].items():
            if name.startswith("enc."):
                assert not np.any(g), name
            elif name.endswith("fc0.w"):
                assert not np.any(g[:, :feat]), name
    for name, v in Ss["params"].items():
        w = Sv["params"][name]
        if name.endswith("fc0.w"):
            assert np.array_equal(w[:, :feat], Pv[name][:, :feat]), name
            w = w[:, feat:]
        assert np.allclose(w, v, rtol=0, atol=1e-12), name
    for name, v in Sv["params"].items():
        if name.startswith("enc."):
            assert not np.any(v), name


def test_state_based_loss_gradients_finite_differences():
    _, st, _, ring_s = _state_pair(5)
    S = o.init_state(st)
    P = S["params"]
    fe = o.frontend(st, ring_s, 0)
    z1, _ = o.encoder_fwd(P, fe["x_t1"], st)
    eps = px.normal_pairs(st["seed"], px.STREAM_EPS_TARGET, 0, st["batch"], 6)
    m = o.target_distribution(P, S["target"], z1, fe, 0.1, eps, st)["m"]
    res = o.critic_loss(P, fe["x_t"], fe, m, st)
    f = lambda: o.critic_loss(P, fe["x_t"], fe, m, st, with_grads=False)["loss"]
    rng = np.random.default_rng(6)
    assert set(res["grads"]) == {n for n, *_ in o.param_spec(st) if o.group_of(n) == "critic"}
    for name, g in res["grads"].items():
        assert not _check_tensor_fd(f, P[name], g, rng=rng), name
    z, _ = o.encoder_fwd(P, fe["x_t"], st)
    epa = px.normal_pairs(st["seed"], px.STREAM_EPS_ACTOR, 0, st["batch"], 6)
    ra = o.actor_loss(P, z, fe["p_t"], epa, 0.3, st)
    fa = lambda: o.actor_loss(P, z, fe["p_t"], epa, 0.3, st, with_grads=False)["loss"]
    for name, g in ra["grads"].items():
        assert not _check_tensor_fd(fa, P[name], g, rng=rng), name


def test_state_based_act_equals_visual_act_with_a_silent_encoder():
    vis, st, _, _ = _state_pair()
    Ps = o.init_params(st)
    Pv = _silent_encoder_params(Ps, vis, np.random.default_rng(8))
    obs, prop = synth.make_obs_batch(5, vis, 9)
    obs, prop = obs.numpy(), prop.numpy()
    for sample in (True, False):
        a = o.act(Ps, None, prop, 77, sample, st)
        b = o.act(Pv, obs, prop, 77, sample, vis)
        assert np.allclose(a, b, rtol=0, atol=1e-13)
