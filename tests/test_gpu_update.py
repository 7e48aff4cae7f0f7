"""CUDA update path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (FP32 path): integer steps (slots, shifts, box sums) bit-exact;
losses, Q-mean, temperature 1e-4 relative; every gradient tensor 1e-3 relative
in norm; the parameter change of one update 1e-3 relative in norm per group.
"""
import math

import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import flatten, lazy_ring, post_critic_state, rel_err, ring_to_device, split_params

pytestmark = pytest.mark.gpu

LOSS_RTOL = 1e-4
GRAD_RTOL = 1e-3


@pytest.fixture(scope="module")
def L():
    from paper_2602_21203_gb300 import lib
    return lib


def _setup(L, name, seed=0, **over):
    cfg = synth.make_config(name, **over)
    ring_cpu = synth.make_ring(cfg, seed)
    ring = ring_to_device(ring_cpu)
    learner = L.Learner(cfg, ring)
    return cfg, ring_cpu, ring, learner


def _close(a, b, rtol, atol=0.0):
    return abs(a - b) <= rtol * abs(b) + atol


@pytest.mark.parametrize("name", ["small_b32", "train_b512", "tiny_b8"])
def test_initial_parameters_match_oracle_bitwise(L, name):
    cfg = synth.make_config(name)
    learner = L.Learner(cfg, None)
    got = learner.params()
    ref = flatten(o.init_params(cfg), cfg).astype(np.float32)
    assert np.array_equal(got, ref)
    learner.close()


@pytest.mark.parametrize("name,over", [("small_b32", {}), ("tiny_b8", {}),
                                       ("train_b512", dict(ring_size=300, batch=64))])
def test_frontend_is_bit_exact(L, name, over):
    """Slots, shifts, box sums and images of the front end equal the oracle's; the last
    case has the training frames (3 x 128 x 128, pad 8, squint 4 to 32 x 32)."""
    cfg, ring_cpu, ring, learner = _setup(L, name, **over)
    for u in range(2):
        learner.update(1, graph=False)
        fe = o.frontend(cfg, synth.ring_numpy(ring_cpu), u)
        assert np.array_equal(learner.debug("idx", np.int32), fe["idx"])
        assert np.array_equal(learner.debug("nxt", np.int32), fe["nxt"])
        assert np.array_equal(learner.debug("shift_t", np.int32).reshape(-1, 2), fe["shift_t"])
        assert np.array_equal(learner.debug("shift_t1", np.int32).reshape(-1, 2), fe["shift_t1"])
        assert np.array_equal(learner.debug("sums_t", np.uint16).reshape(fe["sums_t"].shape), fe["sums_t"])
        assert np.array_equal(learner.debug("sums_t1", np.uint16).reshape(fe["sums_t1"].shape), fe["sums_t1"])
        x = learner.debug("x_t").reshape(fe["x_t"].shape)
        assert np.abs(x - fe["x_t"]).max() < 1e-6
    learner.close()


@pytest.mark.parametrize("graph", [False, True])
def test_frontend_drawn_ahead_is_bit_exact(L, graph):
    """In a call of k updates, update j + 1's minibatch is drawn while update j runs, into
    the other of two buffer sets: the last update's draws and images are still those of
    its own update index, across calls of odd and even k."""
    cfg, ring_cpu, ring, learner = _setup(L, "small_b32")
    ring_np = synth.ring_numpy(ring_cpu)
    u = 0
    for k in (3, 2, 4):
        stats = learner.update(k, graph=graph)
        u += k
        assert [s["update_idx"] for s in stats] == list(range(u - k, u))
        fe = o.frontend(cfg, ring_np, u - 1)
        assert np.array_equal(learner.debug("idx", np.int32), fe["idx"])
        assert np.array_equal(learner.debug("nxt", np.int32), fe["nxt"])
        assert np.array_equal(learner.debug("shift_t", np.int32).reshape(-1, 2), fe["shift_t"])
        assert np.array_equal(learner.debug("shift_t1", np.int32).reshape(-1, 2), fe["shift_t1"])
        if not graph:   # box sums are kept in eager (debug) updates only
            assert np.array_equal(learner.debug("sums_t1", np.uint16).reshape(fe["sums_t1"].shape), fe["sums_t1"])
        x = learner.debug("x_t1").reshape(fe["x_t1"].shape)
        assert np.abs(x - fe["x_t1"]).max() < 1e-6
    learner.close()


def test_new_ring_after_a_capture_is_read(L):
    """set_replay with another ring after a graph was captured: the next replay of the same
    k reads the new ring (its images equal the oracle's front end on the new contents)."""
    cfg, ring_cpu, ring, learner = _setup(L, "small_b32")
    learner.update(2, graph=True)
    ring_cpu_b = synth.make_ring(cfg, 1)           # other contents, same size
    ring_b = ring_to_device(ring_cpu_b)
    learner.set_replay(ring_b)
    stats = learner.update(2, graph=True)
    assert [s["update_idx"] for s in stats] == [2, 3]
    fe = o.frontend(cfg, synth.ring_numpy(ring_cpu_b), 3)
    assert np.array_equal(learner.debug("idx", np.int32), fe["idx"])
    x = learner.debug("x_t1").reshape(fe["x_t1"].shape)
    assert np.abs(x - fe["x_t1"]).max() < 1e-6
    learner.close()


def _check_update(cfg, learner, state, ring_np, graph):
    p_before = learner.params().astype(np.float64)
    stats = learner.update(1, graph=graph)[0]
    ref, tr = o.update(state, ring_np, cfg)
    for key in ("critic_loss", "alpha_loss", "alpha", "entropy", "actor_loss"):
        assert _close(stats[key], ref[key], LOSS_RTOL, 1e-6), (key, stats[key], ref[key])
    assert _close(stats["q_mean"], ref["q_mean"], LOSS_RTOL, 1e-5), (stats["q_mean"], ref["q_mean"])
    return stats, ref, tr, p_before


@pytest.mark.parametrize("name", ["small_b32", "tiny_b8"])
def test_one_update_matches_oracle(L, name):
    cfg, ring_cpu, ring, learner = _setup(L, name)
    ring_np = synth.ring_numpy(ring_cpu)
    state = o.init_state(cfg)
    stats, ref, tr, p_before = _check_update(cfg, learner, state, ring_np, graph=False)
    # projected target distribution and critic logits
    K = cfg["atoms"]
    m = learner.debug("m").reshape(-1, K)
    assert np.abs(m - tr["target"]["m"]).max() < 1e-5
    assert np.allclose(m.sum(1), 1.0, atol=1e-5)
    logits = learner.debug("logits").reshape(2, -1, K)
    assert rel_err(logits, tr["critic"]["logits"]) < 1e-5
    # every gradient tensor
    g = split_params(learner.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    for k, v in ref_grads.items():
        assert rel_err(g[k], v) < GRAD_RTOL, (k, rel_err(g[k], v))
    # parameter change of the update, per optimiser group
    p_after = learner.params().astype(np.float64)
    ref_after = flatten(state["params"], cfg)
    for grp in ("critic", "actor", "alpha"):
        sel = np.concatenate([np.full(int(np.prod(s)), o.group_of(nm) == grp) for nm, s, _, _ in o.param_spec(cfg)])
        d_gpu = p_after[sel] - p_before[sel]
        d_ref = ref_after[sel] - p_before[sel]
        assert rel_err(d_gpu, d_ref) < 1e-3, (grp, rel_err(d_gpu, d_ref))
    tgt = learner.debug("target")
    ref_t = np.concatenate([state["target"][nm].ravel() for nm, *_ in o.param_spec(cfg) if o.is_target(nm)])
    assert np.abs(tgt - ref_t).max() < 1e-5
    learner.close()


def test_graph_replay_equals_eager_bitwise(L):
    cfg, ring_cpu, ring, a = _setup(L, "small_b32")
    b = L.Learner(cfg, ring)
    sa = a.update(3, graph=True)
    sb = b.update(3, graph=False)
    assert np.array_equal(a.params(), b.params())
    assert sa == sb
    sa = a.update(3, graph=True)      # replay of the captured graph
    sb = b.update(3, graph=False)
    assert np.array_equal(a.params(), b.params())
    assert np.array_equal(a.debug("target"), b.debug("target"))
    assert [s["update_idx"] for s in sa] == [3, 4, 5]
    a.close()
    b.close()


def test_async_update_statistics_equal_the_waiting_call(L):
    """squint_update_async leaves the statistics to the stream: once it is synchronised,
    the caller's page-locked buffer holds what squint_update returns for a twin learner,
    bit for bit, over calls that reuse the buffer; the parameters agree too.  Pageable
    host memory is refused, and squint_update_check reports no timed-out wait."""
    import ctypes
    cfg, ring_cpu, ring, a = _setup(L, "small_b32")
    b = L.Learner(cfg, ring)
    buf = L.PinnedStats(3)
    s = torch.cuda.Stream()
    for call in range(3):
        ref = a.update(3, stream=s)
        b.update_async(3, buf, stream=s)
        s.synchronize()
        assert buf.read() == ref, call
    b.update_check(stream=s)
    assert np.array_equal(a.params(), b.params())
    assert [x["update_idx"] for x in buf.read()] == [6, 7, 8]
    pageable = (L.UpdateStats * 3)()
    rc = b.lib.squint_update_async(b.h, 3, ctypes.cast(pageable, ctypes.c_void_p), ctypes.c_void_p(s.cuda_stream))
    assert rc == L.EINVAL
    b.update_async(3, None, stream=s)     # no statistics: nothing copied back
    b.update_check(stream=s)
    a.close()
    b.close()


def test_k_updates_track_oracle(L):
    cfg, ring_cpu, ring, learner = _setup(L, "small_b32")
    ring_np = synth.ring_numpy(ring_cpu)
    state = o.init_state(cfg)
    stats = learner.update(4, graph=True)
    for j in range(4):
        ref, _ = o.update(state, ring_np, cfg)
        for key in ("critic_loss", "alpha", "entropy", "actor_loss", "alpha_loss"):
            assert _close(stats[j][key], ref[key], 1e-3, 1e-5), (j, key, stats[j][key], ref[key])
    learner.close()


def test_policy_freq_two_delays_the_actor(L):
    cfg, ring_cpu, ring, learner = _setup(L, "tiny_b8", policy_freq=2)
    n0 = learner.params()
    spec = o.param_spec(cfg)
    sel = np.concatenate([np.full(int(np.prod(s)), o.group_of(nm) == "actor") for nm, s, _, _ in spec])
    s1 = learner.update(1, graph=True)[0]
    n1 = learner.params()
    assert np.array_equal(n0[sel], n1[sel]) and math.isnan(s1["actor_loss"])
    s2 = learner.update(1, graph=True)[0]
    n2 = learner.params()
    assert not np.array_equal(n1[sel], n2[sel]) and not math.isnan(s2["actor_loss"])
    learner.close()


def test_state_roundtrip_resumes_bitwise(L):
    cfg, ring_cpu, ring, a = _setup(L, "tiny_b8")
    a.update(2, graph=True)
    blob = a.state()
    b = L.Learner(cfg, ring)
    b.set_state(blob)
    sa = a.update(2, graph=True)
    sb = b.update(2, graph=True)
    assert sa == sb
    assert np.array_equal(a.params(), b.params())
    a.close()
    b.close()


def test_training_shape_update_matches_oracle(L):
    """Full size: 100k-slot 3x128x128 ring on the device, batch 512, 4 conv layers, 256-d heads."""
    cfg = synth.make_config("train_b512")
    ring = synth.make_ring(cfg, 0, device="cuda")
    learner = L.Learner(cfg, ring)
    state = o.init_state(cfg)
    lazy = lazy_ring(ring)
    stats = learner.update(1, graph=True)[0]
    ref, tr = o.update(state, lazy, cfg)
    for key in ("critic_loss", "alpha_loss", "alpha", "entropy", "actor_loss"):
        assert _close(stats[key], ref[key], LOSS_RTOL, 1e-6), (key, stats[key], ref[key])
    assert _close(stats["q_mean"], ref["q_mean"], LOSS_RTOL, 1e-5)
    g = split_params(learner.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    for k, v in ref_grads.items():
        assert rel_err(g[k], v) < GRAD_RTOL, (k, rel_err(g[k], v))
    # the UTD-4 graph of the timed configuration runs and stays finite
    more = learner.update(4, graph=True)
    assert all(math.isfinite(s["critic_loss"]) and math.isfinite(s["actor_loss"]) for s in more)
    assert [s["update_idx"] for s in more] == [1, 2, 3, 4]
    learner.close()
    del ring
    torch.cuda.empty_cache()


def test_errors_are_codes_not_crashes(L):
    cfg = synth.make_config("tiny_b8")
    learner = L.Learner(cfg, None)
    with pytest.raises(L.SquintError) as e:
        learner.update(1)
    assert e.value.code == L.ESTATE
    ring = ring_to_device(synth.make_ring(cfg, 0))
    learner.set_replay(ring)
    for k in (0, 99):
        with pytest.raises(L.SquintError) as e:
            learner.update(k)
        assert e.value.code == L.EINVAL
    learner.update(1)
    with pytest.raises(L.SquintError):
        learner.set_params(np.zeros(3, dtype=np.float32))
    learner.close()


# ---------------------------------------------------------------- BF16 tensor-core path
# Per-quantity bounds for BF16 operands with FP32 accumulation (relative, or absolute
# below 1 for the actor loss): Q-mean 2e-2, critic CE 1e-2, actor loss 3e-2,
# gradient norm 5e-2; gradients must also point the same way (cosine > 0.98).
BF16_BOUNDS = dict(q_mean=2e-2, critic_loss=1e-2, actor_loss=3e-2, grad_norm=5e-2)


def _bf16_close(key, got, ref):
    tol = BF16_BOUNDS[key]
    if key == "actor_loss" and abs(ref) < 1:
        return abs(got - ref) <= tol
    return abs(got - ref) <= tol * abs(ref) + 1e-6


@pytest.mark.parametrize("name", ["small_b32", "tiny_b8", "train_b512"])
def test_bf16_update_within_stated_bounds(L, name):
    cfg = synth.make_config(name)
    if name == "train_b512":
        ring = synth.make_ring(cfg, 0, device="cuda")
        ring_np = lazy_ring(ring)
    else:
        ring_cpu = synth.make_ring(cfg, 0)
        ring = ring_to_device(ring_cpu)
        ring_np = synth.ring_numpy(ring_cpu)
    learner = L.Learner(cfg, ring, precision=L.PREC_BF16)
    state = o.init_state(cfg)
    stats = learner.update(1, graph=True)[0]
    ref, tr = o.update(state, ring_np, cfg)
    for key in ("q_mean", "critic_loss", "actor_loss"):
        assert _bf16_close(key, stats[key], ref[key]), (key, stats[key], ref[key])
    g = split_params(learner.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    for k, v in ref_grads.items():
        n_got, n_ref = np.linalg.norm(g[k]), np.linalg.norm(v)
        assert abs(n_got - n_ref) <= BF16_BOUNDS["grad_norm"] * n_ref + 1e-7, (k, n_got, n_ref)
        cos = float((g[k].ravel() @ v.ravel()) / max(n_got * n_ref, 1e-30))
        assert cos > 0.98 or n_ref < 1e-6, (k, cos)
    more = learner.update(4, graph=True)
    assert all(np.isfinite([s["critic_loss"], s["actor_loss"], s["q_mean"]]).all() for s in more)
    learner.close()


def test_bf16_graph_equals_eager_bitwise(L):
    cfg = synth.make_config("small_b32")
    ring = ring_to_device(synth.make_ring(cfg, 0))
    a = L.Learner(cfg, ring, precision=L.PREC_BF16)
    b = L.Learner(cfg, ring, precision=L.PREC_BF16)
    sa = a.update(3, graph=True)
    sb = b.update(3, graph=False)
    assert sa == sb
    assert np.array_equal(a.params(), b.params())
    a.close()
    b.close()


@pytest.mark.parametrize("name,prec", [("small_b32", "BF16"), ("train_b512", "BF16"), ("train_b512", "MXFP8"),
                                       ("state_small_b64", "BF16")])
def test_optimiser_written_low_precision_weights_equal_a_fresh_cast(L, name, prec):
    """Adam and polyak write the BF16 weight copies the next update reads.  A learner that
    resumes from the same state casts its copies from the FP32 masters instead; the next
    updates of the two must agree bit for bit."""
    over = {"ring_size": 4096} if name == "train_b512" else {}
    cfg = synth.make_config(name, **over)
    ring = synth.make_ring(cfg, 0, device="cuda") if name == "train_b512" else ring_to_device(synth.make_ring(cfg, 0))
    p = getattr(L, "PREC_" + prec)
    a = L.Learner(cfg, ring, precision=p)
    a.update(3, graph=True)
    b = L.Learner(cfg, ring, precision=p)
    b.set_state(a.state())
    sa = a.update(2, graph=True)
    sb = b.update(2, graph=True)
    assert sa == sb
    assert np.array_equal(a.params(), b.params())
    assert np.array_equal(a.debug("target"), b.debug("target"))
    a.close()
    b.close()


def test_bf16_k_updates_track_oracle(L):
    """Four BF16 updates in one graph against four oracle updates: every update's losses
    within the per-update BF16 bounds (the later ones read the weights Adam wrote)."""
    cfg = synth.make_config("small_b32")
    ring_cpu = synth.make_ring(cfg, 0)
    ring = ring_to_device(ring_cpu)
    ring_np = synth.ring_numpy(ring_cpu)
    learner = L.Learner(cfg, ring, precision=L.PREC_BF16)
    state = o.init_state(cfg)
    stats = learner.update(4, graph=True)
    for j in range(4):
        ref, _ = o.update(state, ring_np, cfg)
        for key in ("q_mean", "critic_loss", "actor_loss"):
            assert _bf16_close(key, stats[j][key], ref[key]), (j, key, stats[j][key], ref[key])
    learner.close()


# ---------------------------------------------------------------- FP8 forward layers
def test_fp8_update_runs_and_replays_bitwise(L):
    """FP8 mode (e4m3 forward linear layers, per-tensor scales): graph == eager bit for
    bit, finite, and the first update's losses near the oracle's (printed)."""
    cfg = synth.make_config("train_b512", ring_size=4096)
    ring = synth.make_ring(cfg, 0, device="cuda")
    a = L.Learner(cfg, ring, precision=L.PREC_FP8)
    b = L.Learner(cfg, ring, precision=L.PREC_FP8)
    sa = a.update(3, graph=True)
    sb = b.update(3, graph=False)
    assert sa == sb
    assert np.array_equal(a.params(), b.params())
    assert all(np.isfinite([s["critic_loss"], s["actor_loss"], s["q_mean"]]).all() for s in sa)
    c = L.Learner(cfg, ring, precision=L.PREC_FP8)
    st = c.update(1, graph=False)[0]
    ref, _ = o.update(o.init_state(cfg), lazy_ring(ring), cfg)
    print("\nfp8 vs oracle:", {k: (st[k], ref[k]) for k in ("q_mean", "critic_loss", "actor_loss")})
    assert abs(st["critic_loss"] - ref["critic_loss"]) <= 5e-2 * abs(ref["critic_loss"])
    # the FP8 bounds of the precision sweep: Q-mean 1e-1 relative to max(|Q|, 1), actor
    # loss 3e-1 (absolute below 1)
    assert abs(st["q_mean"] - ref["q_mean"]) <= 1e-1 * max(abs(ref["q_mean"]), 1.0), (st["q_mean"], ref["q_mean"])
    assert abs(st["actor_loss"] - ref["actor_loss"]) <= 3e-1 * max(abs(ref["actor_loss"]), 1.0), \
        (st["actor_loss"], ref["actor_loss"])
    for x in (a, b, c):
        x.close()


def test_mxfp8_update_runs_and_replays_bitwise(L):
    """MX-FP8 mode (e4m3 forward linear layers with block scales): graph == eager bit for
    bit, finite, and the first update's losses near the oracle's (printed)."""
    cfg = synth.make_config("train_b512", ring_size=4096)
    ring = synth.make_ring(cfg, 0, device="cuda")
    a = L.Learner(cfg, ring, precision=L.PREC_MXFP8)
    b = L.Learner(cfg, ring, precision=L.PREC_MXFP8)
    sa = a.update(3, graph=True)
    sb = b.update(3, graph=False)
    assert sa == sb
    assert np.array_equal(a.params(), b.params())
    assert all(np.isfinite([s["critic_loss"], s["actor_loss"], s["q_mean"]]).all() for s in sa)
    c = L.Learner(cfg, ring, precision=L.PREC_MXFP8)
    st = c.update(1, graph=False)[0]
    ref, _ = o.update(o.init_state(cfg), lazy_ring(ring), cfg)
    print("\nmxfp8 vs oracle:", {k: (st[k], ref[k]) for k in ("q_mean", "critic_loss", "actor_loss")})
    assert abs(st["critic_loss"] - ref["critic_loss"]) <= 5e-2 * abs(ref["critic_loss"])
    # the FP8 bounds of the precision sweep: Q-mean 1e-1 relative to max(|Q|, 1), actor
    # loss 3e-1 (absolute below 1)
    assert abs(st["q_mean"] - ref["q_mean"]) <= 1e-1 * max(abs(ref["q_mean"]), 1.0), (st["q_mean"], ref["q_mean"])
    assert abs(st["actor_loss"] - ref["actor_loss"]) <= 3e-1 * max(abs(ref["actor_loss"]), 1.0), \
        (st["actor_loss"], ref["actor_loss"])
    for x in (a, b, c):
        x.close()


def test_fp8_with_fused_layernorm_matches_separate_layernorm(L, monkeypatch):
    """The LayerNorm fused into the FP8 GEMM epilogue takes its row statistics from the
    rescaled accumulator, like the separate LayerNorm kernel: same update up to rounding."""
    cfg = synth.make_config("train_b512", ring_size=4096)
    ring = synth.make_ring(cfg, 0, device="cuda")
    a = L.Learner(cfg, ring, precision=L.PREC_FP8)
    monkeypatch.setenv("SQUINT_FUSED_LN", "1")
    b = L.Learner(cfg, ring, precision=L.PREC_FP8)
    sa = a.update(1, graph=False)[0]
    sb = b.update(1, graph=False)[0]
    for k in ("critic_loss", "q_mean", "actor_loss", "entropy"):
        assert abs(sa[k] - sb[k]) <= 1e-3 * max(abs(sa[k]), 1.0), (k, sa[k], sb[k])
    ga, gb = a.debug("grads").astype(np.float64), b.debug("grads").astype(np.float64)
    assert float(ga @ gb) / (np.linalg.norm(ga) * np.linalg.norm(gb)) > 0.999
    a.close()
    b.close()


# ---------------------------------------------------------------- ragged batches
@pytest.mark.parametrize("prec", ["FP32", "BF16"])
@pytest.mark.parametrize("batch", [37, 500])
def test_ragged_batch_update_matches_oracle(L, batch, prec):
    """The training architecture (3x128x128 frames, 4 conv layers, 256-d heads, 512-512
    critics and actor) at batches that are no multiple of 8 or of a 128-row tile: the
    integer steps bit-exact; FP32 losses 1e-4 and gradients 1e-3 (the actor step and the
    first conv's weight gradient on the GPU's own post-critic-step state and first-layer
    gradient, as in the precision sweep); BF16 within the sweep's BF16 bounds."""
    cfg = synth.make_config("train_b512", ring_size=4096, batch=batch)
    ring = synth.make_ring(cfg, 0, device="cuda")
    lazy = lazy_ring(ring)
    learner = L.Learner(cfg, ring, precision=getattr(L, "PREC_" + prec), max_k=2)
    state = o.init_state(cfg)
    P0 = {k: v.copy() for k, v in state["params"].items()}
    stats = learner.update(1, graph=prec == "BF16")[0]
    ref, tr = o.update(state, lazy, cfg)
    fe = tr["frontend"]
    assert np.array_equal(learner.debug("idx", np.int32), fe["idx"])
    assert np.array_equal(learner.debug("shift_t", np.int32).reshape(-1, 2), fe["shift_t"])
    assert np.array_equal(learner.debug("shift_t1", np.int32).reshape(-1, 2), fe["shift_t1"])
    g = split_params(learner.debug("grads"), cfg)
    p_gpu = split_params(learner.params(), cfg)
    mix = post_critic_state(P0, p_gpu, cfg)
    act = o.actor_loss(mix, tr["critic"]["z"], fe["p_t"], tr["eps_actor"], math.exp(float(mix["log_alpha"][0])), cfg)
    if prec == "FP32":
        for key in ("critic_loss", "alpha_loss", "alpha", "entropy"):
            assert _close(stats[key], ref[key], LOSS_RTOL, 1e-6), (key, stats[key], ref[key])
        assert abs(stats["q_mean"] - ref["q_mean"]) <= LOSS_RTOL * max(abs(ref["q_mean"]), 1.0)
        assert abs(stats["actor_loss"] - act["loss"]) <= LOSS_RTOL * max(abs(act["loss"]), 1e-2), \
            (stats["actor_loss"], act["loss"], ref["actor_loss"])
        c0 = o.dims(cfg)["conv"][0]
        dy0 = learner.debug("dconv0").astype(np.float64).reshape(batch, c0["cout"], c0["oh"], c0["ow"])
        _, dw0, db0 = o.conv3x3_bwd(fe["x_t"], P0["enc.conv0.w"], dy0, c0["s"], need_dx=False)
        assert rel_err(g["enc.conv0.w"], dw0) < GRAD_RTOL and rel_err(g["enc.conv0.b"], db0) < GRAD_RTOL
        for k, v in tr["critic"]["grads"].items():
            if k != "enc.conv0.w":
                assert rel_err(g[k], v) < GRAD_RTOL, (k, rel_err(g[k], v))
        for k, v in act["grads"].items():
            assert rel_err(g[k], v) < GRAD_RTOL, (k, rel_err(g[k], v))
    else:
        assert abs(stats["q_mean"] - ref["q_mean"]) <= 2e-2 * max(abs(ref["q_mean"]), 1.0)
        assert abs(stats["critic_loss"] - ref["critic_loss"]) <= 1e-2 * abs(ref["critic_loss"])
        assert abs(stats["actor_loss"] - act["loss"]) <= 3e-2 * max(abs(act["loss"]), 1.0)
        ref_grads = dict(tr["critic"]["grads"])
        ref_grads.update(act["grads"])
        for k, v in ref_grads.items():
            n_got, n_ref = np.linalg.norm(g[k]), np.linalg.norm(v)
            assert abs(n_got - n_ref) <= 5e-2 * n_ref + 1e-7, (k, n_got, n_ref)
            cos = float((g[k].ravel() @ v.ravel()) / max(n_got * n_ref, 1e-30))
            assert cos > 0.98 or n_ref < 1e-6, (k, cos)
    more = learner.update(2, graph=True)
    assert all(np.isfinite([s["critic_loss"], s["actor_loss"], s["q_mean"]]).all() for s in more)
    learner.close()
    del ring
    torch.cuda.empty_cache()


# ---------------------------------------------------------------- fused backward chains
@pytest.mark.parametrize("cluster", ["4", "8"])
def test_fused_backward_update_within_bf16_bounds(L, monkeypatch, cluster):
    """The BF16 update with the head MLPs' backward chains as fused launches (one per
    chain, the ReLU mask rebuilt from the fused forward's pre-activations) against the
    oracle within the BF16 bounds, and graph replay equal to eager bit for bit."""
    monkeypatch.setenv("SQUINT_MLP_BWD", "1")
    monkeypatch.setenv("SQUINT_MLP_BWD_CL", cluster)
    cfg = synth.make_config("train_b512", ring_size=4096)
    ring = synth.make_ring(cfg, 0, device="cuda")
    lazy = lazy_ring(ring)
    learner = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=2)
    twin = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=2)
    state = o.init_state(cfg)
    P0 = {k: v.copy() for k, v in state["params"].items()}
    stats = learner.update(1, graph=False)[0]
    twin.update(1, graph=True)
    assert np.array_equal(learner.params(), twin.params())
    ref, tr = o.update(state, lazy, cfg)
    g = split_params(learner.debug("grads"), cfg)
    mix = post_critic_state(P0, split_params(learner.params(), cfg), cfg)
    act = o.actor_loss(mix, tr["critic"]["z"], tr["frontend"]["p_t"], tr["eps_actor"],
                       math.exp(float(mix["log_alpha"][0])), cfg)
    assert abs(stats["q_mean"] - ref["q_mean"]) <= 2e-2 * max(abs(ref["q_mean"]), 1.0)
    assert abs(stats["critic_loss"] - ref["critic_loss"]) <= 1e-2 * abs(ref["critic_loss"])
    assert abs(stats["actor_loss"] - act["loss"]) <= 3e-2 * max(abs(act["loss"]), 1.0)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(act["grads"])
    for k, v in ref_grads.items():
        n_got, n_ref = np.linalg.norm(g[k]), np.linalg.norm(v)
        assert abs(n_got - n_ref) <= 5e-2 * n_ref + 1e-7, (k, n_got, n_ref)
    learner.close()
    twin.close()


def test_actor_step_input_gradients_kept_apart_match_their_gemm_sum(L, monkeypatch):
    """The actor step's gradient at the action through the two critics: each critic's part
    left by its fused chain launch and added in the tanh-Gaussian head backward, against
    one GEMM over both critics' products.  Only the FP32 summation order differs: the
    critic range (gradients and updated parameters) is bit-identical, the actor
    gradients agree to 1e-3 relative in norm per tensor and the actor loss exactly."""
    cfg = synth.make_config("train_b512", ring_size=4096)
    ring = synth.make_ring(cfg, 0, device="cuda")
    monkeypatch.setenv("SQUINT_MLP_FIN_SPLIT", "0")
    a = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=2)
    monkeypatch.setenv("SQUINT_MLP_FIN_SPLIT", "1")
    b = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=2)
    sa = a.update(1, graph=True)[0]
    sb = b.update(1, graph=True)[0]
    assert sa["critic_loss"] == sb["critic_loss"] and sa["actor_loss"] == sb["actor_loss"]
    ga, gb = split_params(a.debug("grads"), cfg), split_params(b.debug("grads"), cfg)
    pa, pb = split_params(a.params(), cfg), split_params(b.params(), cfg)
    for k in ga:
        if o.group_of(k) == "actor":
            n = np.linalg.norm(ga[k])
            assert np.linalg.norm(ga[k] - gb[k]) <= 1e-3 * n + 1e-9, k
        else:
            assert np.array_equal(ga[k], gb[k]), k
            assert np.array_equal(pa[k], pb[k]), k
    a.close()
    b.close()


@pytest.mark.parametrize("name", ["train_b512", "small_b32"])
def test_actor_forward_in_two_launches_equals_one(L, monkeypatch, name):
    """The actor's fused forward split in two launches (the target's o_{t+1} half on the
    critical chain without saved activations, the o_t half with its saves and its sample
    on a side branch) gives the same bits as one launch over both halves: statistics,
    parameters and target over three updates (rows are independent in the fused kernel)."""
    cfg = synth.make_config(name, **({"ring_size": 4096} if name == "train_b512" else {}))
    ring = synth.make_ring(cfg, 0, device="cuda")
    monkeypatch.setenv("SQUINT_SPLIT_ACTOR_FWD", "0")
    a = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=4)
    monkeypatch.setenv("SQUINT_SPLIT_ACTOR_FWD", "1")
    b = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=4)
    sa = a.update(3)
    sb = b.update(3)
    assert sa == sb
    assert np.array_equal(a.params(), b.params())
    assert np.array_equal(a.debug("target"), b.debug("target"))
    a.close()
    b.close()


# ---------------------------------------------------------------- update timeline
def test_trace_update_reports_every_launch_on_its_branch(L):
    """The traced update has every launch with 0 <= start <= end, the main stream's
    launches in issue order without overlap, launches on the side branches, and the
    kernel classes of the in-order profile."""
    cfg = synth.make_config("small_b32")
    ring = synth.make_ring(cfg, 0, device="cuda")
    learner = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=2)
    learner.update(1)
    tr = learner.trace_update()
    assert len(tr) > 10
    assert all(0.0 <= a <= b for _, _, a, b in tr)
    main = [(a, b) for _, lane, a, b in tr if lane == 0]
    assert all(main[i][1] <= main[i + 1][0] + 1e-6 for i in range(len(main) - 1))
    assert any(lane > 0 for _, lane, _, _ in tr)
    classes = set(learner.profile_kernels())
    assert {n for n, _, _, _ in tr} == classes
    learner.close()


# ---------------------------------------------------------------- polyak in the Adam pass
@pytest.mark.parametrize("prec", ["FP32", "BF16"])
def test_polyak_fused_into_adam_equals_its_own_launch(L, monkeypatch, prec):
    """The target critics' polyak done inside the critic Adam's pass gives the same bits
    (parameters, target, Adam moments, statistics) as its own launch after it."""
    cfg = synth.make_config("small_b32")
    ring = synth.make_ring(cfg, 0, device="cuda")
    monkeypatch.setenv("SQUINT_FUSE_POLYAK", "0")
    a = L.Learner(cfg, ring, precision=getattr(L, "PREC_" + prec), max_k=2)
    monkeypatch.setenv("SQUINT_FUSE_POLYAK", "1")
    b = L.Learner(cfg, ring, precision=getattr(L, "PREC_" + prec), max_k=2)
    sa = a.update(2)
    sb = b.update(2)
    for x, y in zip(sa, sb):
        for k in ("critic_loss", "actor_loss", "q_mean"):
            assert x[k] == y[k] or (math.isnan(x[k]) and math.isnan(y[k])), k
    assert np.array_equal(a.params(), b.params())
    assert np.array_equal(a.debug("target"), b.debug("target"))
    assert a.state() == b.state()
    a.close()
    b.close()
