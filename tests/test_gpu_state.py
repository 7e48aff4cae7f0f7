"""State-based SAC (Sec. VII, Fig. 6 left: the same UTD update with the encoder removed)
on the CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances as for the visual update: FP32 losses 1e-4 relative, every gradient tensor
1e-3 relative in norm, slots bit-exact; BF16 / FP8 at the training shapes (1M-slot ring of
48-d states, batch 512) with the bounds of the precision sweep.
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import flatten, lazy_ring, rel_err, ring_to_device, split_params

pytestmark = pytest.mark.gpu

SMALL = "state_small_b64"
TRAIN = "state_b512"


@pytest.fixture(scope="module")
def L():
    from paper_2602_21203_gb300 import lib
    return lib


def _close(a, b, rtol, atol=0.0):
    return abs(a - b) <= rtol * abs(b) + atol


@pytest.mark.parametrize("name", [SMALL, TRAIN])
def test_state_initial_parameters_match_oracle_bitwise(L, name):
    cfg = synth.make_config(name)
    learner = L.Learner(cfg, None)
    assert np.array_equal(learner.params(), flatten(o.init_params(cfg), cfg).astype(np.float32))
    learner.close()


def test_state_config_validation(L):
    with pytest.raises(L.SquintError) as e:
        L.Learner(synth.make_config(SMALL, proj_dim=64), None)       # no features to project
    assert e.value.code == L.EINVAL
    with pytest.raises(L.SquintError):
        L.Learner(synth.make_config(SMALL, proprio_dim=0), None)     # no input at all


@pytest.mark.parametrize("graph", [False, True])
def test_state_updates_match_oracle_fp32(L, graph):
    """Update 0 at the FP32 bounds (statistics, target, every gradient, parameter change);
    updates 1-2 continue both sides independently, statistics within 1e-3 (Adam's first
    steps move near-zero-gradient elements by about lr whatever their rounding)."""
    cfg = synth.make_config(SMALL)
    ring_cpu = synth.make_ring(cfg, 0)
    assert "obs" not in ring_cpu
    learner = L.Learner(cfg, ring_to_device(ring_cpu))
    ring_np = synth.ring_numpy(ring_cpu)
    state = o.init_state(cfg)
    for u in range(3):
        p_before = learner.params().astype(np.float64)
        st = learner.update(1, graph=graph)[0]
        ref, tr = o.update(state, ring_np, cfg)
        tol = 1e-4 if u == 0 else 1e-3
        for key in ("critic_loss", "alpha_loss", "alpha", "entropy", "actor_loss"):
            assert _close(st[key], ref[key], tol, 1e-6), (u, key, st[key], ref[key])
        assert _close(st["q_mean"], ref["q_mean"], tol, 1e-5), (u, st["q_mean"], ref["q_mean"])
        assert np.array_equal(learner.debug("idx", np.int32), tr["frontend"]["idx"])
        assert np.array_equal(learner.debug("nxt", np.int32), tr["frontend"]["nxt"])
        if u:
            continue
        K = cfg["atoms"]
        assert np.abs(learner.debug("m").reshape(-1, K) - tr["target"]["m"]).max() < 1e-5
        g = split_params(learner.debug("grads"), cfg)
        ref_grads = dict(tr["critic"]["grads"])
        ref_grads.update(tr["actor"]["grads"])
        assert set(ref_grads) == {n for n, *_ in o.param_spec(cfg) if n != "log_alpha"}
        for k, v in ref_grads.items():
            assert rel_err(g[k], v) < 1e-3, (k, rel_err(g[k], v))
        p_after = learner.params().astype(np.float64)
        ref_after = flatten(state["params"], cfg)
        assert rel_err(p_after - p_before, ref_after - p_before) < 1e-3
    learner.close()


def test_state_graph_replay_equals_eager_bitwise(L):
    cfg = synth.make_config(SMALL)
    ring = ring_to_device(synth.make_ring(cfg, 1))
    a = L.Learner(cfg, ring)
    b = L.Learner(cfg, ring)
    for _ in range(2):
        sa = a.update(4, graph=True)
        sb = b.update(4, graph=False)
        assert sa == sb
        assert np.array_equal(a.params(), b.params())
    a.close()
    b.close()


@pytest.mark.parametrize("prec,bounds", [
    ("bf16", dict(q_mean=2e-2, critic_loss=1e-2, actor_loss=5e-2, grad_norm=5e-2, cos=0.98)),
    ("fp8", dict(q_mean=1e-1, critic_loss=1e-2, actor_loss=3e-1, grad_norm=3e-1, cos=0.9)),
    ("mxfp8", dict(q_mean=1e-1, critic_loss=1e-2, actor_loss=3e-1, grad_norm=3e-1, cos=0.9)),
])
def test_state_training_shape_low_precision(L, prec, bounds):
    cfg = synth.make_config(TRAIN)
    ring = synth.make_ring(cfg, 0, device="cuda")
    learner = L.Learner(cfg, ring, precision={"bf16": L.PREC_BF16, "fp8": L.PREC_FP8, "mxfp8": L.PREC_MXFP8}[prec])
    st = learner.update(1, graph=False)[0]
    ref, tr = o.update(o.init_state(cfg), lazy_ring(ring), cfg)
    assert abs(st["q_mean"] - ref["q_mean"]) <= bounds["q_mean"] * max(abs(ref["q_mean"]), 1.0)
    assert abs(st["critic_loss"] - ref["critic_loss"]) <= bounds["critic_loss"] * abs(ref["critic_loss"])
    al = abs(st["actor_loss"] - ref["actor_loss"])
    assert al <= bounds["actor_loss"] * (1.0 if abs(ref["actor_loss"]) < 1 else abs(ref["actor_loss"]))
    g = split_params(learner.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    for k, v in ref_grads.items():
        n_ref = float(np.linalg.norm(v))
        if n_ref < 1e-6:
            continue
        n_got = float(np.linalg.norm(g[k]))
        assert abs(n_got - n_ref) <= bounds["grad_norm"] * n_ref, (k, n_got, n_ref)
        assert float(g[k].ravel() @ v.ravel()) / (n_got * n_ref) > bounds["cos"], k
    # UTD-4 graph replays run and keep finite statistics
    for s in learner.update(4, graph=True):
        assert all(np.isfinite(s[k]) for k in ("critic_loss", "actor_loss", "q_mean", "alpha"))
    learner.close()
    del ring
    torch.cuda.empty_cache()


@pytest.mark.parametrize("sample", [True, False])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_state_act_matches_oracle(L, sample, prec):
    cfg = synth.make_config(SMALL)
    learner = L.Learner(cfg, None, precision={"fp32": L.PREC_FP32, "bf16": L.PREC_BF16}[prec])
    P = o.init_params(cfg)
    obs, prop = synth.make_obs_batch(37, cfg, 5, device="cuda")
    assert obs is None
    out = torch.full((37, cfg["action_dim"]), float("nan"), device="cuda")
    learner.act([L.Learner.request(None, prop, out, key=4321, sample=sample)])
    torch.cuda.synchronize()
    ref = o.act(P, None, prop.cpu().numpy(), 4321, sample, cfg)
    tol = 1e-5 if prec == "fp32" else 3e-2
    assert np.abs(out.cpu().numpy() - ref).max() < tol
    # a row's action does not depend on the other rows of the batch
    part = torch.full((5, cfg["action_dim"]), float("nan"), device="cuda")
    learner.act([L.Learner.request(None, prop[:5], part, key=4321, sample=sample)])
    torch.cuda.synchronize()
    assert torch.equal(part, out[:5])
    learner.close()
