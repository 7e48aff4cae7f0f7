"""Critic variants (Sec. IV "Critic Design Choices"): MSE critic (Eq. 1-2) and clipped
double Q, through the C ABI vs the FP64 oracle (needs a GB300).

FP32: losses and Q-mean 1e-4, every gradient tensor 1e-3 relative in norm (the first
convolution's 5e-3, as in the precision sweep); BF16: critic loss 1e-2, gradient norms
5e-2; graph replays equal eager updates bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import lazy_ring, rel_err, ring_to_device, split_params

pytestmark = pytest.mark.gpu

# the MSE critic, clipped double Q, both; 201 atoms (more than four a lane in the warp-per-
# sample head kernels) with and without clipped double Q
VARIANTS = {"mse": dict(critic="mse"), "cdq": dict(cdq=True), "mse_cdq": dict(critic="mse", cdq=True),
            "atoms201": dict(atoms=201), "atoms201_cdq": dict(atoms=201, cdq=True)}


@pytest.fixture(scope="module")
def L():
    from paper_2602_21203_gb300 import lib
    return lib


def _close(a, b, rtol, floor=1e-6):
    return abs(a - b) <= rtol * max(abs(b), floor)


@pytest.mark.parametrize("var", list(VARIANTS))
def test_variant_update_matches_oracle_fp32(L, var):
    cfg = synth.make_config("small_b32", **VARIANTS[var])
    ring_cpu = synth.make_ring(cfg, 2)
    learner = L.Learner(cfg, ring_to_device(ring_cpu))
    assert learner.n_params == sum(int(np.prod(s)) for _, s, *_ in o.param_spec(cfg))
    state = o.init_state(cfg)
    st = learner.update(1, graph=True)[0]
    ref, tr = o.update(state, synth.ring_numpy(ring_cpu), cfg)
    for key in ("critic_loss", "alpha_loss", "alpha", "entropy"):
        assert _close(st[key], ref[key], 1e-4), (var, key, st[key], ref[key])
    assert abs(st["actor_loss"] - ref["actor_loss"]) <= 1e-4 * max(abs(ref["actor_loss"]), 1.0)
    assert abs(st["q_mean"] - ref["q_mean"]) <= 1e-4 * max(abs(ref["q_mean"]), 1.0)
    g = split_params(learner.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    for k, v in ref_grads.items():
        if np.linalg.norm(v) > 1e-7:
            assert rel_err(g[k], v) < (5e-3 if k == "enc.conv0.w" else 1e-3), (var, k, rel_err(g[k], v))
    more = learner.update(3, graph=True)
    assert all(np.isfinite([s["critic_loss"], s["actor_loss"]]).all() for s in more)
    learner.close()


def test_variant_bf16_training_shape_and_graph(L):
    cfg = synth.make_config("train_b512", ring_size=4096, critic="mse", cdq=True)
    ring = synth.make_ring(cfg, 0, device="cuda")
    a = L.Learner(cfg, ring, precision=L.PREC_BF16)
    st = a.update(1, graph=False)[0]
    ref, tr = o.update(o.init_state(cfg), lazy_ring(ring), cfg)
    assert _close(st["critic_loss"], ref["critic_loss"], 1e-2)
    g = split_params(a.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    for k, v in ref_grads.items():
        n_ref = float(np.linalg.norm(v))
        if n_ref > 1e-6:
            assert abs(float(np.linalg.norm(g[k])) - n_ref) <= 5e-2 * n_ref, k
    b = L.Learner(cfg, ring, precision=L.PREC_BF16)
    c = L.Learner(cfg, ring, precision=L.PREC_BF16)
    assert b.update(3, graph=True) == c.update(3, graph=False)
    assert np.array_equal(b.params(), c.params())
    for x in (a, b, c):
        x.close()
