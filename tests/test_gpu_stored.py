"""Squint at insert (the paper's replay layout, Alg. 1; needs a GB300).

The insert kernel stores rounded area means of 3x128x128 renders as 3x32x32 uint8
frames, bit-exact against the oracle, wrapping around the ring; a learner reading
such a ring (f = 1, shift at 32x32) matches the oracle's update on the same ring.
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import lazy_ring, rel_err, split_params

pytestmark = pytest.mark.gpu


def test_squint_store_is_bit_exact_and_wraps():
    from paper_2602_21203_gb300 import ops
    cfg = synth.make_config("stored_b512")
    frames = synth.render_frames(37, cfg, 5, device="cuda")
    ring = torch.full((50, 3, 32, 32), 7, dtype=torch.uint8, device="cuda")
    ops.squint_store(frames, ring, 30, 4)
    torch.cuda.synchronize()
    ref = o.squint_store(frames.cpu().numpy(), 4)
    got = ring.cpu().numpy()
    slots = [(30 + i) % 50 for i in range(37)]
    assert np.array_equal(got[slots], ref)
    untouched = [s for s in range(50) if s not in slots]
    assert (got[untouched] == 7).all()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_update_on_a_stored_ring_matches_oracle(prec):
    from paper_2602_21203_gb300 import lib, ops
    cfg = synth.make_config("stored_b512", ring_size=3000)
    ring = synth.make_ring(cfg, 0, device="cuda")
    for c0 in range(0, 3000, 1000):                 # fill the frames through the insert kernel
        ops.squint_store(synth.render_frames(1000, cfg, 100 + c0, device="cuda"), ring["obs"], c0, 4)
    torch.cuda.synchronize()
    learner = lib.Learner(cfg, ring, precision=lib.PREC_FP32 if prec == "fp32" else lib.PREC_BF16)
    st = learner.update(1, graph=True)[0]
    ref, tr = o.update(o.init_state(cfg), lazy_ring(ring), cfg)
    g = split_params(learner.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    if prec == "fp32":
        assert abs(st["critic_loss"] - ref["critic_loss"]) <= 1e-4 * abs(ref["critic_loss"])
        assert abs(st["q_mean"] - ref["q_mean"]) <= 1e-4 * max(abs(ref["q_mean"]), 1.0)
        for k, v in ref_grads.items():   # first-conv weight gradient: 5e-3 (ReLU ties, see the sweep)
            if np.linalg.norm(v) > 1e-6:
                assert rel_err(g[k], v) < (5e-3 if k == "enc.conv0.w" else 1e-3), k
    else:
        assert abs(st["critic_loss"] - ref["critic_loss"]) <= 1e-2 * abs(ref["critic_loss"])
        for k, v in ref_grads.items():
            n_ref = float(np.linalg.norm(v))
            if n_ref > 1e-6:
                assert abs(float(np.linalg.norm(g[k])) - n_ref) <= 5e-2 * n_ref, k
    more = learner.update(4, graph=True)
    assert all(np.isfinite(s["critic_loss"]) for s in more)
    learner.close()
