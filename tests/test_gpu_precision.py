"""Precision sweep at the training shapes: FP32, BF16 and FP8 updates vs the FP64
oracle over 100 seeded batches (needs a GB300).

Batch s uses learner and oracle seed s (its own initial parameters and its own
Philox draws of slots, shifts and noise) on one 100k-slot ring.  For each batch
and precision the first update's Q-mean, critic cross entropy, actor loss and
every gradient tensor are compared with the oracle's (per batch, the worst
tensor: relative error in norm, relative error of the norm, direction cosine).  Every batch must
meet the stated tolerances:

  FP32: Q-mean (relative to max(|Q|, 1)) and critic CE 1e-4, actor loss 1e-3
        (absolute below 1), every gradient tensor 1e-3 relative in norm except the
        first convolution's weight gradient, 5e-3;
  BF16: Q-mean 2e-2, critic CE 1e-2, actor loss 5e-2 (absolute below 1),
        gradient norm 5e-2 relative, direction cosine > 0.98;
  FP8:  Q-mean 1e-1, critic CE 1e-2, actor loss 3e-1, gradient norm 3e-1, cosine > 0.9;
  MX-FP8: the FP8 bounds.

The table of median / 90th percentile / maximum errors is printed (pytest -s).
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import lazy_ring, split_params

pytestmark = pytest.mark.gpu

N_BATCHES = 100
# Q-mean and the critic loss are computed before any parameter moves and keep the
# tight bound; Q-mean relative to max(|Q|, 1) (one return unit on the +-20 support),
# since Q is near zero at initialisation.  The actor loss is taken through the
# critics after their Adam step, whose first step is close to lr * sign(g): a critic
# gradient element near zero whose sign differs by rounding moves by 2 lr, so the
# actor loss gets 1e-3 (absolute below 1).  Gradient tensors keep 1e-3 except the
# first convolution's weight gradient: it is a sum over batch x 15 x 15 pixels with
# heavy cancellation at the end of the longest chain of ReLUs, so one pre-activation
# within rounding distance of zero that takes the other branch moves it by about
# 1/sqrt(terms) ~ 3e-3 relative; it gets 5e-3 in FP32 and is covered by the norm and
# direction bounds in BF16.
FP32 = dict(q_mean=1e-4, critic_loss=1e-4, actor_loss=1e-3, grad_critic=1e-3, grad_actor=1e-3, grad_conv0=5e-3)
BF16 = dict(q_mean=2e-2, critic_loss=1e-2, actor_loss=5e-2, grad_norm=5e-2)
# FP8 (e4m3 forward linear layers, per-tensor scale amax / 448; backward in BF16): e4m3
# keeps 3 mantissa bits, so one rounding is up to 2^-4 = 6.25% relative (1.8% RMS), and
# small entries of a tensor scaled to its maximum lose more.  Forward activations carry
# a few per cent, Q-mean up to 10%; gradients, computed in BF16 from those activations
# and ReLU decisions, keep their norms within 30% and their directions (cosine > 0.9).
FP8 = dict(q_mean=1e-1, critic_loss=1e-2, actor_loss=3e-1, grad_norm=3e-1)
# MX-FP8 (one power-of-two scale per 32 elements of a row): every element keeps e4m3's 3
# mantissa bits within its block's range (the block maximum lands in (224, 448], and
# elements down to 2^-15 of it stay normal), so the per-element rounding bound is the
# same 2^-4 as for per-tensor FP8 and the same bounds apply; the finer scales only spare
# the small entries of a tensor the extra loss of subnormal codes.
MXFP8 = FP8
FIRST_CONV = "enc.conv0.w"


def _err(key, got, ref):
    if key == "q_mean":
        return abs(got - ref) / max(abs(ref), 1.0)
    if key == "actor_loss" and abs(ref) < 1:
        return abs(got - ref)
    return abs(got - ref) / max(abs(ref), 1e-12)


def test_precision_sweep_100_batches():
    from paper_2602_21203_gb300 import lib
    base = synth.make_config("train_b512")
    ring = synth.make_ring(base, 0, device="cuda")
    lazy = lazy_ring(ring)
    rows = {p: {k: [] for k in ("q_mean", "critic_loss", "actor_loss", "grad_critic", "grad_actor", "grad_conv0",
                                "grad_norm", "grad_cos")}
            for p in ("fp32", "bf16", "fp8", "mxfp8")}
    worst_name = {}
    for s in range(N_BATCHES):
        cfg = synth.make_config("train_b512", seed=s)
        ref, tr = o.update(o.init_state(cfg), lazy, cfg)
        ref_grads = dict(tr["critic"]["grads"])
        ref_grads.update(tr["actor"]["grads"])
        for name, prec in (("fp32", lib.PREC_FP32), ("bf16", lib.PREC_BF16), ("fp8", lib.PREC_FP8),
                           ("mxfp8", lib.PREC_MXFP8)):
            learner = lib.Learner(cfg, ring, precision=prec, max_k=1)
            st = learner.update(1, graph=False)[0]
            g = split_params(learner.debug("grads"), cfg)
            learner.close()
            r = rows[name]
            for key in ("q_mean", "critic_loss", "actor_loss"):
                r[key].append(_err(key, st[key], ref[key]))
            gr = {"critic": 0.0, "actor": 0.0, "conv0": 0.0}
            gn, gc = 0.0, 1.0
            for k, v in ref_grads.items():
                n_ref = float(np.linalg.norm(v))
                if n_ref < 1e-6:
                    continue
                grp = "actor" if k in tr["actor"]["grads"] else ("conv0" if k == FIRST_CONV else "critic")
                e = float(np.linalg.norm(g[k] - v)) / n_ref
                if e > gr[grp]:
                    gr[grp] = e
                    worst_name[(name, grp, s)] = k
                gn = max(gn, abs(float(np.linalg.norm(g[k])) - n_ref) / n_ref)
                gc = min(gc, float(g[k].ravel() @ v.ravel()) / max(float(np.linalg.norm(g[k])) * n_ref, 1e-30))
            r["grad_critic"].append(gr["critic"])
            r["grad_actor"].append(gr["actor"])
            r["grad_conv0"].append(gr["conv0"])
            r["grad_norm"].append(gn)
            r["grad_cos"].append(gc)
    print(f"\nerror vs FP64 oracle over {N_BATCHES} batches (train_b512, first update of seed s):")
    print(f"{'quantity':14s} {'prec':5s} {'median':>10s} {'p90':>10s} {'worst':>10s}")
    for name in ("fp32", "bf16", "fp8", "mxfp8"):
        for key, v in rows[name].items():
            a = np.asarray(v)
            print(f"{key:14s} {name:5s} {np.median(a):10.3e} {np.percentile(a, 90):10.3e} "
                  f"{(a.min() if key == 'grad_cos' else a.max()):10.3e}")
    for name in ("fp32", "bf16", "fp8", "mxfp8"):
        for grp in ("critic", "actor"):
            v = rows[name]["grad_" + grp]
            b = int(np.argmax(v))
            print(f"worst {grp}-group gradient, {name}: batch {b}, {worst_name.get((name, grp, b))}, {v[b]:.3e}")
    for name, bounds in (("fp32", FP32), ("bf16", BF16), ("fp8", FP8), ("mxfp8", MXFP8)):
        for key, tol in bounds.items():
            worst = max(rows[name][key])
            assert worst <= tol, (name, key, worst)
    assert min(rows["bf16"]["grad_cos"]) > 0.98
    assert min(rows["fp8"]["grad_cos"]) > 0.9
    assert min(rows["mxfp8"]["grad_cos"]) > 0.9
    del ring
    torch.cuda.empty_cache()
