"""Precision sweep at the training shapes: FP32, BF16 and FP8 updates vs the FP64
oracle over 100 seeded batches (needs a GB300).

Batch s uses learner and oracle seed s (its own initial parameters and its own
Philox draws of slots, shifts and noise) on one 100k-slot ring.  For each batch
and precision the first update's Q-mean, critic cross entropy, actor loss and
every gradient tensor are compared with the oracle's.

Two quantities of one update are ill-conditioned functions of the update's input
and are compared where the conditioning is taken out, at the benchmark spec's bounds:

* The actor loss and the actor gradients are evaluated (Eq. 3, Alg. 1 "Update
  actor") through the critics after their Adam step and with the new temperature.
  Adam's first step from zero moments is lr g / (|g| + eps), close to lr sign(g):
  a critic gradient element within rounding distance of zero whose sign differs
  moves by 2 lr.  So the oracle's actor step is evaluated on the GPU's own
  post-critic-step parameters and temperature (with the oracle's pre-update actor,
  encoder features and noise); a separate check shows that every critic parameter
  whose step differs by more than lr / 2 is one whose oracle gradient is below 1e-3
  of its tensor's norm (an element the FP32 gradient tolerance cannot tell from
  zero), with the opposite sign on the GPU unless it is within ten times eps of zero.
* The first convolution's weight gradient sums batch x 15 x 15 pixels at the end
  of the longest ReLU chain: a pre-activation within rounding distance of zero that
  takes the other branch changes one pixel's whole upstream gradient.  It is
  compared with the oracle's conv3x3_bwd applied to the GPU's own gradient at the
  first layer's pre-activation (the GPU's ReLU masks), and a separate check shows
  that every ReLU on which the GPU and the oracle disagree, in every conv layer,
  has a pre-activation within 1e-5 of the layer's largest one of zero.

Bounds:
  FP32: Q-mean (relative to max(|Q|, 1)) and critic CE 1e-4; actor loss on the
        GPU's post-critic-step state 1e-4 (relative to max(|L|, 1e-2)); every
        gradient tensor 1e-3 relative in norm (the first conv's as above);
  BF16: Q-mean 2e-2, critic CE 1e-2, actor loss on the GPU's post-critic-step
        state 3e-2 (absolute below 1), gradient norm 5e-2 relative, direction
        cosine > 0.98;
  FP8:  Q-mean 1e-1, critic CE 1e-2, actor loss 3e-1, gradient norm 3e-1, cosine > 0.9;
  MX-FP8: the FP8 bounds.
The end-to-end actor loss and first-conv gradient errors are printed beside them.

The table of median / 90th percentile / maximum errors is printed (pytest -s).
"""
import math

import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import lazy_ring, post_critic_state, split_params

pytestmark = pytest.mark.gpu

N_BATCHES = 100
FP32 = dict(q_mean=1e-4, critic_loss=1e-4, actor_loss_iso=1e-4, grad_critic=1e-3, grad_actor=1e-3,
            grad_actor_iso=1e-3, grad_conv0_iso=1e-3)
BF16 = dict(q_mean=2e-2, critic_loss=1e-2, actor_loss_iso=3e-2, grad_norm=5e-2)
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
KEYS = ("q_mean", "critic_loss", "actor_loss", "actor_loss_iso", "grad_critic", "grad_actor", "grad_actor_iso",
        "grad_conv0", "grad_conv0_iso", "grad_norm", "grad_cos")


def _err(key, got, ref, prec):
    if key == "q_mean":
        return abs(got - ref) / max(abs(ref), 1.0)
    if key.startswith("actor_loss"):
        # FP32: relative, floored at 1e-2 (the loss can pass through zero); reduced
        # precision: absolute below 1
        return abs(got - ref) / max(abs(ref), 1e-2 if prec == "fp32" else 1.0)
    return abs(got - ref) / max(abs(ref), 1e-12)


def _rel(a, b):
    n = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / n if n > 0 else float(np.linalg.norm(a))


def _encoder_preacts(P0, x, cfg):
    """FP64 pre-activations of every conv layer on the o_t images."""
    out, h = [], x
    for l, c in enumerate(o.dims(cfg)["conv"]):
        pre = o.conv3x3_fwd(h, P0[f"enc.conv{l}.w"], P0[f"enc.conv{l}.b"], c["s"])
        out.append(pre)
        h = np.maximum(pre, 0.0)
    return out


def test_precision_sweep_100_batches():
    from paper_2602_21203_gb300 import lib
    base = synth.make_config("train_b512")
    ring = synth.make_ring(base, 0, device="cuda")
    lazy = lazy_ring(ring)
    rows = {p: {k: [] for k in KEYS} for p in ("fp32", "bf16", "fp8", "mxfp8")}
    worst_name = {}
    flips = {"adam": 0, "adam_ratio": 0.0, "relu": 0, "batches_relu": 0}
    lr = base["lr"]
    for s in range(N_BATCHES):
        cfg = synth.make_config("train_b512", seed=s)
        state = o.init_state(cfg)
        P0 = {k: v.copy() for k, v in state["params"].items()}
        ref, tr = o.update(state, lazy, cfg)
        fe = tr["frontend"]
        ref_grads = dict(tr["critic"]["grads"])
        ref_grads.update(tr["actor"]["grads"])
        for name, prec in (("fp32", lib.PREC_FP32), ("bf16", lib.PREC_BF16), ("fp8", lib.PREC_FP8),
                           ("mxfp8", lib.PREC_MXFP8)):
            learner = lib.Learner(cfg, ring, precision=prec, max_k=1)
            st = learner.update(1, graph=False)[0]
            g = split_params(learner.debug("grads"), cfg)
            p_gpu = split_params(learner.params(), cfg)
            extra = {}
            if name == "fp32":
                extra["dconv0"] = learner.debug("dconv0")
                for l in range(cfg["conv_layers"]):
                    extra[f"conv{l}"] = learner.debug(f"conv{l}")
            learner.close()
            r = rows[name]
            for key in ("q_mean", "critic_loss", "actor_loss"):
                r[key].append(_err(key, st[key], ref[key], name))
            gr = {"critic": 0.0, "actor": 0.0, "conv0": 0.0}
            gn, gc = 0.0, 1.0
            for k, v in ref_grads.items():
                n_ref = float(np.linalg.norm(v))
                if n_ref < 1e-6:
                    continue
                grp = "actor" if k in tr["actor"]["grads"] else ("conv0" if k == FIRST_CONV else "critic")
                e = _rel(g[k], v)
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
            if name not in ("fp32", "bf16"):
                continue
            # the actor step on the state the GPU's actor step read
            P_mix = post_critic_state(P0, p_gpu, cfg)
            alpha = math.exp(float(P_mix["log_alpha"][0]))
            act = o.actor_loss(P_mix, tr["critic"]["z"], fe["p_t"], tr["eps_actor"], alpha, cfg)
            r["actor_loss_iso"].append(_err("actor_loss_iso", st["actor_loss"], act["loss"], name))
            r["grad_actor_iso"].append(max(_rel(g[k], v) for k, v in act["grads"].items()))
            if name != "fp32":
                continue
            # every critic parameter whose Adam step differs by more than lr / 2 has a
            # gradient within rounding distance of zero, with the opposite sign on the GPU
            for k, v in tr["critic"]["grads"].items():
                d_gpu = p_gpu[k] - P0[k]
                d_ref = state["params"][k] - P0[k]
                bad = np.abs(d_gpu - d_ref) > 0.5 * lr
                if bad.any():
                    # an element the FP32 gradient tolerance (1e-3 of the tensor's norm)
                    # cannot tell from zero
                    scale = float(np.linalg.norm(v))
                    assert np.all(np.abs(v[bad]) <= 1e-3 * scale), (s, k, float(np.abs(v[bad]).max()), scale)
                    flips["adam_ratio"] = max(flips["adam_ratio"], float(np.abs(v[bad]).max()) / scale)
                    # the other sign, or a gradient near Adam's eps (a step short of lr)
                    unsat = np.minimum(np.abs(g[k][bad]), np.abs(v[bad])) < 10.0 * cfg["adam_eps"]
                    assert np.all((np.sign(g[k][bad]) != np.sign(v[bad])) | unsat), (s, k)
                    flips["adam"] += int(bad.sum())
            # the first conv's weight gradient from the GPU's own gradient at its pre-activation
            c0 = o.dims(cfg)["conv"][0]
            dy0 = extra["dconv0"].astype(np.float64).reshape(cfg["batch"], c0["cout"], c0["oh"], c0["ow"])
            _, dw0, db0 = o.conv3x3_bwd(fe["x_t"], P0["enc.conv0.w"], dy0, c0["s"], need_dx=False)
            r["grad_conv0_iso"].append(max(_rel(g["enc.conv0.w"], dw0), _rel(g["enc.conv0.b"], db0)))
            # ReLU decisions the GPU and the oracle disagree on sit at rounding-size pre-activations
            n_flip = 0
            for l, pre in enumerate(_encoder_preacts(P0, fe["x_t"], cfg)):
                on_gpu = extra[f"conv{l}"].reshape(pre.shape) > 0
                diff = on_gpu != (pre > 0)
                if diff.any():
                    scale = float(np.abs(pre).max())
                    assert np.all(np.abs(pre[diff]) <= 1e-5 * scale), (s, l, float(np.abs(pre[diff]).max()), scale)
                    n_flip += int(diff.sum())
            flips["relu"] += n_flip
            flips["batches_relu"] += n_flip > 0
    print(f"\nerror vs FP64 oracle over {N_BATCHES} batches (train_b512, first update of seed s):")
    print(f"{'quantity':15s} {'prec':5s} {'median':>10s} {'p90':>10s} {'worst':>10s}")
    for name in ("fp32", "bf16", "fp8", "mxfp8"):
        for key, v in rows[name].items():
            if not v:
                continue
            a = np.asarray(v)
            print(f"{key:15s} {name:5s} {np.median(a):10.3e} {np.percentile(a, 90):10.3e} "
                  f"{(a.min() if key == 'grad_cos' else a.max()):10.3e}")
    for name in ("fp32", "bf16", "fp8", "mxfp8"):
        for grp in ("critic", "actor"):
            v = rows[name]["grad_" + grp]
            b = int(np.argmax(v))
            print(f"worst {grp}-group gradient, {name}: batch {b}, {worst_name.get((name, grp, b))}, {v[b]:.3e}")
    print(f"FP32: {flips['adam']} critic parameters took the other sign of Adam's first step (largest "
          f"|g| there {flips['adam_ratio']:.2e} of its tensor's norm); "
          f"{flips['relu']} encoder ReLU decisions differ, in {flips['batches_relu']} of {N_BATCHES} batches")
    for name, bounds in (("fp32", FP32), ("bf16", BF16), ("fp8", FP8), ("mxfp8", MXFP8)):
        for key, tol in bounds.items():
            worst = max(rows[name][key])
            assert worst <= tol, (name, key, worst)
    assert min(rows["bf16"]["grad_cos"]) > 0.98
    assert min(rows["fp8"]["grad_cos"]) > 0.9
    assert min(rows["mxfp8"]["grad_cos"]) > 0.9
    del ring
    torch.cuda.empty_cache()
