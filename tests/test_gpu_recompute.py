"""Encoder activation recompute (BF16 tensor-core encoder; needs a GB300).

With `recompute_chunk` the encoder runs in chunks of images, keeps only the
features, and recomputes each chunk's activations in the backward.  Forward
kernels compute each image independently and the weight gradient keeps the
whole-batch partition of images over CTAs, so the update is bit-identical to
the one that keeps the activations; the learner allocates less device memory.
At batch 2048 one update is also checked against the FP64 oracle (BF16 bounds)
and UTD-8 graph replays are compared bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import lazy_ring, split_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2602_21203_gb300 import lib
    return lib


def _pair(L, batch, chunk, ring_size, k):
    cfg = synth.make_config("train_b512", batch=batch, ring_size=ring_size)
    ring = synth.make_ring(cfg, 0, device="cuda")
    keep = L.Learner(cfg, ring, precision=L.PREC_BF16, max_k=k)
    rc = L.Learner(dict(cfg, recompute_chunk=chunk), ring, precision=L.PREC_BF16, max_k=k)
    return cfg, ring, keep, rc


def test_recompute_is_bit_identical_and_smaller(L):
    cfg, ring, keep, rc = _pair(L, 160, 48, 4096, 2)
    assert rc.device_bytes() < keep.device_bytes()
    sa = keep.update(2, graph=True)
    sb = rc.update(2, graph=True)
    assert sa == sb
    assert np.array_equal(keep.params(), rc.params())
    assert np.array_equal(keep.debug("grads"), rc.debug("grads"))
    keep.close()
    rc.close()


def test_recompute_rejected_without_tensor_core_encoder(L):
    cfg = dict(synth.make_config("tiny_b8"), recompute_chunk=4)
    with pytest.raises(L.SquintError) as e:
        L.Learner(cfg, None, precision=L.PREC_BF16)
    assert e.value.code == L.EINVAL
    with pytest.raises(L.SquintError):
        L.Learner(dict(synth.make_config("train_b512"), recompute_chunk=64), None, precision=L.PREC_FP32)


def test_recompute_batch_2048_utd_8(L):
    """Training shapes at batch 2048: memory saved, one update vs the oracle, k = 8 bitwise."""
    cfg, ring, keep, rc = _pair(L, 2048, 256, 20000, 8)
    saved = keep.device_bytes() - rc.device_bytes()
    print(f"\nbatch 2048: {keep.device_bytes() / 2**20:.1f} MiB keeping activations, "
          f"{rc.device_bytes() / 2**20:.1f} MiB with recompute (saves {saved / 2**20:.1f} MiB)")
    assert saved > 200 * 2**20
    st = rc.update(1, graph=False)[0]
    ref, tr = o.update(o.init_state(cfg), lazy_ring(ring), cfg)
    assert abs(st["critic_loss"] - ref["critic_loss"]) <= 1e-2 * abs(ref["critic_loss"])
    assert abs(st["q_mean"] - ref["q_mean"]) <= 2e-2 * max(abs(ref["q_mean"]), 1.0)
    g = split_params(rc.debug("grads"), cfg)
    ref_grads = dict(tr["critic"]["grads"])
    ref_grads.update(tr["actor"]["grads"])
    for k, v in ref_grads.items():
        n_ref = float(np.linalg.norm(v))
        if n_ref < 1e-6:
            continue
        n_got = float(np.linalg.norm(g[k]))
        assert abs(n_got - n_ref) <= 5e-2 * n_ref, (k, n_got, n_ref)
        assert float(g[k].ravel() @ v.ravel()) / (n_got * n_ref) > 0.98, k
    keep.update(1, graph=False)
    sa = keep.update(8, graph=True)
    sb = rc.update(8, graph=True)
    assert sa == sb
    assert np.array_equal(keep.params(), rc.params())
    keep.close()
    rc.close()
    del ring
    torch.cuda.empty_cache()
