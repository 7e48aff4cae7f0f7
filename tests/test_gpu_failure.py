"""Failure detection on the GPU without a fault (needs a GB300).

A bounded wait of a tensor-core kernel is made to run out: the update's GEMMs are
told to issue no operand loads, so the first wait of every MMA issuer, on an
mbarrier that nothing completes, gives up after a short limit.  The kernels record
the code in the learner's device error word, free their tensor memory and return;
the update reports SQUINT_ETIMEOUT and the handle refuses further work.  The
context stays usable: a fresh learner afterwards still matches the oracle.
"""
import numpy as np
import pytest

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import ring_to_device

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports_timeout():
    from paper_2602_21203_gb300 import lib as L
    cfg = synth.make_config("small_b32")
    ring_cpu = synth.make_ring(cfg, 0)
    ring = ring_to_device(ring_cpu)
    a = L.Learner(cfg, ring, precision=L.PREC_BF16)
    a.set_debug("wait_cycles", 200_000)          # about 0.1 ms per wait
    a.set_debug("stall_gemm_loads", 1)
    with pytest.raises(L.SquintError) as e:
        a.update(1, graph=False)
    assert e.value.code == L.ETIMEOUT
    with pytest.raises(L.SquintError) as e:      # the failed handle does no more work
        a.update(1, graph=False)
    assert e.value.code == L.ESTATE
    a.close()
    # tensor memory was freed and the context works: a fresh learner's update matches
    b = L.Learner(cfg, ring, precision=L.PREC_BF16)
    st = b.update(1, graph=True)[0]
    ref, _ = o.update(o.init_state(cfg), synth.ring_numpy(ring_cpu), cfg)
    assert abs(st["critic_loss"] - ref["critic_loss"]) <= 1e-2 * abs(ref["critic_loss"])
    assert abs(st["q_mean"] - ref["q_mean"]) <= 2e-2 * max(abs(ref["q_mean"]), 1.0)
    b.close()


def test_debug_settings_are_validated():
    from paper_2602_21203_gb300 import lib as L
    cfg = synth.make_config("tiny_b8")
    a = L.Learner(cfg, None, precision=L.PREC_BF16)
    for name, value in (("nope", 1), ("stall_gemm_loads", 2), ("wait_cycles", -1)):
        with pytest.raises(L.SquintError) as e:
            a.set_debug(name, value)
        assert e.value.code == L.EINVAL
    a.set_debug("wait_cycles", 0)
    a.close()
