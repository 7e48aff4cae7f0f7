"""Actor inference and the continuous-batching server vs the FP64 oracle (needs a GB300)."""
import time

import numpy as np
import pytest
import torch

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth
from util import ring_to_device, split_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2602_21203_gb300 import lib
    return lib


def _batch(cfg, n, seed):
    obs, prop = synth.make_obs_batch(n, cfg, seed, device="cuda")
    out = torch.full((n, cfg["action_dim"]), float("nan"), device="cuda")
    return obs, prop, out


@pytest.mark.parametrize("name,n", [("small_b32", 37), ("train_b512", 24)])
@pytest.mark.parametrize("sample", [True, False])
def test_act_matches_oracle(L, name, n, sample):
    cfg = synth.make_config(name)
    learner = L.Learner(cfg, None)
    P = o.init_params(cfg)
    obs, prop, out = _batch(cfg, n, 5)
    learner.act([L.Learner.request(obs, prop, out, key=1234, sample=sample)])
    torch.cuda.synchronize()
    ref = o.act(P, obs.cpu().numpy(), prop.cpu().numpy(), 1234, sample, cfg)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-5
    learner.close()


def test_act_row_results_do_not_depend_on_the_batch(L):
    cfg = synth.make_config("small_b32")
    learner = L.Learner(cfg, None)
    sizes = [1, 5, 17, 3, 64]
    groups = [_batch(cfg, n, 10 + i) for i, n in enumerate(sizes)]
    alone = []
    for i, (obs, prop, out) in enumerate(groups):
        learner.act([L.Learner.request(obs, prop, out, key=100 + i)])
        torch.cuda.synchronize()
        alone.append(out.clone())
        out.fill_(float("nan"))
    learner.act([L.Learner.request(obs, prop, out, key=100 + i) for i, (obs, prop, out) in enumerate(groups)])
    torch.cuda.synchronize()
    for (obs, prop, out), a in zip(groups, alone):
        assert torch.equal(out, a)
    learner.close()


def test_act_uses_updated_weights_after_refresh(L):
    cfg = synth.make_config("tiny_b8")
    ring = ring_to_device(synth.make_ring(cfg, 0))
    learner = L.Learner(cfg, ring)
    obs, prop, out = _batch(cfg, 4, 3)
    req = L.Learner.request(obs, prop, out, key=9, sample=False)
    learner.act([req])
    torch.cuda.synchronize()
    before = out.clone()
    learner.update(2)
    learner.act([req])                       # snapshot not refreshed yet: same weights
    torch.cuda.synchronize()
    assert torch.equal(out, before)
    learner.refresh_policy()
    learner.act([req])
    torch.cuda.synchronize()
    P = split_params(learner.params(), cfg)
    ref = o.act(P, obs.cpu().numpy(), prop.cpu().numpy(), 9, False, cfg)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-5
    assert not torch.equal(out, before)
    learner.close()


def test_serving_loop_results_equal_alone_and_admission(L):
    cfg = synth.make_config("small_b32")
    learner = L.Learner(cfg, None)
    rng = np.random.default_rng(0)
    sizes = [int(s) for s in rng.integers(1, 60, size=24)]
    groups = [_batch(cfg, n, 50 + i) for i, n in enumerate(sizes)]
    alone = []
    for i, (obs, prop, out) in enumerate(groups):
        learner.act([L.Learner.request(obs, prop, out, key=7 + i)])
        torch.cuda.synchronize()
        alone.append(out.clone())
        out.fill_(float("nan"))
    learner.serve_start(max_rows=128, mem_budget_bytes=1 << 30)
    tickets = []
    for i, (obs, prop, out) in enumerate(groups):
        t = learner.serve_submit(L.Learner.request(obs, prop, out, key=7 + i, group_id=i))
        assert t is not None
        tickets.append(t)
        if i % 5 == 0:
            time.sleep(0.001)                # arrivals spread over time
    lats = []
    for t in tickets:
        r = None
        deadline = time.time() + 30
        while r is None and time.time() < deadline:
            r = learner.serve_poll(t, timeout_us=100_000)
        assert r is not None
        lats.append(r[0])
    for (obs, prop, out), a in zip(groups, alone):
        assert torch.equal(out, a)
    assert all(x > 0 for x in lats)
    # a group larger than the admission limit is refused, not queued
    big = _batch(cfg, 200, 1)
    with pytest.raises(L.SquintError) as e:
        learner.serve_submit(L.Learner.request(*big, key=1))
    assert e.value.code == L.EINVAL
    learner.serve_stop()
    learner.close()


def test_serving_beside_updates_sees_consistent_snapshots(L):
    """Requests served while the update stream runs UTD steps and refreshes the policy."""
    cfg = synth.make_config("tiny_b8")
    ring = ring_to_device(synth.make_ring(cfg, 0))
    learner = L.Learner(cfg, ring)
    upd = torch.cuda.Stream()
    learner.serve_start(max_rows=64, mem_budget_bytes=1 << 28)
    obs, prop, out = _batch(cfg, 8, 4)
    versions = []
    snapshots = {}
    for step in range(6):
        with torch.cuda.stream(upd):
            learner.update(2, stats=False, stream=upd)
            learner.refresh_policy(stream=upd)
        t = learner.serve_submit(L.Learner.request(obs, prop, out, key=3, sample=False))
        r = None
        deadline = time.time() + 30
        while r is None and time.time() < deadline:
            r = learner.serve_poll(t, timeout_us=1_000_000)
        assert r is not None
        versions.append(r[1])
        snapshots.setdefault(r[1], out.clone())
    upd.synchronize()
    assert versions == sorted(versions)
    assert torch.isfinite(out).all() and (out.abs() < 1).all()
    learner.serve_stop()
    learner.close()


# ---------------------------------------------------------------- BF16 policy
# BF16 operands (8-bit mantissa, relative rounding 2^-9) with FP32 accumulation through
# the encoder, the projection and three actor layers leave about 1e-2 relative error
# in the pre-tanh outputs; with |d tanh| <= 1 the actions stay within 5e-2 of the FP64
# oracle, 1e-2 on average.
BF16_ACT_MAX, BF16_ACT_MEAN = 5e-2, 1e-2


@pytest.mark.parametrize("name,n", [("small_b32", 37), ("train_b512", 24)])
@pytest.mark.parametrize("sample", [True, False])
def test_bf16_act_matches_oracle(L, name, n, sample):
    cfg = synth.make_config(name)
    learner = L.Learner(cfg, None, precision=L.PREC_BF16)
    P = o.init_params(cfg)
    obs, prop, out = _batch(cfg, n, 6)
    learner.act([L.Learner.request(obs, prop, out, key=4321, sample=sample)])
    torch.cuda.synchronize()
    ref = o.act(P, obs.cpu().numpy(), prop.cpu().numpy(), 4321, sample, cfg)
    err = np.abs(out.cpu().numpy() - ref)
    assert err.max() < BF16_ACT_MAX and err.mean() < BF16_ACT_MEAN, (err.max(), err.mean())
    learner.close()


def test_bf16_serving_results_equal_alone(L):
    """Training shapes (tensor-core convs and GEMMs): each group's actions are bit-identical
    whether it runs alone or batched with other groups by the serving loop."""
    cfg = synth.make_config("train_b512")
    learner = L.Learner(cfg, None, precision=L.PREC_BF16)
    rng = np.random.default_rng(1)
    sizes = [int(s) for s in rng.integers(1, 200, size=12)]
    groups = [_batch(cfg, n, 80 + i) for i, n in enumerate(sizes)]
    alone = []
    for i, (obs, prop, out) in enumerate(groups):
        learner.act([L.Learner.request(obs, prop, out, key=11 + i)])
        torch.cuda.synchronize()
        alone.append(out.clone())
        out.fill_(float("nan"))
    learner.serve_start(max_rows=1024, mem_budget_bytes=4 << 30)
    tickets = [learner.serve_submit(L.Learner.request(obs, prop, out, key=11 + i, group_id=i))
               for i, (obs, prop, out) in enumerate(groups)]
    for t in tickets:
        r = None
        deadline = time.time() + 30
        while r is None and time.time() < deadline:
            r = learner.serve_poll(t, timeout_us=100_000)
        assert r is not None
    for (obs, prop, out), a in zip(groups, alone):
        assert torch.equal(out, a)
    learner.serve_stop()
    learner.close()


def test_serving_overlaps_batches_and_each_result_matches_alone(L):
    """Continuous batching: groups submitted together run as batches in several slots at
    once (their device intervals overlap), and every group's actions are the same bits as
    the group evaluated alone (the BF16 training-shape policy)."""
    cfg = synth.make_config("train_b512")
    learner = L.Learner(cfg, None, precision=L.PREC_BF16)
    groups = [_batch(cfg, n, 40 + i) for i, n in enumerate([512, 512, 300, 512, 77, 512])]
    alone = []
    for i, (obs, prop, out) in enumerate(groups):
        learner.act([L.Learner.request(obs, prop, out, key=90 + i)])
        torch.cuda.synchronize()
        alone.append(out.clone())
        out.fill_(float("nan"))
    learner.serve_start(max_rows=512, mem_budget_bytes=8 << 30)
    info = learner.serve_info()
    assert info["slots"] >= 2 and info["slot_rows"] == 512
    overlapped = False
    for attempt in range(5):
        tickets = [learner.serve_submit(L.Learner.request(obs, prop, out, key=90 + i, group_id=i))
                   for i, (obs, prop, out) in enumerate(groups)]
        res = []
        for t in tickets:
            r = None
            deadline = time.time() + 30
            while r is None and time.time() < deadline:
                r = learner.serve_poll_ex(t, timeout_us=100_000)
            assert r is not None
            res.append(r)
        for (obs, prop, out), a in zip(groups, alone):
            assert torch.equal(out, a)
            out.fill_(float("nan"))
        for i in range(len(res)):
            for j in range(len(res)):
                a, b = res[i], res[j]
                if a["slot"] != b["slot"] and max(a["device_begin_us"], b["device_begin_us"]) < \
                        min(a["device_end_us"], b["device_end_us"]):
                    overlapped = True
        assert all(r["latency_us"] > 0 and r["device_end_us"] > r["device_begin_us"] for r in res)
        if overlapped:
            break
    assert overlapped, res
    learner.serve_stop()
    learner.close()


def test_serving_admission_follows_the_memory_budget(L):
    """A budget that holds one slot of 256 rows runs one slot; a group larger than a slot is refused."""
    cfg = synth.make_config("small_b32")
    learner = L.Learner(cfg, None)
    rb = None
    learner.serve_start(max_rows=4096, mem_budget_bytes=1 << 34)
    big = learner.serve_info()
    learner.serve_stop()
    rb = big["arena_bytes"] / big["slots"] / ((big["slot_rows"] + 255) // 256 * 256)
    learner.serve_start(max_rows=4096, mem_budget_bytes=int(rb * 300))
    info = learner.serve_info()
    assert info["slots"] == 1 and info["slot_rows"] <= 300
    obs, prop, out = _batch(cfg, info["slot_rows"] + 1, 2)
    with pytest.raises(L.SquintError) as e:
        learner.serve_submit(L.Learner.request(obs, prop, out, key=1))
    assert e.value.code == L.EINVAL
    learner.serve_stop()
    learner.close()
