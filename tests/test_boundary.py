"""The C-ABI library builds, loads and exports every declared symbol (no GPU needed).

These tests call only entry points that do no device work: presets, parameter
counts, struct sizes, error strings and argument validation.
"""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import squint_sac as o
from paper_2602_21203_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_21203_gb300 import build, lib as L
    if not os.path.exists(L.LIB_PATH):
        build.build()
    return L


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(squint_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol(lib):
    L = lib.load()
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in sorted(declared) if not hasattr(L, n)]
    assert not missing, missing


def test_struct_layouts_match(lib):
    L = lib.load()
    assert L.squint_struct_size(b"squint_config") == ctypes.sizeof(lib.Config)
    assert L.squint_struct_size(b"squint_replay") == ctypes.sizeof(lib.Replay)
    assert L.squint_struct_size(b"squint_update_stats") == ctypes.sizeof(lib.UpdateStats)
    assert L.squint_struct_size(b"squint_act_request") == ctypes.sizeof(lib.ActRequest)
    assert L.squint_struct_size(b"squint_serve_result") == ctypes.sizeof(lib.ServeResult)
    assert L.squint_struct_size(b"nope") == 0


@pytest.mark.parametrize("name", ["small_b32", "train_b512", "tiny_b8"])
def test_param_layout_matches_oracle(lib, name):
    cfg = synth.make_config(name)
    n_oracle = sum(int(np.prod(s)) for _, s, _, _ in o.param_spec(cfg))
    assert lib.param_count(cfg) == n_oracle


@pytest.mark.parametrize("name", ["small_b32", "train_b512", "tiny_b8"])
def test_presets_match_workload_configs(lib, name):
    L = lib.load()
    c = lib.Config()
    assert L.squint_config_preset(name.encode(), ctypes.byref(c)) == 0
    ref = lib.make_config(synth.make_config(name))
    for f, _ in lib.Config._fields_:
        a, b = getattr(c, f), getattr(ref, f)
        if f == "max_k":
            continue
        if isinstance(a, float):
            assert (math.isnan(a) and math.isnan(b)) or a == b, f
        elif hasattr(a, "__len__"):
            assert list(a)[:len(synth.make_config(name)["hidden"])] == list(b)[:len(synth.make_config(name)["hidden"])], f
        else:
            assert a == b, f


def test_invalid_configs_are_rejected_without_a_device(lib):
    L = lib.load()
    bad = [
        dict(squint_f=3),          # 64 not divisible by 3
        dict(n_critics=3),
        dict(atoms=1),
        dict(batch=0),
        dict(v_min=5.0, v_max=5.0),
        dict(conv_layers=9),
    ]
    for over in bad:
        cfg = synth.make_config("small_b32", **over)
        c = lib.make_config(cfg) if over.get("conv_layers", 0) <= 8 else None
        if c is None:
            c = lib.make_config(synth.make_config("small_b32"))
            c.conv_layers = 9
        assert L.squint_param_count(ctypes.byref(c)) == -1
        h = ctypes.c_void_p()
        assert L.squint_create(ctypes.byref(c), None, ctypes.byref(h)) == lib.EINVAL
        assert not h.value
    assert L.squint_config_preset(b"unknown", ctypes.byref(lib.Config())) == lib.EINVAL
    assert L.squint_destroy(None) == 0
    assert L.squint_update(None, 1, None, None) == lib.EINVAL
    assert L.squint_set_debug(None, b"wait_cycles", 100) == lib.EINVAL
    assert L.squint_strerror(lib.ETIMEOUT).decode() == "timed out"
