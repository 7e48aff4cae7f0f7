"""The allocation-free conv weight gradient against the workspace entry point and the
FP64 oracle (needs a GB300).

Callers that cannot allocate device memory (a frozen pool, an allocator-free
real-time loop, a foreign allocator) use squint_op_conv3x3_wgrad_noalloc, whose
scratch is a fixed array in the library's device image.  This file runs last so
that a failure here cannot hide the result of any other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import squint_sac as o

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(L, x, dy, stride):
    n, cin, h, w = x.shape
    cout = dy.shape[1]
    dw = torch.full((cout, cin, 3, 3), float("nan"), device="cuda")
    db = torch.full((cout,), float("nan"), device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.squint_op_conv3x3_wgrad_noalloc(n, cin, h, w, cout, stride, _p(x), _p(dy), _p(dw), _p(db), stream)
    return rc, dw, db


def test_noalloc_weight_gradient_equals_workspace_entry_on_two_calls():
    from paper_2602_21203_gb300 import lib, ops
    L = lib.load()
    g = torch.Generator().manual_seed(123)
    # the encoder's second layer at the training shape (batch 512, 32 -> 32, 15x15), then a
    # stride-2 first layer shape: two calls in a row on the shared scratch array
    for n, cin, h, cout, stride in [(512, 32, 15, 32, 1), (64, 3, 32, 32, 2)]:
        x = torch.randn(n, cin, h, h, generator=g).cuda()
        oh = (h - 3) // stride + 1
        dy = torch.randn(n, cout, oh, oh, generator=g).cuda()
        w = torch.randn(cout, cin, 3, 3, generator=g).cuda()
        _, dw_ref, db_ref = ops.conv3x3_bwd(x, w, dy, stride, need_dx=False)
        rc, dw, db = _noalloc(L, x, dy, stride)
        torch.cuda.synchronize()
        assert rc == 0, L.squint_last_error().decode()
        for a, b in ((dw, dw_ref), (db, db_ref)):
            a, b = a.cpu().double().numpy(), b.cpu().double().numpy()
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
        # and against the FP64 oracle's weight gradient of the same operands
        _, dw_o, db_o = o.conv3x3_bwd(x.cpu().double().numpy(), w.cpu().double().numpy(),
                                      dy.cpu().double().numpy(), stride, need_dx=False)
        for a, b in ((dw, dw_o), (db, db_o)):
            a = a.cpu().double().numpy()
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


def test_noalloc_rejects_shapes_beyond_its_fixed_scratch():
    from paper_2602_21203_gb300 import lib
    L = lib.load()
    assert L.squint_op_conv3x3_wgrad_noalloc_max() == 1 << 20
    x = torch.zeros(4, 256, 16, 16, device="cuda")
    dy = torch.zeros(4, 256, 14, 14, device="cuda")
    rc, _, _ = _noalloc(L, x, dy, 1)
    assert rc == lib.EINVAL
    assert "scratch" in L.squint_last_error().decode()
