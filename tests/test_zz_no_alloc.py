"""The allocation-free L1 entry point (gs_l1_loss_noalloc) against the
regular one (gs_l1_loss), through the C ABI, on two calls in a row.

gs_l1_loss_noalloc serves callers that may not allocate device memory (a host
that owns every allocation, a loop that must never allocate once running); it
keeps its partial sums in a static array instead of a context buffer.  This
file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_05216_gb300 import gs

pytestmark = pytest.mark.gpu


def test_noalloc_l1_matches_regular_l1_twice_in_a_row():
    ctx = gs.Context(0)
    rng = np.random.default_rng(11)
    for count in (1_000_003, 300_017):  # two calls in a row, different sizes
        x = torch.from_numpy(rng.uniform(size=count).astype(np.float32)).cuda()
        y = torch.from_numpy(rng.uniform(size=count).astype(np.float32)).cuda()
        y[::101] = x[::101]  # exact ties: sign(0) = 0
        loss_ref = torch.zeros(1, device="cuda")
        grad_ref = torch.zeros(count, device="cuda")
        ctx.gs_l1_loss(x, y, loss_ref, grad_ref)
        loss = torch.full((1,), float("nan"), device="cuda")
        grad = torch.full((count,), float("nan"), device="cuda")
        gs.gs_l1_loss_noalloc(x, y, loss, grad)
        torch.cuda.synchronize()
        assert abs(loss.item() - loss_ref.item()) <= 1e-6 * loss_ref.item()
        np.testing.assert_allclose(grad.cpu().numpy(), grad_ref.cpu().numpy(), rtol=1e-6, atol=0)
    ctx.close()


def test_noalloc_l1_rejects_counts_beyond_its_limit():
    L = gs.load()
    x = torch.zeros(4, device="cuda")
    # the count is checked on the host before anything is launched
    st = L.gs_l1_loss_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                              268_435_457, None, None, None)
    assert st == gs.GS_EINVAL
    st = L.gs_l1_loss_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 0, None, None, None)
    assert st == gs.GS_EINVAL
