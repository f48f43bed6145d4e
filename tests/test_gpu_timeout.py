"""The bounded waits of the binning's look-backs (GPU only: the depth sort,
the emission and the tile sort): with the wait limit at 0 every partition
that has to look back gives up at once (the blocks return; nothing hangs),
the next gs_sync reports GS_ETIMEOUT and clears the status, and the same
context then bins correctly with the default limit."""
import numpy as np
import pytest
import torch

from paper_2509_05216_gb300 import gs, inputs
from tests.gpu_helpers import expected_binning

pytestmark = pytest.mark.gpu


def test_sort_wait_limit_reports_timeout_and_the_context_recovers():
    scene = inputs.random_scene(20000, 0, 21, extent=0.8)
    cams = [inputs.pinhole(inputs.look_at((0.4, -2.8, 1.0)), 256, 256)]
    ctx = gs.Context(0)
    try:
        p = torch.from_numpy(scene["params"]).cuda()
        assert ctx.gs_get_option(gs.GS_OPT_SORT_WAIT) == 1 << 20
        with pytest.raises(gs.GsError) as bad:
            ctx.gs_set_option(gs.GS_OPT_SORT_WAIT, -1)
        assert bad.value.status == gs.GS_EINVAL

        ctx.gs_set_option(gs.GS_OPT_SORT_WAIT, 0)
        ctx.gs_project(p, scene["n"], scene["deg"], cams)
        ctx.gs_bin_sort()
        inst, _, _ = ctx.gs_get_counts()
        # several partitions of 4096 keys in the view, so some must look back
        assert inst > 3 * 4096
        with pytest.raises(gs.GsError) as e:
            ctx.gs_sync()
        assert e.value.status == gs.GS_ETIMEOUT
        ctx.gs_sync()  # the status was cleared

        ctx.gs_set_option(gs.GS_OPT_SORT_WAIT, 1 << 20)
        ctx.gs_project(p, scene["n"], scene["deg"], cams)
        ctx.gs_bin_sort()
        ctx.gs_sync()
        keys = ctx.gs_get_buffer(gs.GS_BUF_KEYS).cpu().numpy().view(np.uint32)
        assert keys.size == inst and np.all(keys[1:] >= keys[:-1])
        stride = scene["params"].shape[1]
        r0 = ctx.gs_get_buffer(gs.GS_BUF_REC0).cpu().numpy()
        r2 = ctx.gs_get_buffer(gs.GS_BUF_REC2).cpu().numpy()
        r3 = ctx.gs_get_buffer(gs.GS_BUF_REC3).cpu().numpy()
        ek, ev, er, _ = expected_binning(r0, r2, r3, cams, scene["n"], stride)
        assert np.array_equal(keys, (ek >> np.uint64(32)).astype(np.uint32))
        assert np.array_equal(ctx.gs_get_buffer(gs.GS_BUF_VALS).cpu().numpy().astype(np.int64), ev)
    finally:
        ctx.close()
