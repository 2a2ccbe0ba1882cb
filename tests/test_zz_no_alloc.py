"""The allocation-free reorder plan (gsc_plan_reorder_static) against the workspace form.

Some callers cannot call cudaMalloc (a host framework that owns all device memory, or a
loop that must not allocate). For them the library keeps the plan's scratch in a static
device array. This file is collected last on purpose, so that a run which stops at the
first failure has already run every other test; it passes alone and after the others.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def _static_plan(ctx, pos, sh, group_size, sort):
    from paper_2607_14513_gb300 import gsc
    n = sh.shape[0]
    ns = (n + 15) // 16 * 16
    perm = torch.full((max(ns, 1),), -7, dtype=torch.int32, device="cuda")[:ns]
    scales = torch.zeros(16, dtype=torch.float32, device="cuda")
    pp = gsc.PlanParams(n, group_size, sort, 995)
    rc = ctx.lib.gsc_plan_reorder_static(ctx.h, gsc._ptr(pos), gsc._ptr(sh), ctypes.byref(pp), gsc._ptr(perm),
                                         gsc._ptr(scales), gsc._stream(None))
    return rc, perm, scales


def test_static_plan_matches_workspace_plan_twice(ctx):
    from paper_2607_14513_gb300 import gsc
    # two calls in a row on different scenes: the shared array keeps the previous contents,
    # and the second result must not depend on them
    for n, seed, gs in [(65536, 41, 4096), (3001, 42, 256)]:
        sc = S.make_scene(n, seed, clusters=6, heavy_frac=0.1)
        pos = torch.from_numpy(sc.pos).cuda()
        sh = torch.from_numpy(sc.sh).cuda()
        rc, perm_s, scales_s = _static_plan(ctx, pos, sh, gs, 1)
        assert rc == 0
        perm_w, scales_w = gsc.gsc_plan_reorder(ctx, pos, sh, group_size=gs, sort=1)
        ctx.sync()
        assert torch.equal(perm_s, perm_w)
        assert torch.equal(scales_s, scales_w)


def test_static_plan_rejects_oversize(ctx):
    n = 65537
    sh = torch.zeros((n, 16, 3), device="cuda")
    pos = torch.zeros((n, 3), device="cuda")
    rc, perm, _ = _static_plan(ctx, pos, sh, 4096, 1)
    assert rc == 1                                  # GSC_ERR_INVALID_ARG, nothing launched
    torch.cuda.synchronize()
    assert bool((perm == -7).all())
