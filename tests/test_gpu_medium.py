"""The 262,144-Gaussian workload at full size: rate control at 3, 4, 6 and 8 bits per texel
and the fused evaluation for one view direction per Gaussian from a camera centre.

Every output is compared with the oracle on the whole scene: the slot order, the rate
streams (lambda, bits, stream table, every block, final slot order), every decoded texel
(software and texture unit), and every Gaussian's colour within the SH tolerance of FP64.
The oracle codes the scene once on all host cores and runs the rate control per target.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

SH_TOL = 1e-5
TARGETS = (12, 16, 24, 32)


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def test_medium_scene_rate_targets_and_eval(ctx, O):
    from paper_2607_14513_gb300 import gsc
    sc = S.make_scene(**S.MEDIUM)
    n = sc.pos.shape[0]
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh)
    ctx.sync()
    osc = O.scales(sc.sh)
    q = O.quantise(sc.sh, osc)
    operm = O.plan(sc.pos, q, 4096, 1)
    assert np.array_equal(scales.cpu().numpy(), osc)
    assert np.array_equal(perm.cpu().numpy(), operm)
    refs = O.encode_rates(q, operm, osc, TARGETS, threads=os.cpu_count() or 1)
    cam = S.make_cams(1, 1102)  # one camera centre: one view direction per Gaussian
    for t4, ref in zip(TARGETS, refs):
        blocks, perm_out, tab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_RATE, t4)
        ctx.sync()
        rt = ref["table"]
        assert (tab.lambda_, tab.used_bits, tab.budget_bits) == (rt.lambda_, rt.used_bits, rt.budget_bits), t4
        assert [(tab.s[i].n_groups, tab.s[i].byte_offset) for i in range(14)] == \
            [(rt.s[i].n_groups, rt.s[i].byte_offset) for i in range(14)], t4
        assert np.array_equal(blocks.cpu().numpy(), ref["blocks"]), t4
        assert np.array_equal(perm_out.cpu().numpy(), ref["perm"]), t4
        tex_ref = O.decode(rt, ref["blocks"], ref["perm"])
        tex = gsc.gsc_decode(ctx, tab, blocks, perm_out)
        tex_hw = gsc.gsc_decode_tex(ctx, tab, blocks, perm_out)
        ctx.sync()
        assert np.array_equal(tex.cpu().numpy(), tex_ref), t4
        assert np.array_equal(tex_hw.cpu().numpy(), tex_ref), t4
        rgb = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, pos=pos, cams=torch.from_numpy(cam).cuda(),
                                     out_order=gsc.OUT_VIEW_MAJOR).cpu().numpy()
        out, ab = O.eval_sh(tex_ref, osc, pos=sc.pos, cams=cam, want_abs=True)
        assert np.all(np.abs(rgb.astype(np.float64) - out) <= SH_TOL * ab + 1e-30), t4
