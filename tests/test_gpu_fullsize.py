"""The bench's own workload at full size, in the launch configuration bench.py times.

3,000,000 Gaussians (64 clusters, 10% heavy tail), reorder plan, rate-controlled encode at
6 bits per texel that also keeps the all-BC1 and all-BC7 codings, software and texture-unit
decode, fused decode + SH evaluation for 8 cameras into Gaussian-major rows. The oracle
checks what it can compute one by one at this size: scales, quantised texels and the whole
slot order bit for bit; sampled groups' BC1 and BC7 blocks against its encoder; the rate
streams of the sampled groups decoded as their mode dictates (BC7 bands, BC1 bands, dropped
bands = 128); every texel of the texture path against the software decoder; and the FP32
colours of the sampled groups' Gaussians against its FP64 evaluation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

SH_TOL = 1e-5
RATE_TARGET_X4 = 24
N_CAMS = 8


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def test_scene_scale_step(ctx, O):
    from paper_2607_14513_gb300 import gsc
    cfg = dict(S.SCENE)
    n = cfg["n"]
    sc = S.make_scene(**cfg)
    cams = S.make_cams(N_CAMS, 1100)
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    ng = (n + 15) // 16
    bc1 = torch.empty(ng * 128, dtype=torch.uint8, device="cuda")
    bc7 = torch.empty(ng * 256, dtype=torch.uint8, device="cuda")
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh)
    rblk, rperm, rtab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_RATE, RATE_TARGET_X4, bc1_all=bc1, bc7_all=bc7)
    ctx.sync()

    # scales, texels and the whole slot order
    osc = O.scales(sc.sh)
    assert np.array_equal(scales.cpu().numpy(), osc)
    q = O.quantise(sc.sh, osc)
    assert np.array_equal(gsc.gsc_quantise(ctx, sh, scales).cpu().numpy(), q)
    pp = perm.cpu().numpy()
    assert np.array_equal(pp, O.plan(sc.pos, q, 4096, 1))

    # sampled groups (first, last, 62 random) of both full codings against the oracle encoder
    rng = np.random.default_rng(1004)
    groups = np.unique(np.concatenate([[0, ng - 1], rng.integers(0, ng, size=62)]))
    st = O.stage(q, np.concatenate([pp[16 * g:16 * g + 16] for g in groups])).reshape(-1, 16, 3)
    ob1, _ = O.encode_blocks(st, 1)
    ob7, _ = O.encode_blocks(st, 7)
    gb1 = bc1.cpu().numpy().reshape(ng, 16, 8)[groups].reshape(-1, 8)
    gb7 = bc7.cpu().numpy().reshape(ng, 16, 16)[groups].reshape(-1, 16)
    assert np.array_equal(gb1, np.asarray(ob1).reshape(-1, 8))
    assert np.array_equal(gb7, np.asarray(ob7).reshape(-1, 16))

    # rate streams: budget, and each sampled group decodes as its stream's mode says
    assert rtab.used_bits <= RATE_TARGET_X4 * 4 * n
    rp = rperm.cpu().numpy()
    first_slot = {int(rp[16 * g2]): g2 for g2 in range(ng)}
    mode_of = np.zeros((ng, 2), np.int64)
    for s in rtab.streams():
        mode_of[s["first_group"]:s["first_group"] + s["n_groups"]] = (s["bands"], s["bc7_blocks"])
    tex_rate = gsc.gsc_decode(ctx, rtab, rblk, rperm).cpu().numpy()
    dec1 = O.decode_blocks(np.asarray(ob1).reshape(-1, 8), 1)[:, :, :3].reshape(len(groups), 16, 16, 3)
    dec7 = O.decode_blocks(np.asarray(ob7).reshape(-1, 16), 7)[:, :, :3].reshape(len(groups), 16, 16, 3)
    for gi, g in enumerate(groups):
        b, j = mode_of[first_slot[int(pp[16 * g])]]
        for t in range(16):
            o = pp[16 * g + t]
            if o < 0:
                continue
            want = np.full((16, 3), 128, np.uint8)
            want[:j] = dec7[gi, :j, t]
            want[j:b] = dec1[gi, j:b, t]
            assert np.array_equal(tex_rate[o], want), (g, t, b, j)

    # texture unit against the software decoder, every texel, both full codings
    t1, t7 = gsc.forced_table(rtab, gsc.FMT_BC1), gsc.forced_table(rtab, gsc.FMT_BC7)
    for tab, blk in ((t7, bc7), (t1, bc1)):
        sw = gsc.gsc_decode(ctx, tab, blk, perm)
        hw = gsc.gsc_decode_tex(ctx, tab, blk, perm)
        ctx.sync()
        assert torch.equal(sw, hw)

    # fused evaluation, 8 cameras, Gaussian-major: the sampled groups' Gaussians against FP64
    dc = torch.from_numpy(cams).cuda()
    for tab, blk, dec in ((t7, bc7, dec7), (t1, bc1, dec1)):
        rgb = gsc.gsc_decode_eval_sh(ctx, tab, blk, perm, pos=pos, cams=dc, out_order=gsc.OUT_GAUSS_MAJOR).cpu().numpy()
        sel, texels = [], []
        for gi, g in enumerate(groups):
            for t in range(16):
                o = pp[16 * g + t]
                if o >= 0:
                    sel.append(o)
                    texels.append(dec[gi, :, t])
        sel = np.array(sel)
        out, ab = O.eval_sh(np.stack(texels), osc, pos=sc.pos[sel], cams=cams, want_abs=True)
        got = rgb[sel].transpose(1, 0, 2).astype(np.float64)
        assert np.all(np.abs(got - out) <= SH_TOL * ab + 1e-30)
