"""Layouts A and B (Figs. SetupA / SetupB) and the fixed BC7/BC1 mixes of Table I, through the
C-ABI: blocks bit for bit against the oracle, software and texture-unit decode against the
oracle decoder, fused evaluation against the FP64 oracle (and texture == software bit for bit),
and the argument checks of the layout fields."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

SH_TOL = 1e-5
D, A, B = 0, 1, 2
# (layout, format, BC7 blocks per group): Table I's A-BC1, A-BC7, B "BC7 on the first block",
# B all-BC1 / all-BC7, and layout D with BC7 on block 0 / blocks 0-3
CODINGS = [(A, 1, 0), (A, 7, 16), (B, 2, 4), (B, 1, 0), (B, 7, 16), (B, 2, 12), (D, 2, 1), (D, 2, 4)]


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def scene(ctx, O):
    from paper_2607_14513_gb300 import gsc
    n = 2003                      # 126 groups, the last with 3 valid slots
    sc = S.make_scene(**S.TINY)
    pos, sh = sc.pos[:n].copy(), sc.sh[:n].copy()
    dpos, dsh = torch.from_numpy(pos).cuda(), torch.from_numpy(sh).cuda()
    perm, scales = gsc.gsc_plan_reorder(ctx, dpos, dsh)
    osc = O.scales(sh)
    q = O.quantise(sh, osc)
    assert np.array_equal(perm.cpu().numpy(), O.plan(pos, q, 4096, 1))
    return dict(n=n, pos=pos, sh=sh, dpos=dpos, dsh=dsh, perm=perm, scales=scales, osc=osc, q=q)


@pytest.mark.parametrize("lay,fmt,j", CODINGS)
def test_layout_coding_matches_oracle(ctx, O, scene, lay, fmt, j):
    from paper_2607_14513_gb300 import gsc
    n = scene["n"]
    blk, po, tab = gsc.gsc_encode(ctx, scene["dsh"], scene["perm"], scene["scales"], fmt, layout=lay, bc7_blocks=j)
    ctx.sync()
    ref = O.encode_layout(scene["q"], scene["perm"].cpu().numpy(), scene["osc"], lay, j)
    assert tab.layout == lay and tab.n_streams == 1 and tab.s[0].bc7_blocks == j and tab.s[0].bands == 16
    assert tab.total_bytes == ref["table"].total_bytes == ((n + 15) // 16) * (16 * j + 8 * (16 - j))
    assert np.array_equal(blk.cpu().numpy(), ref["blocks"])
    assert torch.equal(po, scene["perm"])

    # decoders: software and texture unit against the oracle decoder
    want = O.decode(ref["table"], ref["blocks"], ref["perm"])
    sw = gsc.gsc_decode(ctx, tab, blk, po)
    hw = gsc.gsc_decode_tex(ctx, tab, blk, po)
    ctx.sync()
    assert np.array_equal(sw.cpu().numpy(), want)
    assert torch.equal(sw, hw)

    # fused evaluation: 5 cameras, every output order, against FP64; texture path == software path
    cams = S.make_cams(5, 1200 + lay)
    dc = torch.from_numpy(cams).cuda()
    out, ab = O.eval_sh(want, scene["osc"], pos=scene["pos"], cams=cams, want_abs=True)   # [V][n][3]
    tex_scene = gsc.TexScene(ctx, tab, blk, perm=po, pos=scene["dpos"])
    try:
        for order in (gsc.OUT_VIEW_MAJOR, gsc.OUT_GAUSS_MAJOR, gsc.OUT_SLOT_ORDER):
            a = gsc.gsc_decode_eval_sh(ctx, tab, blk, po, pos=scene["dpos"], cams=dc, out_order=order)
            b = gsc.gsc_decode_eval_sh_tex(ctx, tex_scene, po, cams=dc, out_order=order)
            ctx.sync()
            assert torch.equal(a, b), order
            got = a.cpu().numpy().astype(np.float64)
            if order == gsc.OUT_GAUSS_MAJOR:
                got = got.transpose(1, 0, 2)
            elif order == gsc.OUT_SLOT_ORDER:
                pp = po.cpu().numpy()
                valid = pp >= 0
                full = np.zeros_like(out)
                full[:, pp[valid]] = got[:, valid]
                assert np.all(got[:, ~valid] == 0.0)
                got = full
            assert np.all(np.abs(got - out) <= SH_TOL * ab + 1e-30), order
    finally:
        tex_scene.close()


def test_layout_arguments_are_checked(ctx, scene):
    from paper_2607_14513_gb300 import gsc
    args = (ctx, scene["dsh"], scene["perm"], scene["scales"])
    for fmt, lay, j in ((gsc.FMT_MIXED, A, 4), (gsc.FMT_MIXED, B, 2), (gsc.FMT_MIXED, B, 20), (gsc.FMT_RATE, B, 0),
                        (gsc.FMT_RATE, A, 0), (gsc.FMT_BC7, 3, 0), (gsc.FMT_MIXED, D, 17), (gsc.FMT_MIXED, D, -1)):
        with pytest.raises(gsc.GscError) as e:
            gsc.gsc_encode(*args, fmt, 16, layout=lay, bc7_blocks=j)
        assert e.value.code == 1, (fmt, lay, j)
    # a too-small workspace is reported, not overrun
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(gsc.GscError) as e:
        gsc.gsc_encode(*args, gsc.FMT_MIXED, layout=B, bc7_blocks=4, ws=small)
    assert e.value.code == 3
    # a table whose layout and BC7 count do not fit together is rejected by the decoders
    blk, po, tab = gsc.gsc_encode(*args, gsc.FMT_MIXED, layout=B, bc7_blocks=4)
    tab.s[0].bc7_blocks = 6
    tab.total_bytes = tab.n_groups * (16 * 6 + 8 * 10)
    with pytest.raises(gsc.GscError) as e:
        gsc.gsc_decode(ctx, tab, blk, po)
    assert e.value.code == 1
    tab.s[0].bc7_blocks, tab.total_bytes, tab.layout = 4, tab.n_groups * 160, 5
    with pytest.raises(gsc.GscError) as e:
        gsc.gsc_decode(ctx, tab, blk, po)
    assert e.value.code == 1


@pytest.mark.parametrize("lay,fmt,j", [(A, 7, 16), (B, 2, 4)])
def test_full_size_sampled_groups(ctx, O, lay, fmt, j):
    # the 3M-Gaussian scene of the default workload: sampled groups' blocks against the oracle's
    # encoder on the same staged texels, and their decoded texels through both decoders
    from paper_2607_14513_gb300 import gsc
    cfg = dict(S.SCENE)
    n = cfg["n"]
    sc = S.make_scene(**cfg)
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh)
    blk, po, tab = gsc.gsc_encode(ctx, sh, perm, scales, fmt, layout=lay, bc7_blocks=j)
    ctx.sync()
    ng = (n + 15) // 16
    gbytes = 16 * j + 8 * (16 - j)
    assert tab.total_bytes == ng * gbytes
    osc = O.scales(sc.sh)
    assert np.array_equal(scales.cpu().numpy(), osc)
    pp = perm.cpu().numpy()
    rng = np.random.default_rng(2000 + lay)
    groups = np.unique(np.concatenate([[0, ng - 1], rng.integers(0, ng, size=46)]))
    sub = np.concatenate([pp[16 * g:16 * g + 16] for g in groups])
    # the oracle stages the sampled groups from the full quantised scene (slot entries index it)
    q = O.quantise(sc.sh, osc)
    st = O.stage_layout(q, sub, lay)                      # [len(groups), 16, 16, 3]
    k7 = [k for k in range(16) if O.layout_bc7(lay, j, k)]
    k1 = [k for k in range(16) if not O.layout_bc7(lay, j, k)]
    gb = blk.cpu().numpy().reshape(ng, gbytes)[groups]
    if k7:
        ob7 = np.asarray(O.encode_blocks(st[:, k7].reshape(-1, 16, 3), 7)[0]).reshape(len(groups), -1)
        assert np.array_equal(gb[:, :16 * len(k7)], ob7)
    if k1:
        ob1 = np.asarray(O.encode_blocks(st[:, k1].reshape(-1, 16, 3), 1)[0]).reshape(len(groups), -1)
        assert np.array_equal(gb[:, 16 * len(k7):], ob1)
    sw = gsc.gsc_decode(ctx, tab, blk, po)
    hw = gsc.gsc_decode_tex(ctx, tab, blk, po)
    ctx.sync()
    assert torch.equal(sw, hw)
