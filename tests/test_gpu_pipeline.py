"""End-to-end GPU path against the oracle through the C ABI: scales and quantisation
(Sec. V-A), reorder plan (Sec. III-C), layout-D encode (Sec. IV-B, Fig. SetupD), rate
control and streams (Sec. IV-B), decode through the inverse permutation, the texture
path, and FP32 SH evaluation against FP64 (Sec. II).

Bit-exact for every integer result; SH colour within 1e-5 of the absolute term sum.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

SH_TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,gs,srt", [(4096, 4096, 1), (1000, 256, 1), (17, 16, 1), (1, 16, 1), (333, 0, 1),
                                      (500, 4096, 0), (40000, 4096, 1)])
def test_plan_bit_exact(ctx, O, n, gs, srt):
    from paper_2607_14513_gb300 import gsc
    sc = S.make_scene(n, 500 + n, clusters=8)
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh), group_size=gs, sort=srt)
    ctx.sync()
    osc = O.scales(sc.sh)
    assert np.array_equal(scales.cpu().numpy(), osc)
    q = O.quantise(sc.sh, osc)
    assert np.array_equal(perm.cpu().numpy(), O.plan(sc.pos, q, gs, srt))
    gq = gsc.gsc_quantise(ctx, _dev(sc.sh), scales)
    assert np.array_equal(gq.cpu().numpy(), q)


def test_plan_empty_scene(ctx):
    from paper_2607_14513_gb300 import gsc
    perm, scales = gsc.gsc_plan_reorder(ctx, torch.zeros((0, 3), device="cuda"), torch.zeros((0, 16, 3), device="cuda"))
    ctx.sync()
    assert perm.numel() == 0 and torch.all(scales.cpu() == 1.0)


@pytest.mark.parametrize("fmt,n", [(1, 4096), (1, 4099), (7, 1000), (7, 33)])
def test_forced_encode_decode_bit_exact(ctx, O, fmt, n):
    from paper_2607_14513_gb300 import gsc
    sc = S.make_scene(n, 600 + n)
    ref = O.full_encode(sc.pos, sc.sh, fmt, group_size=1024)
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh), group_size=1024)
    blocks, perm_out, tab = gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, fmt)
    ctx.sync()
    assert tab.total_bytes == ref["table"].total_bytes and tab.n_streams == 1
    gb = blocks.cpu().numpy()
    bpb = 16 if fmt == 7 else 8
    bad = np.nonzero((gb.reshape(-1, bpb) != ref["blocks"].reshape(-1, bpb)).any(axis=1))[0]
    assert bad.size == 0, "first mismatching block %d" % bad[0]
    assert np.array_equal(perm_out.cpu().numpy(), ref["perm"])
    tex_ref = O.decode(ref["table"], ref["blocks"], ref["perm"])
    tex = gsc.gsc_decode(ctx, tab, blocks, perm_out)
    tex_hw = gsc.gsc_decode_tex(ctx, tab, blocks, perm_out)
    ctx.sync()
    assert np.array_equal(tex.cpu().numpy(), tex_ref)
    assert np.array_equal(tex_hw.cpu().numpy(), tex_ref)


@pytest.mark.parametrize("target_x4", [12, 16, 24, 32])
def test_rate_streams_bit_exact(ctx, O, target_x4):
    from paper_2607_14513_gb300 import gsc
    n = 2000
    sc = S.make_scene(n, 700, heavy_frac=0.1)
    ref = O.full_encode(sc.pos, sc.sh, 0, target_x4=target_x4, group_size=512)
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh), group_size=512)
    blocks, perm_out, tab = gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, gsc.FMT_RATE, target_x4)
    ctx.sync()
    rt = ref["table"]
    assert tab.lambda_ == rt.lambda_ and tab.used_bits == rt.used_bits and tab.budget_bits == rt.budget_bits
    assert [tab.s[i].n_groups for i in range(14)] == [rt.s[i].n_groups for i in range(14)]
    assert [tab.s[i].byte_offset for i in range(14)] == [rt.s[i].byte_offset for i in range(14)]
    assert list(tab.weights) == list(rt.weights)
    assert np.array_equal(blocks.cpu().numpy(), ref["blocks"])
    assert np.array_equal(perm_out.cpu().numpy(), ref["perm"])
    tex_ref = O.decode(rt, ref["blocks"], ref["perm"])
    tex = gsc.gsc_decode(ctx, tab, blocks, perm_out)
    tex_hw = gsc.gsc_decode_tex(ctx, tab, blocks, perm_out)
    ctx.sync()
    assert np.array_equal(tex.cpu().numpy(), tex_ref)
    assert np.array_equal(tex_hw.cpu().numpy(), tex_ref)
    # fused evaluation of the mixed streams (dropped coefficients decode to zero)
    dirs = S.make_dirs(5, 703)
    rgb = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, dirs=_dev(dirs))
    out, ab = O.eval_sh(tex_ref, ref["scales"], dirs=dirs, want_abs=True)
    ctx.sync()
    _check_sh(rgb.cpu().numpy(), out, ab)


@pytest.mark.parametrize("fmt,n", [(1, 300_000), (7, 40_000)])
def test_texture_path_spans_rows(ctx, O, fmt, n):
    # more blocks than one texture row (16384 blocks): the texture unit and the software
    # decoder agree on every texel, twice in a row (the cached arrays are reused), and
    # sampled groups match the oracle block for block
    from paper_2607_14513_gb300 import gsc
    sc = S.make_scene(n, 950 + fmt, heavy_frac=0.1)
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh))
    blocks, perm_out, tab = gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, fmt)
    for _ in range(2):
        tex = gsc.gsc_decode(ctx, tab, blocks, perm_out)
        tex_hw = gsc.gsc_decode_tex(ctx, tab, blocks, perm_out)
        ctx.sync()
        assert torch.equal(tex, tex_hw)
    q = O.quantise(sc.sh, scales.cpu().numpy())
    pc = perm_out.cpu().numpy()
    ng = pc.size // 16
    rng = np.random.default_rng(951)
    groups = np.unique(np.concatenate([[0, ng - 1], rng.integers(0, ng, size=14)]))
    st = O.stage(q, np.concatenate([pc[16 * g:16 * g + 16] for g in groups]))
    ob, _ = O.encode_blocks(st.reshape(-1, 16, 3), fmt)
    bpb = 16 if fmt == 7 else 8
    gb = blocks.cpu().numpy().reshape(ng, 16, bpb)[groups].reshape(-1, bpb)
    assert np.array_equal(gb, ob)


def test_decode_eval_at_scale(ctx, O):
    # 200k Gaussians, 8 cameras, every output order: FP32 against FP64 evaluated from the
    # GPU-decoded texels (the decode itself is pinned bit for bit elsewhere)
    from paper_2607_14513_gb300 import gsc
    n = 200_000
    sc = S.make_scene(n, 960, clusters=16)
    cams = S.make_cams(8, 961)
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh))
    blocks, perm_out, tab = gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, 1)
    tex = gsc.gsc_decode(ctx, tab, blocks, perm_out).cpu().numpy()
    sel = np.random.default_rng(962).choice(n, 3000, replace=False)
    out, ab = O.eval_sh(tex[sel], scales.cpu().numpy(), pos=sc.pos[sel], cams=cams, want_abs=True)
    pc = perm_out.cpu().numpy()
    slot_of = np.empty(n, np.int64)
    slot_of[pc[pc >= 0]] = np.nonzero(pc >= 0)[0]
    for order in (0, 1, 2):
        rgb = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, pos=_dev(sc.pos), cams=_dev(cams), out_order=order)
        ctx.sync()
        g = rgb.cpu().numpy()
        got = {0: lambda: g[:, sel], 1: lambda: g[:, slot_of[sel]], 2: lambda: g[sel].transpose(1, 0, 2)}[order]()
        _check_sh(got, out, ab)


@pytest.mark.parametrize("fmt,n", [(1, 50_000), (7, 20_000), (0, 6_000)])
def test_eval_through_texture_unit_equals_software(ctx, fmt, n):
    # texels fetched through the texture unit, dequantised exactly, same SH code: the colours
    # equal the software-decoded fused kernel bit for bit, in every order and direction mode
    from paper_2607_14513_gb300 import gsc
    sc = S.make_scene(n, 970 + fmt, heavy_frac=0.1)
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh))
    blocks, perm_out, tab = gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, fmt, 16 if fmt == 0 else 0)
    dirs, cams, pos = _dev(S.make_dirs(3, 971)), _dev(S.make_cams(8, 972)), _dev(sc.pos)
    scene = gsc.TexScene(ctx, tab, blocks)                       # positions gathered per call
    scene_p = gsc.TexScene(ctx, tab, blocks, perm_out, pos)      # positions resident in slot order
    for order in (0, 1, 2):
        for kw in (dict(dirs=dirs), dict(pos=pos, cams=cams)):
            a = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, out_order=order, **kw)
            b = gsc.gsc_decode_eval_sh_tex(ctx, scene, perm_out, out_order=order, **kw)
            kw2 = dict(kw)
            kw2.pop("pos", None)
            c = gsc.gsc_decode_eval_sh_tex(ctx, scene_p, perm_out, out_order=order, **kw2)
            ctx.sync()
            assert torch.equal(a, b)
            assert torch.equal(a, c)
    # odd view counts take the unvectorised store path
    a = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, dirs=_dev(S.make_dirs(5, 973)), out_order=2)
    b = gsc.gsc_decode_eval_sh_tex(ctx, scene_p, perm_out, dirs=_dev(S.make_dirs(5, 973)), out_order=2)
    ctx.sync()
    assert torch.equal(a, b)
    scene.close()
    scene_p.close()


def test_rate_budget_error(ctx):
    from paper_2607_14513_gb300 import gsc
    sc = S.make_scene(500, 701)                    # 32 groups: the cheapest coding needs 2048 bits > 4 * 500
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh))
    with pytest.raises(gsc.GscError) as e:
        gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, gsc.FMT_RATE, 0 + 1)   # 0.25 bpt: below 64 bits / group
    assert e.value.code == 4


def _check_sh(got, ref, ab):
    err = np.abs(got.astype(np.float64) - ref)
    bound = SH_TOL * ab + 1e-30
    worst = np.max(err / bound)
    assert np.all(err <= bound), "worst error / bound = %g" % worst


@pytest.mark.parametrize("fmt", [1, 7])
def test_decode_eval_sh_tolerance(ctx, O, fmt):
    from paper_2607_14513_gb300 import gsc
    n = 4096 if fmt == 1 else 600
    sc = S.make_scene(n, 800 + fmt)
    dirs = S.make_dirs(16, 801)
    cams = S.make_cams(3, 802)
    ref = O.full_encode(sc.pos, sc.sh, fmt)
    tex = O.decode(ref["table"], ref["blocks"], ref["perm"])
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh))
    blocks, perm_out, tab = gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, fmt)
    # shared directions, view-major original order
    rgb = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, dirs=_dev(dirs))
    out, ab = O.eval_sh(tex, ref["scales"], dirs=dirs, want_abs=True)
    ctx.sync()
    _check_sh(rgb.cpu().numpy(), out, ab)
    # camera centres, all three output orders
    out, ab = O.eval_sh(tex, ref["scales"], pos=sc.pos, cams=cams, want_abs=True)
    pc = perm_out.cpu().numpy()
    for order in (0, 1, 2):
        rgb = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, pos=_dev(sc.pos), cams=_dev(cams), out_order=order)
        ctx.sync()
        g = rgb.cpu().numpy()
        if order == 1:
            valid = pc >= 0
            g2 = np.zeros((3, n, 3), np.float32)
            g2[:, pc[valid]] = g[:, valid]
            assert np.all(g[:, ~valid] == 0)
            g = g2
        elif order == 2:
            g = g.transpose(1, 0, 2)
        _check_sh(g, out, ab)


def test_decode_eval_camera_on_gaussian(ctx, O):
    from paper_2607_14513_gb300 import gsc
    sc = S.make_scene(64, 900)
    cams = sc.pos[:2].copy()                      # cameras exactly on two Gaussians: direction +z
    ref = O.full_encode(sc.pos, sc.sh, 1)
    tex = O.decode(ref["table"], ref["blocks"], ref["perm"])
    perm, scales = gsc.gsc_plan_reorder(ctx, _dev(sc.pos), _dev(sc.sh))
    blocks, perm_out, tab = gsc.gsc_encode(ctx, _dev(sc.sh), perm, scales, 1)
    rgb = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, pos=_dev(sc.pos), cams=_dev(cams))
    out, ab = O.eval_sh(tex, ref["scales"], pos=sc.pos, cams=cams, want_abs=True)
    ctx.sync()
    _check_sh(rgb.cpu().numpy(), out, ab)


def test_invalid_arguments(ctx):
    from paper_2607_14513_gb300 import gsc
    import ctypes
    lib = ctx.lib
    pp = gsc.PlanParams(100, 24, 1, 995)                     # group size not a multiple of 16
    sh = torch.zeros((100, 16, 3), device="cuda")
    perm = torch.zeros(112, dtype=torch.int32, device="cuda")
    scales = torch.zeros(16, device="cuda")
    ws = ctx.workspace(100)
    rc = lib.gsc_plan_reorder(ctx.h, gsc._ptr(sh), gsc._ptr(sh), ctypes.byref(pp), gsc._ptr(perm), gsc._ptr(scales),
                              gsc._ptr(ws), ws.numel(), None)
    assert rc == 1
    pp = gsc.PlanParams(100, 16, 1, 995)
    rc = lib.gsc_plan_reorder(ctx.h, gsc._ptr(sh), gsc._ptr(sh), ctypes.byref(pp), gsc._ptr(perm), gsc._ptr(scales),
                              gsc._ptr(ws), 16, None)
    assert rc == 3                                            # workspace too small
    tab = gsc.StreamTable()
    rc = lib.gsc_decode(ctx.h, ctypes.byref(tab), None, None, None, None)
    assert rc == 1                                            # empty table is invalid
