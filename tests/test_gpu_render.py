"""The splatting renderer through the C-ABI (Sec. II, Fig. GSRend) against the oracle: the
(Gaussian, tile) overlap count exactly (every culling and footprint decision), and every pixel's
colour and transmittance within the FP32 bound, for several codings, cameras and image sizes;
the degenerate cases; and sampled tiles of the 3M-Gaussian scene at 1080p."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

# FP32 blending of a few hundred splats per pixel against FP64: relative to the sum of the
# absolute terms, plus a floor for pixels whose terms cancel
IMG_TOL, IMG_FLOOR, TR_TOL = 1e-4, 1e-6, 2e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def scene(ctx, O):
    from paper_2607_14513_gb300 import gsc
    n = 2003
    sc = S.make_scene(**S.TINY)
    pos, sh = sc.pos[:n].copy(), sc.sh[:n].copy()
    geo = S.make_geometry(n, 77, scale=0.02)
    d = dict(n=n, pos=pos, sh=sh, geo=geo, dpos=torch.from_numpy(pos).cuda(), dsh=torch.from_numpy(sh).cuda(),
             dscale=torch.from_numpy(geo.scale).cuda(), drot=torch.from_numpy(geo.rot).cuda(),
             dlogit=torch.from_numpy(geo.logit).cuda())
    d["perm"], d["scales"] = gsc.gsc_plan_reorder(ctx, d["dpos"], d["dsh"])
    d["osc"] = O.scales(sh)
    return d


def _oracle_image(O, d, table_o, blocks, perm, cam, tiles=None):
    tex = O.decode(table_o, blocks, perm)
    f = O.camera_centre(cam)
    colour = O.eval_sh(tex, d["osc"], pos=d["pos"], cams=f[None, :])[0]
    return O.render(d["pos"], d["geo"].scale, d["geo"].rot, d["geo"].logit, colour, cam, tiles=tiles, want_abs=True)


def _pairs(O, d, cam):
    n = 0
    for i in range(d["n"]):
        sp = O.splat_setup(d["pos"][i], d["geo"].scale[i], d["geo"].rot[i], cam)
        if sp.visible:
            n += (sp.x1 - sp.x0) * (sp.y1 - sp.y0)
    return n


def _check(img, tr, ref):
    want, wtr, ab = ref
    img, tr = img.cpu().numpy().astype(np.float64), tr.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(img - want) <= IMG_TOL * ab + IMG_FLOOR)
    assert np.all(np.abs(tr - wtr) <= TR_TOL)


@pytest.mark.parametrize("coding", ["bc7", "rate", "b_mixed"])
def test_render_matches_oracle(ctx, O, scene, coding):
    from paper_2607_14513_gb300 import gsc
    args = (ctx, scene["dsh"], scene["perm"], scene["scales"])
    if coding == "bc7":
        blk, po, tab = gsc.gsc_encode(*args, gsc.FMT_BC7)
    elif coding == "rate":
        blk, po, tab = gsc.gsc_encode(*args, gsc.FMT_RATE, 24)
    else:
        blk, po, tab = gsc.gsc_encode(*args, gsc.FMT_MIXED, layout=gsc.LAYOUT_B, bc7_blocks=4)
    ctx.sync()
    # the oracle decodes the same blocks (their equality with the oracle's coders is tested elsewhere)
    tab_o = O.Table()
    tab_o.n_streams, tab_o.n, tab_o.n_groups, tab_o.layout = tab.n_streams, tab.n, tab.n_groups, tab.layout
    for i in range(tab.n_streams):
        tab_o.s[i].bands, tab_o.s[i].bc7_blocks = tab.s[i].bands, tab.s[i].bc7_blocks
        tab_o.s[i].first_group, tab_o.s[i].n_groups = tab.s[i].first_group, tab.s[i].n_groups
        tab_o.s[i].byte_offset = tab.s[i].byte_offset
    blocks, perm = blk.cpu().numpy(), po.cpu().numpy()
    r = gsc.Renderer(ctx)
    for k, (w, h) in enumerate([(160, 120), (100, 37), (64, 64)]):
        cam = S.make_views(1, 500 + k, w, h, radius=1.6)[0]
        tr = torch.empty((h, w), dtype=torch.float32, device="cuda")
        img, tr, pairs = r.render(tab, blk, po, scene["dpos"], scene["dscale"], scene["drot"], scene["dlogit"], cam,
                                  trans=tr)
        ctx.sync()
        assert pairs == _pairs(O, scene, cam) and pairs > 0
        _check(img, tr, _oracle_image(O, scene, tab_o, blocks, perm, cam))


def test_render_degenerate_cases(ctx, scene):
    from paper_2607_14513_gb300 import gsc
    blk, po, tab = gsc.gsc_encode(ctx, scene["dsh"], scene["perm"], scene["scales"], gsc.FMT_BC1)
    ctx.sync()
    r = gsc.Renderer(ctx)
    # looking away from the scene: nothing in front of the camera
    cam = S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, -3.0], 48, 40)
    tr = torch.empty((40, 48), dtype=torch.float32, device="cuda")
    img, tr, pairs = r.render(tab, blk, po, scene["dpos"], scene["dscale"], scene["drot"], scene["dlogit"], cam,
                              trans=tr)
    ctx.sync()
    assert pairs == 0 and torch.all(img == 0) and torch.all(tr == 1)
    # a workspace too small for the overlaps is reported with the count, and nothing is written
    cam = S.make_views(1, 500, 160, 120, radius=1.6)[0]
    c = gsc.camera(cam)
    nb = ctx.lib.gsc_render_workspace_bytes(tab.n, C_byref(c), 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out = torch.full((120, 160, 3), 7.0, device="cuda")
    pairs = C_int64()
    code = ctx.lib.gsc_render(ctx.h, C_byref(tab), gsc._ptr(blk), gsc._ptr(po), gsc._ptr(scene["dpos"]),
                              gsc._ptr(scene["dscale"]), gsc._ptr(scene["drot"]), gsc._ptr(scene["dlogit"]),
                              C_byref(c), gsc._ptr(out), None, C_byref(pairs), gsc._ptr(ws), ws.numel(), None)
    ctx.sync()
    assert code == 3 and pairs.value > 1 and torch.all(out == 7.0)
    # bad cameras
    bad = dict(cam, width=0)
    with pytest.raises(gsc.GscError):
        r.render(tab, blk, po, scene["dpos"], scene["dscale"], scene["drot"], scene["dlogit"], bad)
    bad = dict(cam, near_z=0.0)
    with pytest.raises(gsc.GscError):
        r.render(tab, blk, po, scene["dpos"], scene["dscale"], scene["drot"], scene["dlogit"], bad)


def C_byref(x):
    import ctypes
    return ctypes.byref(x)


def C_int64():
    import ctypes
    return ctypes.c_int64(0)


def test_render_full_size_sampled_tiles(ctx, O):
    # the 3M-Gaussian scene (all-BC7) at 1920 x 1080, as the render workload draws it; 12 tiles
    # (corners, centre, random) against the oracle
    from paper_2607_14513_gb300 import gsc
    cfg = S.RENDER
    sc = S.make_scene(n=cfg["n"], seed=cfg["seed"], clusters=cfg["clusters"], heavy_frac=cfg["heavy_frac"])
    geo = S.make_geometry(cfg["n"], cfg["geom_seed"], scale=cfg["scale"])
    cam = S.make_views(cfg["views"], cfg["view_seed"], cfg["width"], cfg["height"])[0]
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh)
    blk, po, tab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_BC7)
    r = gsc.Renderer(ctx)
    tr = torch.empty((cfg["height"], cfg["width"]), dtype=torch.float32, device="cuda")
    img, tr, pairs = r.render(tab, blk, po, pos, torch.from_numpy(geo.scale).cuda(), torch.from_numpy(geo.rot).cuda(),
                              torch.from_numpy(geo.logit).cuda(), cam, trans=tr)
    ctx.sync()
    tx, ty = (cfg["width"] + 15) // 16, (cfg["height"] + 15) // 16
    rng = np.random.default_rng(31)
    tiles = np.unique(np.concatenate([[0, tx - 1, (ty - 1) * tx, tx * ty - 1, (ty // 2) * tx + tx // 2],
                                      rng.integers(0, tx * ty, size=7)])).astype(np.int32)
    osc = O.scales(sc.sh)
    tab_o = O.Table()
    tab_o.n_streams, tab_o.n, tab_o.n_groups = 1, tab.n, tab.n_groups
    tab_o.s[0].bands, tab_o.s[0].bc7_blocks, tab_o.s[0].n_groups = 16, 16, tab.n_groups
    tex = O.decode(tab_o, blk.cpu().numpy(), po.cpu().numpy())
    colour = O.eval_sh(tex, osc, pos=sc.pos, cams=O.camera_centre(cam)[None, :])[0]
    want, wtr, ab = O.render(sc.pos, geo.scale, geo.rot, geo.logit, colour, cam, tiles=tiles, want_abs=True)
    got, gtr = img.cpu().numpy().astype(np.float64), tr.cpu().numpy().astype(np.float64)
    for t in tiles:
        y, x = divmod(int(t), tx)
        sl = (slice(16 * y, 16 * y + 16), slice(16 * x, 16 * x + 16))
        assert np.all(np.abs(got[sl] - want[sl]) <= IMG_TOL * ab[sl] + IMG_FLOOR), t
        assert np.all(np.abs(gtr[sl] - wtr[sl]) <= TR_TOL), t
