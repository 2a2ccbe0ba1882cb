"""Geometry streams and chunk hierarchy through the C-ABI (Sec. IV-A): every code and chunk box
bit for bit against the oracle, and the render of a fully coded scene (colour blocks + geometry
streams, chunks culled by the view test) against the oracle's render of the decoded geometry of
the kept chunks: the kept chunk count and overlap count exactly, pixels within the FP32 bound;
then sampled tiles of the 3M-Gaussian scene at 1080p."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

IMG_TOL, IMG_FLOOR, TR_TOL = 1e-4, 1e-6, 2e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def _codes(gsc, geom, ns, chunk_slots):
    off, _ = gsc.geometry_layout(ns, chunk_slots)
    b = geom.cpu().numpy()
    nc = (ns + chunk_slots - 1) // chunk_slots
    return dict(qpos=b[off[0]:off[0] + 6 * ns].view(np.uint16).reshape(ns, 3),
                qscale=b[off[1]:off[1] + 6 * ns].view(np.uint16).reshape(ns, 3),
                qrot=b[off[2]:off[2] + 4 * ns].view(np.uint32), qlogit=b[off[3]:off[3] + ns],
                chunk=b[off[4]:off[4] + 32 * nc].view(np.float32).reshape(nc, 8), chunk_slots=chunk_slots)


def _oracle_coded_render(O, sc_pos, tex_orig, osc, perm, g, cam, tiles=None):
    """The oracle's image of the decoded geometry of the kept chunks (colour for the decoded centres)."""
    P, Sc, Q, T = O.geometry_decode(g)
    ns, cs = perm.shape[0], g["chunk_slots"]
    keep = np.array([O.chunk_visible(g["chunk"][c], cam) for c in range(g["chunk"].shape[0])])
    slots = np.array([s for s in range(ns) if perm[s] >= 0 and keep[s // cs]], np.int64)
    order = np.argsort(perm[slots])                  # ascending original index (the depth ties' order)
    slots = slots[order]
    o = perm[slots]
    colour = O.eval_sh(tex_orig[o], osc, pos=P[slots], cams=O.camera_centre(cam)[None, :])[0]
    img, tr, ab = O.render(P[slots], Sc[slots], Q[slots], T[slots], colour, cam, tiles=tiles, want_abs=True)
    pairs = 0
    for s in slots:
        sp = O.splat_setup(P[s], Sc[s], Q[s], cam)
        if sp.visible:
            pairs += (sp.x1 - sp.x0) * (sp.y1 - sp.y0)
    return img, tr, ab, int(keep.sum()), pairs


def test_geometry_codes_and_coded_render(ctx, O):
    from paper_2607_14513_gb300 import gsc
    n, cs = 2003, 128
    sc = S.make_scene(n, 21, clusters=6)
    geo = S.make_geometry(n, 22, scale=0.008)
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh, group_size=cs)
    blk, po, tab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_BC7)
    geom = gsc.gsc_geometry_encode(ctx, pos, torch.from_numpy(geo.scale).cuda(), torch.from_numpy(geo.rot).cuda(),
                                   torch.from_numpy(geo.logit).cuda(), po, cs)
    ctx.sync()
    pp = po.cpu().numpy()
    g = O.geometry_encode(sc.pos, geo.scale, geo.rot, geo.logit, pp, cs)
    got = _codes(gsc, geom, pp.shape[0], cs)
    for k in ("qpos", "qscale", "qrot", "qlogit", "chunk"):
        assert np.array_equal(got[k], g[k]), k
    # renders: a view of the whole scene, views that keep only part of it, one that keeps nothing
    tab_o = O.Table()
    tab_o.n_streams, tab_o.n, tab_o.n_groups = 1, tab.n, tab.n_groups
    tab_o.s[0].bands, tab_o.s[0].bc7_blocks, tab_o.s[0].n_groups = 16, 16, tab.n_groups
    tex = O.decode(tab_o, blk.cpu().numpy(), pp)
    osc = O.scales(sc.sh)
    r = gsc.Renderer(ctx)
    cams = [S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, 0.5], 96, 72),
            S.look_at([0.5, 0.5, -0.2], [0.9, 0.9, 0.5], 96, 72, fov_x_deg=40),
            S.look_at([0.5, 0.5, 0.5], [1.5, 0.5, 0.5], 96, 72, fov_x_deg=50),
            S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, -3.0], 64, 48)]
    partial = 0
    for cam in cams:
        tr = torch.empty((cam["height"], cam["width"]), dtype=torch.float32, device="cuda")
        img, tr, pairs, kept = r.render_coded(tab, blk, po, geom, cs, cam, trans=tr)
        ctx.sync()
        want, wtr, ab, wkept, wpairs = _oracle_coded_render(O, sc.pos, tex, osc, pp, g, cam)
        assert kept == wkept and pairs == wpairs
        partial += 0 < kept < g["chunk"].shape[0]
        a, t = img.cpu().numpy().astype(np.float64), tr.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(a - want) <= IMG_TOL * ab + IMG_FLOOR)
        assert np.all(np.abs(t - wtr) <= TR_TOL)
    assert partial >= 1


def test_geometry_arguments_are_checked(ctx):
    from paper_2607_14513_gb300 import gsc
    z = torch.zeros(64, device="cuda")
    perm = torch.zeros(16, dtype=torch.int32, device="cuda")
    for ns, cs in ((15, 16), (16, 8), (16, 24)):
        code = ctx.lib.gsc_geometry_encode(ctx.h, gsc._ptr(z), gsc._ptr(z), gsc._ptr(z), gsc._ptr(z), gsc._ptr(perm),
                                           ns, cs, gsc._ptr(torch.empty(4096, dtype=torch.uint8, device="cuda")), None)
        assert code == 1, (ns, cs)
    assert ctx.lib.gsc_geometry_bytes(16, 8) == 0


def test_coded_render_full_size_sampled_tiles(ctx, O):
    from paper_2607_14513_gb300 import gsc
    cfg = S.RENDER
    cs = 4096
    sc = S.make_scene(n=cfg["n"], seed=cfg["seed"], clusters=cfg["clusters"], heavy_frac=cfg["heavy_frac"])
    geo = S.make_geometry(cfg["n"], cfg["geom_seed"], scale=cfg["scale"])
    cam = S.make_views(cfg["views"], cfg["view_seed"], cfg["width"], cfg["height"])[0]
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh, group_size=cs)
    blk, po, tab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_BC7)
    geom = gsc.gsc_geometry_encode(ctx, pos, torch.from_numpy(geo.scale).cuda(), torch.from_numpy(geo.rot).cuda(),
                                   torch.from_numpy(geo.logit).cuda(), po, cs)
    r = gsc.Renderer(ctx)
    tr = torch.empty((cfg["height"], cfg["width"]), dtype=torch.float32, device="cuda")
    img, tr, pairs, kept = r.render_coded(tab, blk, po, geom, cs, cam, trans=tr)
    ctx.sync()
    pp = po.cpu().numpy()
    g = _codes(gsc, geom, pp.shape[0], cs)
    tab_o = O.Table()
    tab_o.n_streams, tab_o.n, tab_o.n_groups = 1, tab.n, tab.n_groups
    tab_o.s[0].bands, tab_o.s[0].bc7_blocks, tab_o.s[0].n_groups = 16, 16, tab.n_groups
    tex = O.decode(tab_o, blk.cpu().numpy(), pp)
    tx, ty = (cfg["width"] + 15) // 16, (cfg["height"] + 15) // 16
    rng = np.random.default_rng(41)
    tiles = np.unique(np.concatenate([[0, tx * ty - 1, (ty // 2) * tx + tx // 2],
                                      rng.integers(0, tx * ty, size=5)])).astype(np.int32)
    P, Sc, Q, T = O.geometry_decode(g)
    keep = np.array([O.chunk_visible(g["chunk"][c], cam) for c in range(g["chunk"].shape[0])])
    assert kept == keep.sum()
    valid = (pp >= 0) & keep[np.arange(pp.shape[0]) // cs]
    slots = np.nonzero(valid)[0]
    slots = slots[np.argsort(pp[slots])]
    colour = O.eval_sh(tex[pp[slots]], O.scales(sc.sh), pos=P[slots], cams=O.camera_centre(cam)[None, :])[0]
    want, wtr, ab = O.render(P[slots], Sc[slots], Q[slots], T[slots], colour, cam, tiles=tiles, want_abs=True)
    got, gtr = img.cpu().numpy().astype(np.float64), tr.cpu().numpy().astype(np.float64)
    for t in tiles:
        y, x = divmod(int(t), tx)
        sl = (slice(16 * y, 16 * y + 16), slice(16 * x, 16 * x + 16))
        assert np.all(np.abs(got[sl] - want[sl]) <= IMG_TOL * ab[sl] + IMG_FLOOR), t
        assert np.all(np.abs(gtr[sl] - wtr[sl]) <= TR_TOL), t
