"""Fused decode + SH evaluation (Sec. II, c(f) = H w(f - p); Sec. III-B decoding) through the
C-ABI: gsc_decode_eval_sh (centres in original order, gathered through the slot order) and
gsc_decode_eval_sh_slots (centres in slot order, built by gsc_positions_to_slots) on the all-BC7,
all-BC1 and 6-bpt rate-stream codings.

Expected values come from the oracle alone: it codes the scene itself (the GPU blocks are checked
against its blocks bit for bit first), decodes its own blocks and evaluates them in FP64; the GPU
colours must lie within 1e-5 of the sum of absolute terms. Both software entry points must also
equal each other and the texture-unit evaluation bit for bit (the same arithmetic per Gaussian
and view). Sizes straddle group and launch boundaries (1, 17, 383, 385, ...); blocks that are only
8-byte aligned (the all-BC7 fast path then takes 8-byte loads) and slot entries and centres that
are only 4-byte aligned must give the same bits; shared view directions and view counts that are
not a multiple of four are covered too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

SH_TOL = 1e-5
SIZES = [1, 17, 383, 385, 1537, 6001]
CODINGS = (("bc7", 7, 0), ("bc1", 1, 0), ("rate", 0, 24))


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def _oracle(O, pos, sh):
    osc = O.scales(sh)
    q = O.quantise(sh, osc)
    operm = O.plan(pos, q, 4096, 1)
    refs = {name: O.encode(q, operm, osc, fmt, t4) for name, fmt, t4 in CODINGS}
    return osc, operm, refs


def _view_major(got, order, perm, n):
    """GPU output in any order -> [V][n][3] float64 (slot order: padding slots must be 0)."""
    g = got.cpu().numpy().astype(np.float64)
    if order == 2:
        return g.transpose(1, 0, 2)
    if order == 3:                     # slot-order rows [ns][V][3] -> view-major slot order
        g = g.transpose(1, 0, 2)
    if order in (1, 3):
        pp = perm.cpu().numpy()
        valid = pp >= 0
        assert np.all(g[:, ~valid] == 0.0)
        full = np.zeros((g.shape[0], n, 3))
        full[:, pp[valid]] = g[:, valid]
        return full
    return g


def _scene(n, seed):
    sc = S.make_scene(n, seed, clusters=4, heavy_frac=0.1)
    return sc.pos.copy(), sc.sh.copy()


@pytest.mark.parametrize("n", SIZES)
def test_eval_matches_oracle_and_texture_unit(ctx, O, n):
    from paper_2607_14513_gb300 import gsc
    pos, sh = _scene(n, 3000 + n)
    dpos, dsh = torch.from_numpy(pos).cuda(), torch.from_numpy(sh).cuda()
    osc, operm, refs = _oracle(O, pos, sh)
    perm, scales = gsc.gsc_plan_reorder(ctx, dpos, dsh)
    ctx.sync()
    assert np.array_equal(perm.cpu().numpy(), operm)
    cams = S.make_cams(8, 1300 + n)
    dc = torch.from_numpy(cams).cuda()
    for name, fmt, t4 in CODINGS:
        blk, po, tab = gsc.gsc_encode(ctx, dsh, perm, scales, fmt, t4)
        ctx.sync()
        ref = refs[name]
        assert np.array_equal(blk.cpu().numpy(), ref["blocks"]), name
        assert np.array_equal(po.cpu().numpy(), ref["perm"]), name
        tex = O.decode(ref["table"], ref["blocks"], ref["perm"])
        want, ab = O.eval_sh(tex, osc, pos=pos, cams=cams, want_abs=True)
        pslot = gsc.gsc_positions_to_slots(ctx, dpos, po)
        scene = gsc.TexScene(ctx, tab, blk, perm=po, pos=dpos)
        try:
            for order in (gsc.OUT_VIEW_MAJOR, gsc.OUT_GAUSS_MAJOR, gsc.OUT_SLOT_ORDER, gsc.OUT_SLOT_ROWS):
                a = gsc.gsc_decode_eval_sh(ctx, tab, blk, po, pos=dpos, cams=dc, out_order=order)
                b = gsc.gsc_decode_eval_sh_slots(ctx, tab, blk, po, pos_slot=pslot, cams=dc, out_order=order)
                c = gsc.gsc_decode_eval_sh_tex(ctx, scene, po, cams=dc, out_order=order)
                ctx.sync()
                assert torch.equal(a, b), (name, order)
                assert torch.equal(a, c), (name, order)
                got = _view_major(a, order, po, n)
                assert np.all(np.abs(got - want) <= SH_TOL * ab + 1e-30), (name, order)
        finally:
            scene.close()


def test_positions_to_slots(ctx):
    from paper_2607_14513_gb300 import gsc
    n = 1000
    pos, sh = _scene(n, 77)
    dpos = torch.from_numpy(pos).cuda()
    perm, _ = gsc.gsc_plan_reorder(ctx, dpos, torch.from_numpy(sh).cuda())
    ps = gsc.gsc_positions_to_slots(ctx, dpos, perm)
    ctx.sync()
    pp = perm.cpu().numpy()
    want = np.zeros((pp.shape[0], 3), np.float32)
    want[pp >= 0] = pos[pp[pp >= 0]]
    assert np.array_equal(ps.cpu().numpy(), want)


def _offset(t, elems):
    """A copy of t whose data pointer is `elems` elements past a fresh allocation."""
    buf = torch.empty(t.numel() + elems, dtype=t.dtype, device=t.device)
    v = buf[elems:elems + t.numel()].view(t.shape)
    v.copy_(t)
    return v


def test_unaligned_inputs_give_the_same_bits(ctx, O):
    from paper_2607_14513_gb300 import gsc
    n = 2003
    pos, sh = _scene(n, 91)
    dpos, dsh = torch.from_numpy(pos).cuda(), torch.from_numpy(sh).cuda()
    perm, scales = gsc.gsc_plan_reorder(ctx, dpos, dsh)
    dc = torch.from_numpy(S.make_cams(5, 92)).cuda()
    for name, fmt, t4 in CODINGS:
        blk, po, tab = gsc.gsc_encode(ctx, dsh, perm, scales, fmt, t4)
        pslot = gsc.gsc_positions_to_slots(ctx, dpos, po)
        a = gsc.gsc_decode_eval_sh_slots(ctx, tab, blk, po, pos_slot=pslot, cams=dc, out_order=gsc.OUT_GAUSS_MAJOR)
        # blocks 8 bytes past a 16-byte boundary, slot entries and centres 4 bytes past one
        b = gsc.gsc_decode_eval_sh_slots(ctx, tab, _offset(blk, 8), _offset(po, 1), pos_slot=_offset(pslot, 1),
                                         cams=dc, out_order=gsc.OUT_GAUSS_MAJOR)
        c = gsc.gsc_decode_eval_sh(ctx, tab, _offset(blk, 8), _offset(po, 1), pos=_offset(dpos, 1), cams=dc,
                                   out_order=gsc.OUT_GAUSS_MAJOR)
        ctx.sync()
        assert torch.equal(a, b), name
        assert torch.equal(a, c), name


@pytest.mark.parametrize("V", [1, 7, 64])
def test_shared_directions_and_view_counts(ctx, O, V):
    from paper_2607_14513_gb300 import gsc
    n = 1537
    pos, sh = _scene(n, 400 + V)
    dpos, dsh = torch.from_numpy(pos).cuda(), torch.from_numpy(sh).cuda()
    osc, operm, refs = _oracle(O, pos, sh)
    perm, scales = gsc.gsc_plan_reorder(ctx, dpos, dsh)
    dirs = S.make_dirs(V, 500 + V)
    cams = S.make_cams(V, 600 + V)
    dd, dc = torch.from_numpy(dirs).cuda(), torch.from_numpy(cams).cuda()
    for name, fmt, t4 in CODINGS:
        blk, po, tab = gsc.gsc_encode(ctx, dsh, perm, scales, fmt, t4)
        ctx.sync()
        ref = refs[name]
        assert np.array_equal(blk.cpu().numpy(), ref["blocks"]), name
        tex = O.decode(ref["table"], ref["blocks"], ref["perm"])
        for kind in ("dirs", "cams"):
            kw = dict(dirs=dd) if kind == "dirs" else dict(cams=dc, pos=dpos)
            okw = dict(dirs=dirs) if kind == "dirs" else dict(cams=cams, pos=pos)
            want, ab = O.eval_sh(tex, osc, want_abs=True, **okw)
            for order in (gsc.OUT_GAUSS_MAJOR, gsc.OUT_SLOT_ORDER, gsc.OUT_SLOT_ROWS):
                a = gsc.gsc_decode_eval_sh(ctx, tab, blk, po, out_order=order, **kw)
                ctx.sync()
                got = _view_major(a, order, po, n)
                assert np.all(np.abs(got - want) <= SH_TOL * ab + 1e-30), (name, kind, order)
