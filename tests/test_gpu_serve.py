"""The request loop on the GPU (gsc_server_*): every result of a concurrent mix of encode and
evaluation requests (several slots, merged evaluations, host and device outputs, three output
orders, directions and camera centres) equals the single calls' result bit for bit; a scene
re-encoded while evaluations are queued serves each evaluation the version it was submitted
against; the HBM budget holds and evicted scenes are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2607_14513_gb300 import synthetic as S

GiB = 1 << 30


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def _single_encode(ctx, pos, sh, fmt, t4, gs=4096):
    from paper_2607_14513_gb300 import gsc
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh, group_size=gs, sort=1)
    blocks, perm_out, tab = gsc.gsc_encode(ctx, sh, perm, scales, fmt, target_x4=t4)
    ctx.sync()
    return blocks, perm_out, tab


def _single_eval(ctx, enc, pos, views, cams, order):
    from paper_2607_14513_gb300 import gsc
    blocks, perm_out, tab = enc
    kw = dict(cams=views) if cams else dict(dirs=views)
    out = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, pos=pos, out_order=order, **kw)
    ctx.sync()
    return out


def _out_shape(n, V, order):
    from paper_2607_14513_gb300 import gsc
    ns = (n + 15) // 16 * 16
    return {gsc.OUT_VIEW_MAJOR: (V, n, 3), gsc.OUT_SLOT_ORDER: (V, ns, 3), gsc.OUT_GAUSS_MAJOR: (n, V, 3)}[order]


SCENES = [(30000, 1, 0), (7001, 7, 0), (20000, 0, 24), (123, 7, 0), (50000, 1, 0)]


def test_mix_equals_single_calls(ctx):
    from paper_2607_14513_gb300 import gsc
    rng = np.random.default_rng(11)
    data = []
    for i, (n, fmt, t4) in enumerate(SCENES):
        sc = S.make_scene(n, 4000 + i, clusters=6, heavy_frac=0.1)
        host = (torch.from_numpy(sc.pos), torch.from_numpy(sc.sh))
        dev = (host[0].cuda(), host[1].cuda())
        data.append((n, fmt, t4, host, dev))
    srv = gsc.Server(ctx, 8 * GiB, n_slots=4, merge=True)
    try:
        enc_t = []
        for i, (n, fmt, t4, host, dev) in enumerate(data):
            src = host if i % 2 == 0 else dev           # host and device inputs
            enc_t.append(srv.encode(i, src[0], src[1], fmt, target_x4=t4))
        evs = []
        for k in range(40):
            i = int(rng.integers(len(data)))
            n = data[i][0]
            V = int(rng.integers(1, 33))
            cams = bool(rng.integers(2))
            order = int(rng.integers(3))
            views = torch.from_numpy(S.make_cams(V, 50 + k) if cams else S.make_dirs(V, 50 + k))
            views = views.cuda() if k % 3 else views
            on_dev = k % 2 == 0
            out = torch.full(_out_shape(n, V, order), np.nan, dtype=torch.float32,
                             device="cuda" if on_dev else "cpu")
            t = srv.eval(i, n, out, **({"cams": views} if cams else {"dirs": views}), out_order=order)
            evs.append((t, i, views, cams, order, out))
        for t in enc_t:
            assert srv.wait(t).status == 0
        results = [(srv.wait(t), i, views, cams, order, out) for t, i, views, cams, order, out in evs]
        st = srv.stats()
        assert st.failed == 0 and st.done == len(enc_t) + len(evs)
        singles = [_single_encode(ctx, d[4][0], d[4][1], d[1], d[2]) for d in data]
        for i, enc in enumerate(singles):
            tab, blocks, perm = srv.read_scene(i)
            assert torch.equal(blocks, enc[0].cpu()), i
            assert torch.equal(perm, enc[1].cpu()), i
            assert tab.total_bytes == enc[2].total_bytes and tab.used_bits == enc[2].used_bits
        merged = 0
        for res, i, views, cams, order, out in results:
            assert res.status == 0
            merged += res.merged > 1
            ref = _single_eval(ctx, singles[i], data[i][4][0], views.cuda(), cams, order)
            assert torch.equal(out.cpu(), ref.cpu()), (i, order, cams)
        assert res.t_done_ms >= res.t_admit_ms >= res.t_submit_ms
    finally:
        srv.close()


def test_reencode_serves_each_evaluation_its_version(ctx):
    from paper_2607_14513_gb300 import gsc
    n = 40000
    a = S.make_scene(n, 4100, clusters=4)
    b = S.make_scene(n, 4101, clusters=4)
    pa, sa = torch.from_numpy(a.pos).cuda(), torch.from_numpy(a.sh).cuda()
    pb, sb = torch.from_numpy(b.pos).cuda(), torch.from_numpy(b.sh).cuda()
    cams = torch.from_numpy(S.make_cams(8, 77)).cuda()
    srv = gsc.Server(ctx, 8 * GiB, n_slots=3, merge=True)
    try:
        outs = [torch.empty((n, 8, 3), device="cuda") for _ in range(4)]
        t = [srv.encode(0, pa, sa, gsc.FMT_BC7),
             srv.eval(0, n, outs[0], cams=cams), srv.eval(0, n, outs[1], cams=cams),
             srv.encode(0, pb, sb, gsc.FMT_BC7),
             srv.eval(0, n, outs[2], cams=cams), srv.eval(0, n, outs[3], cams=cams)]
        rs = [srv.wait(x) for x in t]
        assert all(r.status == 0 for r in rs)
        ea = _single_encode(ctx, pa, sa, gsc.FMT_BC7, 0)
        eb = _single_encode(ctx, pb, sb, gsc.FMT_BC7, 0)
        ra = _single_eval(ctx, ea, pa, cams, True, gsc.OUT_GAUSS_MAJOR)
        rb = _single_eval(ctx, eb, pb, cams, True, gsc.OUT_GAUSS_MAJOR)
        assert torch.equal(outs[0], ra) and torch.equal(outs[1], ra)
        assert torch.equal(outs[2], rb) and torch.equal(outs[3], rb)
        srv.drain()
        assert srv.stats().resident_versions == 1        # the replaced version was freed
    finally:
        srv.close()


def test_budget_eviction_and_refusals(ctx):
    from paper_2607_14513_gb300 import gsc
    n = 60000
    scs = [S.make_scene(n, 4200 + i, clusters=4) for i in range(3)]
    dev = [(torch.from_numpy(s.pos).cuda(), torch.from_numpy(s.sh).cuda()) for s in scs]
    # find the footprint of one BC1 encode of this size with the host-side policy
    req = gsc.SimRequest(0, 0, n, 1, 0, 0, 0, 0, 1, 0, 0.0, 1.0)
    res, peak = gsc.simulate(gsc.ServerParams(64 * GiB, 1, 1, 64, 1, 0, 0), [req])
    e = res[0].used_bytes_at_admit
    keep = (n + 15) // 16 * 128 + 4 * ((n + 15) // 16 * 16) + 12 * n
    budget = e + keep + keep // 2
    srv = gsc.Server(ctx, budget, n_slots=1, merge=False)
    try:
        for i in range(3):
            assert srv.wait(srv.encode(i, dev[i][0], dev[i][1], gsc.FMT_BC1)).status == 0
        st = srv.stats()
        assert st.peak_bytes <= budget and st.evictions == 1
        cams = torch.from_numpy(S.make_cams(2, 5)).cuda()
        out = torch.empty((n, 2, 3), device="cuda")
        assert srv.wait(srv.eval(0, n, out, cams=cams)).status == 1   # scene 0 was evicted
        assert srv.wait(srv.eval(2, n, out, cams=cams)).status == 0
        assert srv.wait(srv.eval(2, n + 1, out, cams=cams)).status == 1  # wrong size
        srv.evict(2)
        assert srv.stats().resident_versions == 1
        with pytest.raises(gsc.GscError):
            srv.eval(1, n, out, cams=cams, dirs=cams)                  # both view kinds
        with pytest.raises(gsc.GscError):
            srv.encode(1, dev[1][0], dev[1][1], 3)                      # no such format
        big = torch.zeros((2_000_000, 16, 3), device="cuda")
        with pytest.raises(gsc.GscError):
            srv.encode(5, torch.zeros((2_000_000, 3), device="cuda"), big, gsc.FMT_BC7)  # never fits
    finally:
        srv.close()


def test_checkpoint_round_trip_and_server_reload(ctx, tmp_path):
    # a coded scene written from device buffers reads back byte for byte; a server scene saved,
    # evicted and reloaded from its file evaluates exactly as before
    from paper_2607_14513_gb300 import gsc
    n = 30000
    sc = S.make_scene(n, 4300, clusters=5, heavy_frac=0.1)
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    blocks, perm_out, tab = _single_encode(ctx, pos, sh, gsc.FMT_RATE, 24)
    f = str(tmp_path / "s.gsc")
    gsc.scene_write(f, tab, blocks, perm_out, pos)
    t2, b2, p2, q2 = gsc.scene_read(f, device="cuda")
    assert torch.equal(b2, blocks) and torch.equal(p2, perm_out) and torch.equal(q2, pos)
    cams = torch.from_numpy(S.make_cams(8, 88)).cuda()
    ref = _single_eval(ctx, (blocks, perm_out, tab), pos, cams, True, gsc.OUT_GAUSS_MAJOR)
    got = _single_eval(ctx, (b2, p2, t2), q2, cams, True, gsc.OUT_GAUSS_MAJOR)
    assert torch.equal(ref, got)
    srv = gsc.Server(ctx, 8 * GiB, n_slots=2)
    try:
        assert srv.wait(srv.encode(3, pos, sh, gsc.FMT_RATE, target_x4=24)).status == 0
        out0 = torch.empty((n, 8, 3), device="cuda")
        assert srv.wait(srv.eval(3, n, out0, cams=cams)).status == 0
        g = str(tmp_path / "srv.gsc")
        srv.save(3, g)
        srv.evict(3)
        assert srv.wait(srv.eval(3, n, out0, cams=cams)).status == 1      # no longer resident
        assert srv.wait(srv.load(3, g, n)).status == 0
        out1 = torch.empty((n, 8, 3), device="cuda")
        assert srv.wait(srv.eval(3, n, out1, cams=cams)).status == 0
        assert torch.equal(out1, ref)
        with pytest.raises(gsc.GscError):
            srv.load(4, g, n + 1)                                          # the file holds another size
    finally:
        srv.close()


def test_wait_timeout_and_cancel(ctx):
    # failure handling on the host: a bounded wait returns GSC_ERR_TIMEOUT and the request still
    # completes; a queued request can be cancelled, an admitted or finished one cannot
    from paper_2607_14513_gb300 import gsc
    a = S.make_scene(600_000, 4400, clusters=8)
    b = S.make_scene(5_000, 4401, clusters=2)
    pa, sa = torch.from_numpy(a.pos).cuda(), torch.from_numpy(a.sh).cuda()
    pb, sb = torch.from_numpy(b.pos).cuda(), torch.from_numpy(b.sh).cuda()
    srv = gsc.Server(ctx, 8 * GiB, n_slots=1)
    try:
        t1 = srv.encode(0, pa, sa, gsc.FMT_BC7)          # ~30 ms of BC7 search on the only slot
        t2 = srv.encode(1, pb, sb, gsc.FMT_BC1)          # queued behind it
        with pytest.raises(gsc.GscError) as e:
            srv.wait(t1, timeout_ms=0)
        assert e.value.code == 5
        srv.cancel(t2)
        assert srv.wait(t2).status == 8
        assert srv.wait(t1).status == 0
        with pytest.raises(gsc.GscError):
            srv.cancel(t1)                                # already completed and collected
        st = srv.stats()
        assert st.failed == 1 and st.done == 2
        out = torch.empty((5000, 1, 3), device="cuda")
        assert srv.wait(srv.eval(1, 5000, out, cams=torch.zeros((1, 3), device="cuda"))).status == 1
    finally:
        srv.close()
