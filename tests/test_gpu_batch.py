"""Batched coding of many scenes (gsc_batch_*) against the single-scene calls and the oracle.

Per scene the batched plan, blocks, slot order and stream table must equal those of
gsc_plan_reorder + gsc_encode bit for bit (which the pipeline tests pin to the oracle), for
every schedule of the persistent launch; one small scene is also checked against the oracle
directly. The captured evaluation graph must equal the per-scene decode + SH evaluation.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (n, format, target_x4): uneven sizes, all three formats, a ragged and an empty scene
MIX = [(20000, 1, 0), (3001, 7, 0), (12345, 0, 24), (17, 0, 12), (0, 1, 0), (40000, 7, 0), (9000, 0, 32),
       (1, 7, 0), (65536, 1, 0), (5000, 0, 16)]


def _scenes(mix, seed0):
    out = []
    for i, (n, fmt, t4) in enumerate(mix):
        sc = S.make_scene(n, seed0 + i, clusters=5, heavy_frac=0.1)
        out.append((_dev(sc.pos).reshape(n, 3), _dev(sc.sh).reshape(n, 16, 3), fmt, t4, sc))
    return out


def _table_bytes(t):
    return ctypes.string_at(ctypes.addressof(t), ctypes.sizeof(t))


def _single(ctx, pos, sh, fmt, t4, gs):
    from paper_2607_14513_gb300 import gsc
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh, group_size=gs, sort=1)
    blocks, perm_out, tab = gsc.gsc_encode(ctx, sh, perm, scales, fmt, target_x4=t4)
    ctx.sync()
    return perm, scales, blocks, perm_out, tab


@pytest.mark.parametrize("schedule,ctas,tile", [(0, 4, 8), (1, 3, 32), (2, 2, 64), (3, 4, 16)])
def test_batch_equals_single_scene_calls(ctx, schedule, ctas, tile):
    from paper_2607_14513_gb300 import gsc
    sc = _scenes(MIX, 3100)
    gs = 1024
    b = gsc.Batch(ctx, [(p, s, f, t) for p, s, f, t, _ in sc], group_size=gs)
    b.encode(gsc.BatchTuning(schedule, ctas, tile))
    ctx.sync()
    for i, (pos, sh, fmt, t4, _) in enumerate(sc):
        perm, scales, blocks, perm_out, tab = b.result(i)
        r = _single(ctx, pos, sh, fmt, t4, gs)
        assert torch.equal(perm[:r[0].numel()], r[0]), i
        assert torch.equal(scales, r[1]), i
        assert torch.equal(blocks, r[2]), i
        assert torch.equal(perm_out, r[3]), i
        assert _table_bytes(tab) == _table_bytes(r[4]), i


def test_batch_scene_against_oracle(ctx, O):
    from paper_2607_14513_gb300 import gsc
    mix = [(3000, 0, 24), (777, 7, 0), (2048, 1, 0)]
    sc = _scenes(mix, 3300)
    b = gsc.Batch(ctx, [(p, s, f, t) for p, s, f, t, _ in sc], group_size=256)
    b.encode(gsc.BatchTuning(1, 4, 8))
    ctx.sync()
    for i, (_, _, fmt, t4, s) in enumerate(sc):
        perm, scales, blocks, perm_out, tab = b.result(i)
        ref = O.full_encode(s.pos, s.sh, fmt, group_size=256, target_x4=t4)
        assert np.array_equal(blocks.cpu().numpy().ravel(), np.asarray(ref["blocks"]).ravel()), i
        assert np.array_equal(perm_out.cpu().numpy(), ref["perm"]), i


def test_batch_autotune_picks_a_valid_tuning(ctx):
    from paper_2607_14513_gb300 import gsc
    sc = _scenes(MIX[:6], 3200)
    b = gsc.Batch(ctx, [(p, s, f, t) for p, s, f, t, _ in sc], group_size=1024)
    t, ms = b.autotune()
    assert t.schedule in (0, 1, 2, 3) and 1 <= t.ctas_per_sm <= 32 and t.bc1_tile_groups in (8, 32)
    assert ms > 0.0
    b.encode(t)
    ctx.sync()
    pos, sh, fmt, t4, _ = sc[2]
    r = _single(ctx, pos, sh, fmt, t4, 1024)
    assert torch.equal(b.result(2)[2], r[2])


def test_batch_eval_graph_equals_per_scene_eval(ctx):
    from paper_2607_14513_gb300 import gsc
    sc = _scenes(MIX, 3400)
    b = gsc.Batch(ctx, [(p, s, f, t) for p, s, f, t, _ in sc], group_size=4096)
    b.encode(gsc.BatchTuning(1, 4, 8))
    ctx.sync()
    g = torch.Generator().manual_seed(7)
    cams = (torch.rand((8, 3), generator=g, dtype=torch.float64) * 40 - 20).float().cuda()
    outs = [torch.full((max(n, 1), 8, 3), np.nan, device="cuda")[:n] for n, _, _ in MIX]
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = b.eval_graph(cams, outs, stream=st)
    for _ in range(2):
        graph.launch(stream=st)
    st.synchronize()
    for i, (pos, _, _, _, _) in enumerate(sc):
        _, _, blocks, perm_out, tab = b.result(i)
        ref = gsc.gsc_decode_eval_sh(ctx, tab, blocks, perm_out, pos=pos, cams=cams, out_order=gsc.OUT_GAUSS_MAJOR)
        ctx.sync()
        assert torch.equal(outs[i], ref), i
    graph.close()


def test_batch_invalid_arguments(ctx):
    from paper_2607_14513_gb300 import gsc
    sc = _scenes([(100, 1, 0)], 3500)
    b = gsc.Batch(ctx, [(p, s, f, t) for p, s, f, t, _ in sc])
    with pytest.raises(gsc.GscError):
        b.encode(gsc.BatchTuning(4, 4, 8))          # no such schedule
    with pytest.raises(gsc.GscError):
        b.encode(gsc.BatchTuning(0, 0, 8))          # zero CTAs per SM
    with pytest.raises(gsc.GscError):
        b.encode(gsc.BatchTuning(0, 33, 8))         # more than 32 CTAs per SM
    bad = (gsc.BatchScene * 1)()
    bad[0] = b.arr[0]
    bad[0].format = 2
    assert ctx.lib.gsc_batch_workspace_bytes(bad, 1) == 0
    assert ctx.lib.gsc_batch_workspace_bytes(b.arr, 0) == 0


def test_batch_of_many_rate_scenes(ctx):
    # every rate scene takes two entries of the device scene list (its BC1 and BC7 codings)
    from paper_2607_14513_gb300 import gsc
    mix = [(100 + 173 * i, 0, (12, 16, 24, 32)[i % 4]) for i in range(16)] + [(999, 1, 0), (1500, 7, 0)]
    sc = _scenes(mix, 3600)
    b = gsc.Batch(ctx, [(p, s, f, t) for p, s, f, t, _ in sc], group_size=256)
    b.encode(gsc.BatchTuning(1, 4, 8))
    ctx.sync()
    for i, (pos, sh, fmt, t4, _) in enumerate(sc):
        r = _single(ctx, pos, sh, fmt, t4, 256)
        assert torch.equal(b.result(i)[2], r[2]), i
        assert torch.equal(b.result(i)[3], r[3]), i
