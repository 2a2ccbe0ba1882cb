"""One scene split over shards on one GPU (the shards of one process; the collectives are then
plain reductions over the shards' partials): scales, slot order, lambda, stream table, every
rate-stream byte and the final slot order equal the whole-scene calls, which the oracle pins
elsewhere (test_gpu_medium.py, test_gpu_pipeline.py).

Cases: the 262,144-Gaussian scene in 2 uneven input shards at 6 bits per texel; a ragged scene
(not a multiple of 16 or of the chunk size) in 3 shards at 3 and 8 bits per texel; more shards than
chunks, so that some shards own nothing."""
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


def _whole(ctx, pos, sh, t4, group_size):
    from paper_2607_14513_gb300 import gsc
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh, group_size=group_size)
    blocks, perm_out, tab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_RATE, t4)
    ctx.sync()
    return scales, tab, blocks, perm_out


def _split(ctx, pos, sh, cuts, t4, group_size):
    from paper_2607_14513_gb300 import shard
    edges = [0] + list(cuts) + [pos.shape[0]]
    pp = [pos[a:b].contiguous() for a, b in zip(edges[:-1], edges[1:])]
    ss = [sh[a:b].contiguous() for a, b in zip(edges[:-1], edges[1:])]
    out = shard.encode_scene_sharded(ctx, pp, ss, t4, group_size=group_size)
    ctx.sync()
    return out


def _same(whole, split):
    s1, t1, b1, p1 = whole
    s2, t2, b2, p2 = split
    assert torch.equal(s1, s2)
    assert (t1.lambda_, t1.used_bits, t1.budget_bits, t1.total_bytes, t1.n, t1.n_groups) == \
        (t2.lambda_, t2.used_bits, t2.budget_bits, t2.total_bytes, t2.n, t2.n_groups)
    assert [(t1.s[i].n_groups, t1.s[i].first_group, t1.s[i].byte_offset) for i in range(14)] == \
        [(t2.s[i].n_groups, t2.s[i].first_group, t2.s[i].byte_offset) for i in range(14)]
    assert list(t1.weights) == list(t2.weights) and list(t1.scales) == list(t2.scales)
    assert torch.equal(b1[:t1.total_bytes], b2[:t2.total_bytes])
    assert torch.equal(p1, p2)


def test_medium_scene_two_shards(ctx):
    sc = S.make_scene(**S.MEDIUM)
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    _same(_whole(ctx, pos, sh, 24, 4096), _split(ctx, pos, sh, [100000], 24, 4096))


@pytest.mark.parametrize("t4", [12, 32])
def test_ragged_scene_three_shards(ctx, t4):
    sc = S.make_scene(n=50001, seed=77, clusters=8, heavy_frac=0.1)
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    _same(_whole(ctx, pos, sh, t4, 256), _split(ctx, pos, sh, [7, 31000], t4, 256))


def test_more_shards_than_chunks(ctx):
    sc = S.make_scene(n=3001, seed=78, clusters=4, heavy_frac=0.0)
    pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
    # 3001 Gaussians in chunks of 1024: 3 chunks over 5 shards, two of which own nothing
    _same(_whole(ctx, pos, sh, 16, 1024), _split(ctx, pos, sh, [500, 1000, 2000, 2500], 16, 1024))
