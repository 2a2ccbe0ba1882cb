"""GPU block codecs against the oracle, and both decoders against the GB300 texture unit.

Bit-exact: encoded BC1 / BC7 blocks and their squared errors; decoded RGBA of arbitrary
block bytes; texture-object sampling of every BC1 code pair and of BC7 blocks of every
mode, partition, rotation and index selection (Sec. III-B; Sec. I on hardware decoders).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def _texels(rng, n):
    """Mixed content: random, smooth, two-colour, constant, from a scene."""
    from oracle import oracle as O
    from paper_2607_14513_gb300 import synthetic as S
    parts = [rng.integers(0, 256, size=(n // 4, 16, 3))]
    base = rng.integers(20, 236, size=(n // 4, 1, 3))
    parts.append(np.clip(base + rng.integers(-12, 13, size=(n // 4, 16, 3)), 0, 255))
    two = rng.integers(0, 256, size=(n // 8, 2, 3))
    sel = rng.integers(0, 2, size=(n // 8, 16))
    parts.append(np.take_along_axis(two, sel[:, :, None].repeat(3, axis=2), axis=1))
    parts.append(np.repeat(rng.integers(0, 256, size=(n // 16, 1, 3)), 16, axis=1))
    sc = S.make_scene(max(16, n // 8), 77)
    q = O.quantise(sc.sh, O.scales(sc.sh))
    st = O.stage(q, O.plan(sc.pos, q, 256, 1)).reshape(-1, 16, 3)
    parts.append(st[: n - sum(p.shape[0] for p in parts)])
    return np.concatenate(parts).astype(np.uint8)


@pytest.mark.parametrize("fmt", [1, 7])
def test_encode_blocks_bit_exact(ctx, O, fmt):
    from paper_2607_14513_gb300 import gsc
    rng = np.random.default_rng(100 + fmt)
    tex = _texels(rng, 4096 if fmt == 1 else 1536)
    ob, osse = O.encode_blocks(tex, fmt)
    gb, gsse = gsc.gsc_encode_blocks(ctx, torch.from_numpy(tex).cuda(), fmt)
    torch.cuda.synchronize()
    gb, gsse = gb.cpu().numpy(), gsse.cpu().numpy().astype(np.uint64)
    bad = np.nonzero((gb != ob).any(axis=1))[0]
    assert bad.size == 0, "first mismatching block %d: gpu %s oracle %s" % (bad[0], gb[bad[0]], ob[bad[0]])
    assert np.array_equal(gsse, osse)


@pytest.mark.parametrize("fmt", [1, 7])
def test_decode_arbitrary_blocks_bit_exact(ctx, O, fmt):
    from paper_2607_14513_gb300 import gsc
    rng = np.random.default_rng(200 + fmt)
    bpb = 16 if fmt == 7 else 8
    blk = rng.integers(0, 256, size=(3000, bpb)).astype(np.uint8)
    if fmt == 7:
        blk[:8, 0] = 0                                     # reserved mode
        for m in range(8):                                 # every mode, many times
            blk[8 + m::8, 0] = (blk[8 + m::8, 0] & np.uint8(0xFF ^ ((1 << (m + 1)) - 1))) | np.uint8(1 << m)
    ref = O.decode_blocks(blk, fmt)
    got = gsc.gsc_decode_blocks(ctx, torch.from_numpy(blk).cuda(), fmt).cpu().numpy()
    assert np.array_equal(got, ref)


def test_texture_unit_bc1_every_code_pair(ctx, O):
    # every 6-bit G pair and 5-bit B pair in four-colour mode, every R pair in both modes,
    # G / B pairs in three-colour mode; index pattern covers all four entries
    from paper_2607_14513_gb300 import gsc
    blocks = []
    for i in range(64):
        for j in range(64):
            blocks.append(((31 << 11) | (i << 5) | (i & 31), (j << 5) | (j & 31)))
            blocks.append(((i << 5) | (i & 31), (31 << 11) | (j << 5) | (j & 31)))
    for i in range(32):
        for j in range(32):
            blocks.append(((i << 11) | (63 << 5) | 31, j << 11))
    arr = np.zeros((len(blocks), 8), np.uint8)
    for b, (c0, c1) in enumerate(blocks):
        arr[b] = [c0 & 255, c0 >> 8, c1 & 255, c1 >> 8, 0xE4, 0x1B, 0x4E, 0xB1]
    hw = gsc.gsc_decode_blocks_tex(ctx, torch.from_numpy(arr).cuda(), 1).cpu().numpy()
    sw = gsc.gsc_decode_blocks(ctx, torch.from_numpy(arr).cuda(), 1).cpu().numpy()
    ref = O.decode_blocks(arr, 1)
    assert np.array_equal(hw, ref)
    assert np.array_equal(sw, ref)


def test_texture_unit_bc7_every_candidate(ctx, O):
    # blocks the oracle packs for all 285 candidates (every mode, partition, rotation, index
    # selection) on several texel sets, plus random bytes of every mode
    from paper_2607_14513_gb300 import gsc
    rng = np.random.default_rng(300)
    blks = []
    for trial in range(4):
        tex = rng.integers(0, 256, size=(16, 3)).astype(np.uint8)
        if trial == 1:
            tex = np.clip(128 + rng.integers(-20, 21, size=(16, 3)), 0, 255).astype(np.uint8)
        for e in range(O.bc7_n_candidates()):
            blks.append(O.bc7_candidate(tex, e)[1])
    rnd = rng.integers(0, 256, size=(2048, 16)).astype(np.uint8)
    for m in range(8):
        rnd[m::8, 0] = (rnd[m::8, 0] & np.uint8(0xFF ^ ((1 << (m + 1)) - 1))) | np.uint8(1 << m)
    blks = np.concatenate([np.array(blks), rnd])
    hw = gsc.gsc_decode_blocks_tex(ctx, torch.from_numpy(blks).cuda(), 7).cpu().numpy()
    ref = O.decode_blocks(blks, 7)
    bad = np.nonzero((hw != ref).any(axis=(1, 2)))[0]
    assert bad.size == 0, "first mismatch block %d mode byte %d" % (bad[0], blks[bad[0], 0])
    sw = gsc.gsc_decode_blocks(ctx, torch.from_numpy(blks).cuda(), 7).cpu().numpy()
    assert np.array_equal(sw, ref)


def test_bc7_mode1_thread_and_warp_mappings(ctx, O):
    # the mode-1 search mapped thread per block and warp per block: the same least error and
    # partition for every block, and both equal to the oracle's mode-1 candidates (Sec. III-B)
    from paper_2607_14513_gb300 import gsc
    rng = np.random.default_rng(107)
    tex = _texels(rng, 777)
    td = torch.from_numpy(tex).cuda()
    s0, p0, _ = gsc.bc7_mode1(ctx, td, False)
    s1, p1, _ = gsc.bc7_mode1(ctx, td, True)
    torch.cuda.synchronize()
    assert torch.equal(s0, s1) and torch.equal(p0, p1)
    s0, p0 = s0.cpu().numpy(), p0.cpu().numpy()
    for b in range(0, tex.shape[0], 7):
        errs = [O.bc7_candidate(tex[b], 16 + p)[0] for p in range(64)]
        assert int(s0[b]) == min(errs) and int(p0[b]) == int(np.argmin(errs)), b
