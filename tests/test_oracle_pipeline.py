"""Whole-pipeline pins of the oracle: layout D (Sec. IV-B, Fig. SetupD), random access by
block index x block size (Sec. I; Sec. III-A), separate fixed-rate streams (Sec. IV-A/B),
inverse permutation on decode, and the effect the paper reports for colour sorting
(Sec. V-B: sorting lowers the distortion of the diffuse blocks)."""
import numpy as np
import pytest

from paper_2607_14513_gb300 import synthetic as S


@pytest.mark.parametrize("fmt", [1, 7])
def test_forced_format_blocks_are_layout_d(O, fmt):
    n = 300                                     # ragged: 19 groups, 4 padding slots
    sc = S.make_scene(n, 41)
    r = O.full_encode(sc.pos, sc.sh, fmt, group_size=64)
    st = O.stage(r["q"], r["perm_plan"])
    bpb = 16 if fmt == 7 else 8
    blocks = r["blocks"].reshape(-1, 16, bpb)
    assert blocks.shape[0] == 19
    # random access: each block is the encoding of its own staged texels
    for g in [0, 7, 18]:
        for k in [0, 5, 15]:
            b, _ = O.encode_blocks(st[g, k][None], fmt, threads=1)
            assert np.array_equal(b[0], blocks[g, k])
    # decode with the inverse permutation == per-block decode placed through perm
    tex = O.decode(r["table"], r["blocks"], r["perm"])
    dec = O.decode_blocks(r["blocks"], fmt).reshape(19, 16, 16, 4)
    perm = r["perm"]
    for s in range(19 * 16):
        if perm[s] >= 0:
            assert np.array_equal(tex[perm[s]], dec[s // 16, :, s % 16, :3])


def test_rate_streams_random_access_and_dropped_bands(O):
    n = 800
    sc = S.make_scene(n, 42, heavy_frac=0.1)
    r = O.full_encode(sc.pos, sc.sh, 0, target_x4=12, group_size=256)
    t = r["table"]
    blocks, perm = r["blocks"], r["perm"]
    tex = O.decode(t, blocks, perm)
    assert sorted(perm[perm >= 0].tolist()) == list(range(n))
    # the final order moves whole groups: each final group is one planned group
    planned = r["perm_plan"].reshape(-1, 16)
    final = perm.reshape(-1, 16)
    rows = {tuple(x) for x in planned.tolist()}
    assert all(tuple(x) in rows for x in final.tolist())
    seen_bands = set()
    for i in range(t.n_streams):
        s = t.s[i]
        gbytes = 16 * s.bc7_blocks + 8 * (s.bands - s.bc7_blocks)
        for gi in range(0, s.n_groups, max(1, s.n_groups // 3)):
            g = s.first_group + gi
            src = blocks[s.byte_offset + gi * gbytes: s.byte_offset + (gi + 1) * gbytes]
            off = 0
            for k in range(16):
                if k < s.bands:
                    is7 = k < s.bc7_blocks
                    blk = src[off: off + (16 if is7 else 8)]
                    off += 16 if is7 else 8
                    dec = (O.bc7_decode(blk) if is7 else O.bc1_decode(blk))[:, :3]
                else:
                    dec = np.full((16, 3), 128, np.uint8)
                for u in range(16):
                    o = perm[16 * g + u]
                    if o >= 0:
                        assert np.array_equal(tex[o, k], dec[u])
            seen_bands.add(s.bands)
    assert len(seen_bands) > 1


def test_sorting_lowers_diffuse_distortion(O):
    # Sec. V-B / Table I: colour-sorted scenes code their first (diffuse) coefficient block far
    # better than the original order at the same rate
    n = 4096
    sc = S.make_scene(n, 43)
    sse = {}
    for srt in (0, 1):
        r = O.full_encode(sc.pos, sc.sh, 1, sort=srt)
        tex = O.decode(r["table"], r["blocks"], r["perm"])
        sse[srt] = int(((tex[:, 0, :].astype(np.int64) - r["q"][:, 0, :].astype(np.int64)) ** 2).sum())
    assert sse[1] < 0.5 * sse[0]


def test_empty_scene(O):
    r = O.full_encode(np.zeros((0, 3), np.float32), np.zeros((0, 16, 3), np.float32), 1)
    assert r["table"].n_groups == 0 and r["blocks"].size == 0
