"""Pins of the oracle's reorder plan (Sec. III-C, Fig. Bit4Scan; Sec. V-A; Sec. IV-B Fig. SetupD).

The paper fixes the 24-bit RGB bit interleave of the DC colour, a sort by that key,
and the grouping of Gaussians in that order, done inside larger spatial groups.
"""
import numpy as np
import pytest

from paper_2607_14513_gb300 import synthetic as S


def test_colour_key_hand_values(O):
    # bit i of R -> 3i+2, of G -> 3i+1, of B -> 3i
    assert O.colour_key(255, 0, 0) == 0x924924
    assert O.colour_key(0, 255, 0) == 0x492492
    assert O.colour_key(0, 0, 255) == 0x249249
    assert O.colour_key(255, 255, 255) == 0xFFFFFF
    assert O.colour_key(1, 0, 0) == 4 and O.colour_key(0, 1, 0) == 2 and O.colour_key(0, 0, 1) == 1
    assert O.colour_key(2, 0, 0) == 32 and O.colour_key(128, 0, 0) == 1 << 23
    assert O.colour_key(0, 128, 1) == (1 << 22) | 1


def test_morton_hand_values(O):
    assert O.morton30(1023, 0, 0) == 0x24924924
    assert O.morton30(0, 1023, 0) == 0x12492492
    assert O.morton30(0, 0, 1023) == 0x09249249
    assert O.morton30(1, 1, 1) == 7 and O.morton30(512, 0, 0) == 1 << 29


def _np_plan(pos, q, group_size):
    """Independent numpy restatement: Morton rank -> chunks -> (chunk, key, rank) order."""
    n = pos.shape[0]
    lo = pos.min(axis=0)
    ext = (pos.max(axis=0) - lo).astype(np.float32)
    u = np.zeros((n, 3), np.int64)
    for a in range(3):
        if ext[a] != 0:
            t = np.float32(pos[:, a] - lo[a]) / ext[a]
            u[:, a] = np.minimum(1023, np.floor(t.astype(np.float32) * np.float32(1024)).astype(np.int64))
    m = np.zeros(n, np.int64)
    for i in range(10):
        m |= ((u[:, 0] >> i) & 1) << (3 * i + 2)
        m |= ((u[:, 1] >> i) & 1) << (3 * i + 1)
        m |= ((u[:, 2] >> i) & 1) << (3 * i)
    rank_order = np.lexsort((np.arange(n), m))        # by Morton, original index breaks ties
    rank = np.empty(n, np.int64)
    rank[rank_order] = np.arange(n)
    dc = q[:, 0, :].astype(np.int64)
    key = np.zeros(n, np.int64)
    for i in range(8):
        key |= ((dc[:, 0] >> i) & 1) << (3 * i + 2)
        key |= ((dc[:, 1] >> i) & 1) << (3 * i + 1)
        key |= ((dc[:, 2] >> i) & 1) << (3 * i)
    chunk = rank // group_size if group_size else np.zeros(n, np.int64)
    order = np.lexsort((rank, key, chunk))
    return order, key, chunk


@pytest.mark.parametrize("n,gs", [(4096, 4096), (1000, 256), (777, 16), (4096, 0), (33, 32), (1, 16)])
def test_plan_matches_independent_restatement(O, n, gs):
    sc = S.make_scene(n, 100 + n, clusters=5)
    q = O.quantise(sc.sh, O.scales(sc.sh))
    perm = O.plan(sc.pos, q, gs, 1)
    order, key, chunk = _np_plan(sc.pos, q, gs)
    assert perm.shape[0] == (n + 15) // 16 * 16
    assert np.array_equal(perm[:n], order)
    assert np.all(perm[n:] == -1)
    # invariants: bijection, keys non-decreasing inside chunks, chunks non-decreasing
    assert np.array_equal(np.sort(perm[:n]), np.arange(n))
    ch = chunk[perm[:n]]
    k = key[perm[:n]]
    assert np.all(np.diff(ch) >= 0)
    same = np.diff(ch) == 0
    assert np.all(np.diff(k)[same] >= 0)


def test_colour_ties_keep_spatial_order(O):
    # equal colour keys inside a chunk keep the spatial (Morton) order, not the storage order: a
    # scene whose DC colours all quantise alike, stored in a shuffled order
    n = 600
    sc = S.make_scene(n, 41, clusters=4)
    sh = sc.sh.copy()
    sh[:, 0, :] = 0.25                                    # one DC colour for every Gaussian
    q = O.quantise(sh, O.scales(sh))
    assert len({tuple(x) for x in q[:, 0, :]}) == 1
    for gs in (0, 128):
        perm = O.plan(sc.pos, q, gs, 1)
        order, _, _ = _np_plan(sc.pos, q, gs)
        assert np.array_equal(perm[:n], order)
        # with one colour the colour sort changes nothing: the slot order is the spatial rank
        lo, hi = sc.pos.min(axis=0), sc.pos.max(axis=0)
        g = np.minimum(np.floor((sc.pos - lo) / (hi - lo) * 1024).astype(np.int64), 1023)
        m = np.array([O.morton30(*map(int, r)) for r in g], np.int64)
        assert np.array_equal(perm[:n], np.lexsort((np.arange(n), m)))
        assert not np.array_equal(perm[:n], np.arange(n))


def test_plan_group16_sorts_each_group(O):
    # G = 16: every group is its own spatial chunk, sorted by colour inside
    sc = S.make_scene(512, 5)
    q = O.quantise(sc.sh, O.scales(sc.sh))
    p16 = O.plan(sc.pos, q, 16, 1)
    p_all = O.plan(sc.pos, q, 0, 1)
    _, key, _ = _np_plan(sc.pos, q, 16)
    for g in range(32):
        assert np.all(np.diff(key[p16[16 * g:16 * g + 16]]) >= 0)
    # G = 0 sorts the whole scene by colour
    assert np.all(np.diff(key[p_all]) >= 0)


def test_plan_unsorted_is_identity_and_padded(O):
    sc = S.make_scene(50, 9)
    q = O.quantise(sc.sh, O.scales(sc.sh))
    perm = O.plan(sc.pos, q, 4096, 0)
    assert np.array_equal(perm[:50], np.arange(50)) and np.all(perm[50:64] == -1)


def test_plan_empty_and_degenerate(O):
    perm = O.plan(np.zeros((0, 3), np.float32), np.zeros((0, 16, 3), np.uint8), 4096, 1)
    assert perm.size == 0
    # all positions equal: zero extent on every axis, order falls back to colour then index
    pos = np.full((40, 3), 0.25, np.float32)
    q = np.random.default_rng(1).integers(0, 256, size=(40, 16, 3)).astype(np.uint8)
    perm = O.plan(pos, q, 16, 1)
    order, _, _ = _np_plan(pos, q, 16)
    assert np.array_equal(perm[:40], order)
    with pytest.raises(ValueError):
        O.plan(pos, q, 24, 1)          # group size must be a multiple of 16


def test_stage_layout_d(O):
    # Fig. SetupD: block k of group g, texel t = coefficient k of slot 16 g + t; pads repeat the last valid slot
    rng = np.random.default_rng(3)
    n = 37
    q = rng.integers(0, 256, size=(n, 16, 3)).astype(np.uint8)
    perm = np.concatenate([rng.permutation(n).astype(np.int32), np.full(11, -1, np.int32)])
    st = O.stage(q, perm)
    assert st.shape == (3, 16, 16, 3)
    for g in range(3):
        for t in range(16):
            s = 16 * g + t
            src = perm[s] if perm[s] >= 0 else perm[16 * 2 + 4]      # last valid slot is 36
            for k in range(16):
                assert np.array_equal(st[g, k, t], q[src, k])
