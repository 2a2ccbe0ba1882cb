"""Pins of the oracle's BC7 decoder and encoder (Sec. III-B; D3D11 / Khronos BC7 format).

The format fixes the mode table, the bit layout (LSB first: unary mode, partition,
rotation, index selection, colour endpoints R..G..B per subset and endpoint, alpha
endpoints, p-bits, primary then secondary indices, anchors one bit shorter), the
weight tables and interpolation, and the partition and anchor tables. The partition
and anchor tables are also checked against the GB300 texture unit in the GPU tests.
"""
import numpy as np
import pytest

W4 = [0, 4, 9, 13, 17, 21, 26, 30, 34, 38, 43, 47, 51, 55, 60, 64]


class Bits:
    """LSB-first bit writer for hand-built blocks."""

    def __init__(self):
        self.v = 0
        self.n = 0

    def put(self, val, nbits):
        self.v |= (val & ((1 << nbits) - 1)) << self.n
        self.n += nbits
        return self

    def block(self):
        assert self.n == 128, self.n
        return np.frombuffer(self.v.to_bytes(16, "little"), np.uint8).copy()


def test_partition_and_anchor_invariants(O):
    for ns in (2, 3):
        rows = set()
        for p in range(64):
            sub = [O.bc7_subset(ns, p, t) for t in range(16)]
            rows.add(tuple(sub))
            assert sub[0] == 0                                      # texel 0 always opens subset 0
            assert set(sub) == set(range(ns))                       # every subset is used
            anchors = [O.bc7_anchor(ns, p, s) for s in range(ns)]
            assert anchors[0] == 0 and len(set(anchors)) == ns
            for s in range(ns):
                assert sub[anchors[s]] == s                         # each anchor lies in its own subset
        assert len(rows) == 64                                      # all partitions distinct
    # literal rows of the format's tables
    assert [O.bc7_subset(2, 0, t) for t in range(16)] == [0, 0, 1, 1] * 4
    assert [O.bc7_subset(2, 13, t) for t in range(16)] == [0] * 8 + [1] * 8
    assert [O.bc7_subset(3, 8, t) for t in range(16)] == [0] * 8 + [1] * 4 + [2] * 4
    assert [O.bc7_subset(3, 37, t) for t in range(16)] == [0, 1, 2, 0, 1, 2, 0, 1, 2, 0, 1, 2, 0, 1, 2, 0]


def test_hand_built_mode6_gradient(O):
    # mode 6: R endpoints 0 (code 0, p 0) and 255 (code 127, p 1); G, B codes 0 -> 0 / 1; A codes 127 -> 254 / 255
    b = Bits().put(1 << 6, 7)
    for c0, c1 in [(0, 127), (0, 0), (0, 0), (127, 127)]:
        b.put(c0, 7).put(c1, 7)
    b.put(0, 1).put(1, 1)
    b.put(0, 3)
    for t in range(1, 16):
        b.put(t, 4)
    out = O.bc7_decode(b.block())
    expect_r = [0, 16, 36, 52, 68, 84, 104, 120, 135, 151, 171, 187, 203, 219, 239, 255]
    for t in range(16):
        gb = 1 if W4[t] >= 32 else 0
        assert tuple(out[t]) == (expect_r[t], gb, gb, 254 + gb), t


def test_hand_built_mode6_solid(O):
    b = Bits().put(1 << 6, 7)
    for c0, c1 in [(127, 127), (0, 0), (64, 64), (127, 127)]:
        b.put(c0, 7).put(c1, 7)
    b.put(1, 1).put(1, 1).put(5, 3)
    for t in range(1, 16):
        b.put(15 - t, 4)
    out = O.bc7_decode(b.block())
    assert all(tuple(out[t]) == (255, 1, 129, 255) for t in range(16))


def test_hand_built_mode1_membership(O):
    # two subsets: subset 0 black, subset 1 white (codes 63 with shared p-bit 1)
    for p, pattern in [(0, [0, 0, 1, 1] * 4), (13, [0] * 8 + [1] * 8), (33, [0] * 4 + [1] * 4 + [0] * 4 + [1] * 4)]:
        b = Bits().put(2, 2).put(p, 6)
        for _c in range(3):
            b.put(0, 6).put(0, 6).put(63, 6).put(63, 6)
        b.put(0, 1).put(1, 1).put(0, 46)
        out = O.bc7_decode(b.block())
        for t in range(16):
            v = 255 * pattern[t]
            assert tuple(out[t]) == (v, v, v, 255)


def test_hand_built_mode1_shared_pbits_and_weights(O):
    # mode 1, partition 0 (texels 2, 3, 6, 7, 10, 11, 14, 15 in subset 1, anchor 15): 6-bit codes
    # with one p-bit per subset shared by both endpoints, 3-bit indices (anchors 0 and 15 two bits).
    # Subset 0: codes 0 / 63, p-bit 1 -> 7-bit 1 / 127 -> 2 / 255; subset 1: codes 10 / 50, p-bit 0
    # -> 7-bit 20 / 100 -> 40 / 201 (7-bit v expands to v << 1 | v >> 6)
    W3 = [0, 9, 18, 27, 37, 46, 55, 64]
    sub1 = {2, 3, 6, 7, 10, 11, 14, 15}
    idx = [(3 * t) % 8 for t in range(16)]
    idx[15] = 3
    b = Bits().put(2, 2).put(0, 6)
    for _c in range(3):
        b.put(0, 6).put(63, 6).put(10, 6).put(50, 6)
    b.put(1, 1).put(0, 1)
    for t in range(16):
        b.put(idx[t], 2 if t in (0, 15) else 3)
    out = O.bc7_decode(b.block())
    for t in range(16):
        e0, e1 = (40, 201) if t in sub1 else (2, 255)
        v = ((64 - W3[idx[t]]) * e0 + W3[idx[t]] * e1 + 32) >> 6
        assert tuple(out[t]) == (v, v, v, 255), t


def test_hand_built_mode4_rotation(O):
    # mode 4, rotation 1 (alpha <-> red), index selection 0: colour codes 0, alpha codes 63 -> 255
    b = Bits().put(1 << 4, 5).put(1, 2).put(0, 1)
    for _c in range(3):
        b.put(0, 5).put(0, 5)
    b.put(63, 6).put(63, 6)
    b.put(0, 31).put(0, 47)
    out = O.bc7_decode(b.block())
    assert all(tuple(out[t]) == (255, 0, 0, 0) for t in range(16))
    # mode 5, rotation 3 (alpha <-> blue): colour R endpoints 0 / 127 (7-bit -> 255), alpha 8-bit 10 / 20
    b = Bits().put(1 << 5, 6).put(3, 2)
    b.put(0, 7).put(127, 7).put(0, 7).put(0, 7).put(0, 7).put(0, 7)
    b.put(10, 8).put(20, 8)
    # colour indices (2-bit, texel 0 one bit): texel t -> t % 4 (texel 0 -> 0); alpha indices all 3 (texel 0: 1)
    b.put(0, 1)
    for t in range(1, 16):
        b.put(t % 4, 2)
    b.put(1, 1)
    for t in range(1, 16):
        b.put(3, 2)
    out = O.bc7_decode(b.block())
    W2 = [0, 21, 43, 64]
    for t in range(16):
        r = (W2[t % 4] * 255 + 32) >> 6
        a_slot = ((64 - W2[1 if t == 0 else 3]) * 10 + W2[1 if t == 0 else 3] * 20 + 32) >> 6
        assert tuple(out[t]) == (r, 0, a_slot, 0), t


def test_reserved_mode_decodes_to_zero(O):
    assert not O.bc7_decode(np.zeros(16, np.uint8)).any()
    blk = np.zeros(16, np.uint8)
    blk[1:] = 0xFF
    assert not O.bc7_decode(blk).any()


def test_every_candidate_packs_losslessly(O):
    # for every mode / partition / rotation / index selection, the packed block decodes to
    # exactly the error the search reported (this exercises the anchor swap of every subset)
    rng = np.random.default_rng(12)
    ne = O.bc7_n_candidates()
    assert ne == 16 + 64 * 3 + 8 + 4 + 1 + 64
    for trial in range(3):
        tex = rng.integers(0, 256, size=(16, 3)).astype(np.uint8)
        if trial == 1:
            tex = np.clip(rng.integers(90, 110, size=(16, 3)) + rng.integers(-3, 4, size=(16, 3)), 0, 255).astype(np.uint8)
        for e in range(ne):
            sse, blk = O.bc7_candidate(tex, e)
            dec = O.bc7_decode(blk)
            assert int(((dec[:, :3].astype(int) - tex.astype(int)) ** 2).sum()) == int(sse), e
            mode = int(blk[0] & -blk[0].astype(np.int16)).bit_length() - 1
            expect_mode = 0 if e < 16 else (1 + (e - 16) // 64 if e < 208 else (4 if e < 216 else (5 if e < 220 else (6 if e < 221 else 7))))
            assert mode == expect_mode


def test_encoder_is_the_first_minimum(O):
    rng = np.random.default_rng(13)
    ne = O.bc7_n_candidates()
    for _ in range(4):
        tex = rng.integers(0, 256, size=(16, 3)).astype(np.uint8)
        errs = [O.bc7_candidate(tex, e)[0] for e in range(ne)]
        first = int(np.argmin(errs))
        blocks, sse = O.encode_blocks(tex[None], 7, threads=1)
        assert int(sse[0]) == min(errs)
        assert np.array_equal(blocks[0], O.bc7_candidate(tex, first)[1])
    # ties: blocks that many candidates code without error take the first of them
    ties = [np.tile(np.array([64, 128, 200], np.uint8), (16, 1)),
            np.where((np.arange(16) % 2)[:, None] == 0, [16, 32, 48], [200, 100, 50]).astype(np.uint8)]
    for tex in ties:
        errs = np.array([O.bc7_candidate(tex, e)[0] for e in range(ne)])
        assert (errs == errs.min()).sum() > 1
        blocks, _ = O.encode_blocks(tex[None], 7, threads=1)
        assert np.array_equal(blocks[0], O.bc7_candidate(tex, int(np.argmin(errs)))[1])


def test_constant_colours(O):
    # colours whose channels share one parity are exact in mode 6 (7-bit codes + shared p-bit)
    rng = np.random.default_rng(14)
    cols = [(0, 0, 0), (255, 255, 255), (128, 64, 2), (1, 3, 255)]
    cols += [tuple((rng.integers(0, 128, size=3) * 2 + rng.integers(0, 2)).tolist()) for _ in range(10)]
    tex = np.array([np.tile(np.array(c, np.uint8), (16, 1)) for c in cols])
    _, sse = O.encode_blocks(tex, 7, threads=1)
    assert np.all(sse == 0)
    # any constant colour is reproduced within one level per channel
    cols = rng.integers(0, 256, size=(16, 3))
    tex = np.repeat(cols[:, None, :], 16, axis=1).astype(np.uint8)
    _, sse = O.encode_blocks(tex, 7, threads=4)
    assert np.all(sse <= 48)


def test_two_subset_partitions_exact(O):
    # each subset holds two colours with one channel parity each: mode 3 (7-bit + p-bit per
    # endpoint) represents them exactly, for every two-subset partition
    rng = np.random.default_rng(15)
    texs = []
    for p in range(64):
        cols = [(rng.integers(0, 128, size=3) * 2 + rng.integers(0, 2)) for _ in range(4)]
        tex = np.zeros((16, 3), np.uint8)
        for t in range(16):
            s = O.bc7_subset(2, p, t)
            tex[t] = cols[2 * s + (t * 7 + p) % 2]
        texs.append(tex)
    _, sse = O.encode_blocks(np.array(texs), 7, threads=8)
    assert np.all(sse == 0)


def test_three_subset_partitions_exact(O):
    # three subsets of two 5-bit-expandable colours each: mode 2 (5-bit endpoints) is exact
    ex5 = lambda v: (v << 3) | (v >> 2)
    rng = np.random.default_rng(16)
    texs = []
    for p in range(64):
        cols = [ex5(rng.integers(0, 32, size=3)) for _ in range(6)]
        tex = np.zeros((16, 3), np.uint8)
        for t in range(16):
            s = O.bc7_subset(3, p, t)
            tex[t] = cols[2 * s + (t * 5 + p) % 2]
        texs.append(tex)
    _, sse = O.encode_blocks(np.array(texs), 7, threads=8)
    assert np.all(sse == 0)
