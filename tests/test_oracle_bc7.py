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
    # ties: blocks that many candidates code without error take the first of them (constant
    # blocks have their own rule, test_constant_colours_round_trip_wherever_reachable)
    ties = [np.where((np.arange(16) % 2)[:, None] == 0, [16, 32, 48], [200, 100, 50]).astype(np.uint8),
            np.where((np.arange(16) < 8)[:, None], [66, 132, 198], [0, 255, 0]).astype(np.uint8)]
    for tex in ties:
        errs = np.array([O.bc7_candidate(tex, e)[0] for e in range(ne)])
        assert (errs == errs.min()).sum() > 1
        blocks, _ = O.encode_blocks(tex[None], 7, threads=1)
        assert np.array_equal(blocks[0], O.bc7_candidate(tex, int(np.argmin(errs)))[1])


W2 = [0, 21, 43, 64]
W3 = [0, 9, 18, 27, 37, 46, 55, 64]


def _expand(v, n):
    return v if n >= 8 else (v << (8 - n)) | (v >> (2 * n - 8))


def _reach(bits, p0, p1, has_p, w):
    """8-bit values ((64 - w) e0 + w e1 + 32) >> 6 of all endpoint code pairs (with p-bits)."""
    codes = np.arange(1 << bits)
    e0 = np.array([_expand((c << 1) | p0 if has_p else c, bits + has_p) for c in codes])
    e1 = np.array([_expand((c << 1) | p1 if has_p else c, bits + has_p) for c in codes])
    out = np.zeros(256, bool)
    out[((64 - w) * e0[:, None] + w * e1[None, :] + 32) >> 6] = True
    return out


def _constant_reach_sets():
    """Per mode, the (R, G, B) value sets whose product a constant block reaches exactly: every
    texel takes one index weight, p-bits are shared by an endpoint's channels; modes 4 and 5 code
    the rotated channel in the alpha endpoints with their own index."""
    sets = {}
    # mode: colour bits, p-bit kind (0 none, 1 per endpoint, 2 shared by the endpoints), index weights
    for m, bits, pk, ws in ((0, 4, 1, W3), (1, 6, 2, W3), (2, 5, 0, W2), (3, 7, 1, W2), (6, 7, 1, W4), (7, 5, 1, W2)):
        combos = [(0, 0)] if pk == 0 else ([(a, b) for a in (0, 1) for b in (0, 1)] if pk == 1 else [(0, 0), (1, 1)])
        sets[m] = [(r, r, r) for p0, p1 in combos for w in ws for r in [_reach(bits, p0, p1, pk > 0, w)]]
    for m, cb, ab, pairs in ((4, 5, 6, ((W2, W3), (W3, W2))), (5, 7, 8, ((W2, W2),))):
        sets[m] = []
        for cw, aw in pairs:
            alpha = np.zeros(256, bool)
            for w in aw:
                alpha |= _reach(ab, 0, 0, 0, w)
            for w in cw:
                c = _reach(cb, 0, 0, 0, w)
                sets[m] += [(c, c, c), (alpha, c, c), (c, alpha, c), (c, c, alpha)]
    return sets


def test_constant_colours_round_trip_wherever_reachable(O):
    # Sec. III-A: a block whose texels are one colour can be coded without error where the format
    # reaches the colour. The brute force above decides reachability from the format alone; every
    # colour reached by some mode must come back exactly.
    sets = _constant_reach_sets()
    reach = lambda c: [m for m, ss in sets.items() if any(R[c[0]] and G[c[1]] and B[c[2]] for R, G, B in ss)]
    rng = np.random.default_rng(14)
    cols = [(v, v, v) for v in range(256)] + [(v, 37, 200) for v in range(256)] + [(9, v, 90) for v in range(256)]
    cols += [(250, 3, v) for v in range(256)] + [tuple(int(x) for x in rng.integers(0, 256, 3)) for _ in range(1500)]
    modes = [reach(c) for c in cols]
    assert all(5 in ms for ms in modes)      # mode 5 at weight 21 reaches every value ...
    assert any(2 not in ms for ms in modes)  # ... which mode 2 (5-bit, no p-bits) does not
    grey = [sum(any(R[v] and G[v] and B[v] for R, G, B in sets[m]) for v in range(256)) for m in range(8)]
    assert grey == [255, 256, 210, 256, 255, 256, 256, 251]
    tex = np.array([np.tile(np.array(c, np.uint8), (16, 1)) for c in cols])
    blocks, sse = O.encode_blocks(tex, 7, threads=8)
    assert np.all(sse == 0)
    for i in range(len(cols)):
        assert np.array_equal(O.bc7_decode(blocks[i])[:, :3], tex[i]), cols[i]
    # the encoder's constant rule: mode 5 (first byte 0b00100000), rotation 0, colour index 1
    assert np.all(blocks[:, 0] == 0x20)
    bits = [int.from_bytes(bytes(b), "little") for b in blocks[:8]]
    for v in bits:
        assert (v >> 6) & 3 == 0                              # rotation
        ci = v >> 66                                          # 6 + 2 + 42 + 16 header and endpoint bits
        assert ci & 1 == 1 and all((ci >> (1 + 2 * t)) & 3 == 1 for t in range(15))


def test_mode6_fit_least_squares_by_hand(O):
    # One-subset fit of the mode-6 candidate (7-bit endpoints, a p-bit per endpoint, 4-bit
    # indices), worked by hand. R varies, G = 100 and B = 50 are constant.
    R = [255] * 4 + [230] * 4 + [0] * 8
    tex = np.array([[r, 100, 50] for r in R], np.uint8)
    # bounding-box diagonal: R spans most, G and B do not vary: e0 = (255, 100, 50), e1 = (0, 100, 50)
    interp = lambda a, b, w: ((64 - w) * a + w * b + 32) >> 6
    # nearest weights against e0 / e1: 255 -> index 0 (w 0); 230 -> index 1 (w 4: 239, error 9;
    # index 2, w 9: 219, error 11); 0 -> index 15 (w 64)
    assert interp(255, 0, 4) == 239 and interp(255, 0, 9) == 219
    idx = [0] * 4 + [1] * 4 + [15] * 8
    a = [64 - W4[j] for j in idx]
    b = [W4[j] for j in idx]
    # normal equations of the least-squares endpoints E0, E1 minimising sum (a E0 + b E1 - 64 v)^2
    saa = 4 * 64 * 64 + 4 * 60 * 60 + 8 * 0
    sbb = 4 * 0 + 4 * 4 * 4 + 8 * 64 * 64
    sab = 4 * 0 + 4 * 60 * 4 + 8 * 0
    sav = 4 * 64 * 255 + 4 * 60 * 230
    sbv = 4 * 4 * 230
    assert (saa, sbb, sab, sav, sbv) == (30784, 32832, 960, 120480, 3680)
    assert (saa, sbb, sab) == (sum(x * x for x in a), sum(y * y for y in b), sum(x * y for x, y in zip(a, b)))
    assert (sav, sbv) == (sum(x * v for x, v in zip(a, R)), sum(y * v for y, v in zip(b, R)))
    det = saa * sbb - sab * sab
    assert det == 1009778688
    # E0 = 64 (sbb sav - sab sbv) / det = 252932259840 / det = 250.48 -> 250
    # E1 = 64 (saa sbv - sab sav) / det = -152043520 / det = -0.15 -> 0
    assert 64 * (sbb * sav - sab * sbv) == 252932259840 and 64 * (saa * sbv - sab * sav) == -152043520
    # (G and B: 64 (sbb - sab) sum(a) v / det = v exactly for a constant channel)
    # p-bits: (0, 0) codes (250, 100, 50) and (0, 100, 50) exactly (all even); re-indexed, 255 -> 250
    # (error 5), 230 -> interp(250, 0, w 4) = 234 (error 4), 0 -> 0: error 4 (25 + 16) = 164; the other
    # combinations move G or B off by one on every texel and cost more
    assert interp(250, 0, 4) == 234
    sse, blk = O.bc7_candidate(tex, 16 + 192 + 8 + 4)   # the mode-6 candidate
    dec = O.bc7_decode(blk)[:, :3].astype(int)
    assert sse == 164
    assert dec[:, 0].tolist() == [250] * 4 + [234] * 4 + [0] * 8
    assert np.all(dec[:, 1] == 100) and np.all(dec[:, 2] == 50)


def test_nearest_code_ties_go_to_the_lower_code(O):
    # The mode-6 candidate of the constant colour (254, 101, 51): the fit keeps e0 = e1 = the colour.
    # With p-bit 1 an endpoint's values are odd, and 254 lies halfway between 253 (code 126) and 255
    # (code 127): the lower code wins. With p0 = 1, p1 = 0 the block codes (253, 101, 51) and
    # (254, 100, 50); index 0 everywhere costs 1 per texel (16), less than (0, 0) (G and B off by one:
    # 32) and no more than (0, 1) or (1, 1) (16 each, later in the order)
    tex = np.tile(np.array([254, 101, 51], np.uint8), (16, 1))
    sse, blk = O.bc7_candidate(tex, 16 + 192 + 8 + 4)
    assert sse == 16
    assert O.bc7_decode(blk)[:, :3].tolist() == [[253, 101, 51]] * 16


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
