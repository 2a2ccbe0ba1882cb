"""Pins of the oracle's block layouts A and B (Sec. IV-B, Figs. SetupA and SetupB, Table I).

Fig. SetupA moves the 16 RGB vectors of one Gaussian into one 4x4 block; Fig. SetupB moves the
64 RGB vectors of four Gaussians into four blocks, and Table I codes the first four SH
coefficients of that layout in BC7 and the rest in BC1 at 10 bytes per Gaussian. The texel
placement inside a block is not printed (raster order, row = Gaussian in B, is the reading).
The pins: the captions' content per block, the byte column of Table I, lossless BC7 round trips of
data that is constant inside every block of the layout (exactly representable, so the least-error
search must reproduce it; under layout D the layout-A data is not, and comes back lossy), the byte
order of a mixed coding, and the padding rule.
"""
import numpy as np
import pytest

from paper_2607_14513_gb300 import synthetic as S

D, A, B = 0, 1, 2


def test_each_layout_places_every_vector_of_a_group_once(O):
    for lay in (D, A, B):
        seen = {O.layout_map(lay, k, t) for k in range(16) for t in range(16)}
        assert seen == {(u, c) for u in range(16) for c in range(16)}, lay


def test_layout_a_block_is_one_gaussian(O):
    # Fig. SetupA: the 16 vectors of one primitive fill one block
    for k in range(16):
        slots = {O.layout_map(A, k, t)[0] for t in range(16)}
        coefs = sorted(O.layout_map(A, k, t)[1] for t in range(16))
        assert len(slots) == 1 and coefs == list(range(16))
    assert len({O.layout_map(A, k, 0)[0] for k in range(16)}) == 16


def test_layout_b_quad_holds_four_gaussians_first_block_first_coefficients(O):
    # Fig. SetupB: four primitives' 64 vectors in four blocks; Table I: the first of the four blocks
    # carries the first four SH coefficients (bands 0 and 1)
    for v in range(4):
        slots = {O.layout_map(B, 4 * v + b, t)[0] for b in range(4) for t in range(16)}
        assert slots == {4 * v + i for i in range(4)}
        for b in range(4):
            cells = [O.layout_map(B, 4 * v + b, t) for t in range(16)]
            assert {c for _, c in cells} == {4 * b + j for j in range(4)}
            assert sorted(cells) == sorted((u, c) for u in slots for c in range(4 * b, 4 * b + 4))


def test_layout_b_placement_rows_are_gaussians(O):
    # the reading of the placement inside a B block (the figure shows the blocks, not their texel
    # order): raster order, row i = the quad's Gaussian i, column j = coefficient 4b + j; hand values
    for k, t, want in ((0, 0, (0, 0)), (0, 3, (0, 3)), (0, 4, (1, 0)), (1, 6, (1, 6)), (5, 6, (5, 6)),
                       (6, 13, (7, 9)), (15, 15, (15, 15)), (12, 2, (12, 2)), (3, 12, (3, 12))):
        assert O.layout_map(B, k, t) == want, (k, t)


def test_fixed_codings_match_table_one_bytes(O):
    # Table I "SH bytes": layout A BC1 8, BC7 16; layout B BC7 on the first block, BC1 on the rest 10
    sc = S.make_scene(**S.TINY)
    n = 256
    q = O.quantise(sc.sh[:n], O.scales(sc.sh[:n]))
    perm = np.arange(n, dtype=np.int32)
    # (layout D, BC7 first: the block bytes; Table I prints one block per group more, 9)
    for lay, j, want in ((A, 0, 8.0), (A, 16, 16.0), (B, 4, 10.0), (B, 0, 8.0), (B, 16, 16.0), (D, 1, 8.5)):
        r = O.encode_layout(q, perm, O.scales(sc.sh[:n]), lay, j)
        assert r["table"].total_bytes / n == want, (lay, j)
        assert r["table"].layout == lay and r["table"].s[0].bc7_blocks == j
    assert not O.layout_ok(A, 4) and not O.layout_ok(B, 2) and O.layout_ok(B, 12) and O.layout_ok(D, 3)


def _constant_per_block_scene(O, lay, n, rng):
    """Texels that are constant inside every block of `lay` (in slot order = original order). The
    channels are even, so BC7 mode 6 (7-bit endpoints, p-bit 0 on both) codes the block exactly and
    the least-error search must reach zero error."""
    q = np.zeros((n, 16, 3), np.uint8)
    if lay == A:
        q[:] = 2 * rng.integers(0, 128, size=(n, 1, 3))
    else:  # B: one colour per (quad, block)
        col = 2 * rng.integers(0, 128, size=((n + 3) // 4, 4, 3))
        for i in range(n):
            for c in range(16):
                q[i, c] = col[i // 4, c // 4]
    return q


@pytest.mark.parametrize("lay", [A, B])
def test_bc7_round_trip_is_lossless_when_blocks_are_constant(O, lay):
    rng = np.random.default_rng(40 + lay)
    n = 64
    q = _constant_per_block_scene(O, lay, n, rng)
    perm = np.arange(n, dtype=np.int32)
    sc = np.ones(16, np.float32)
    r = O.encode_layout(q, perm, sc, lay, 16)
    assert np.array_equal(O.decode(r["table"], r["blocks"], r["perm"]), q)
    if lay == A:
        # the same data in layout D puts 16 Gaussians' colours in a block: not representable, lossy
        # (layout B's test data is row-structured in D blocks, which two-subset BC7 still codes exactly)
        rd = O.encode_layout(q, perm, sc, D, 16)
        assert not np.array_equal(O.decode(rd["table"], rd["blocks"], rd["perm"]), q)


def test_mixed_b_decodes_each_block_with_its_format(O):
    # layout B, j = 4: block 0 of each quad BC7, blocks 1-3 BC1; every texel equals the
    # corresponding block decoder's output on the staged texels
    sc = S.make_scene(**S.TINY)
    n = 100   # ragged: 7 groups, the last with 4 valid slots
    osc = O.scales(sc.sh[:n])
    q = O.quantise(sc.sh[:n], osc)
    perm = O.plan(sc.pos[:n], q, 4096, 1)
    r = O.encode_layout(q, perm, osc, B, 4)
    dec = O.decode(r["table"], r["blocks"], r["perm"])
    st = O.stage_layout(q, perm, B).reshape(-1, 16, 16, 3)
    ng = st.shape[0]
    b7 = np.asarray(O.encode_blocks(st[:, [0, 4, 8, 12]].reshape(-1, 16, 3), 7)[0]).reshape(ng, 4, 16)
    b1 = np.asarray(O.encode_blocks(st[:, [k for k in range(16) if k % 4]].reshape(-1, 16, 3), 1)[0]).reshape(ng, 12, 8)
    # byte layout: a group's four BC7 blocks (blocks 0, 4, 8, 12), then its twelve BC1 blocks
    grp = r["blocks"].reshape(ng, 160)
    assert np.array_equal(grp[:, :64].reshape(ng, 4, 16), b7)
    assert np.array_equal(grp[:, 64:].reshape(ng, 12, 8), b1)
    d7 = O.decode_blocks(b7.reshape(-1, 16), 7)[:, :, :3].reshape(ng, 4, 16, 3)
    d1 = O.decode_blocks(b1.reshape(-1, 8), 1)[:, :, :3].reshape(ng, 12, 16, 3)
    blk = np.zeros((ng, 16, 16, 3), np.uint8)
    blk[:, [0, 4, 8, 12]] = d7
    blk[:, [k for k in range(16) if k % 4]] = d1
    for g in range(ng):
        for k in range(16):
            for t in range(16):
                u, c = O.layout_map(B, k, t)
                o = perm[16 * g + u]
                if o >= 0:
                    assert np.array_equal(dec[o, c], blk[g, k, t])


@pytest.mark.parametrize("lay", [D, A, B])
def test_padding_slots_repeat_the_last_valid_slot(O, lay):
    rng = np.random.default_rng(7)
    n = 21   # group 1 has slots 16..20 valid, 21..31 padding
    q = rng.integers(0, 256, size=(n, 16, 3)).astype(np.uint8)
    perm = np.full(32, -1, np.int32)
    perm[:n] = rng.permutation(n)
    st = O.stage_layout(q, perm, lay)
    for k in range(16):
        for t in range(16):
            u, c = O.layout_map(lay, k, t)
            src = perm[16 + min(u, 4)]          # slots 21..31 repeat slot 20
            assert np.array_equal(st[1, k, t], q[src, c])
    if lay == D:
        assert np.array_equal(st, O.stage(q, perm))
