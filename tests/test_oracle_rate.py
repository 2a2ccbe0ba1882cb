"""Pins of the oracle's rate control (Sec. IV-B: several fixed-rate bitstreams give a
variable number of bits per primitive while keeping random access; Figs. SetupC/SetupD:
zero high-order coefficients are not stored; Table I rate arithmetic).

The paper gives the mechanism but no allocation algorithm; the integer Lagrangian
choice among 14 group modes is this codec's reading. The pins are the rate arithmetic
the paper prints, an exhaustive knapsack on tiny instances, monotonicity and the budget.
"""
import itertools

import numpy as np
import pytest

from paper_2607_14513_gb300 import synthetic as S


def test_mode_rates_match_table_one_arithmetic(O):
    b, j = O.mode_table()
    assert list(zip(b.tolist(), j.tolist())) == [(1, 0), (1, 1), (4, 0), (4, 1), (4, 4), (9, 0), (9, 1), (9, 4),
                                                 (9, 9), (16, 0), (16, 1), (16, 4), (16, 9), (16, 16)]
    bytes_per_gaussian = {(int(bb), int(jj)): (16 * jj + 8 * (bb - jj)) / 16 for bb, jj in zip(b, j)}
    # Table I, Setup D rows: all BC1 -> 8 B, BC7 first + BC1 rest -> 8.5 B, all BC7 -> 16 B per primitive
    # (8 B per BC1 block, 16 B per BC7 block; the table prints 8.5 / 9 / 17, one more block per group
    # of 16 primitives in the format of the group's other blocks)
    assert bytes_per_gaussian[(16, 0)] == 8.0
    assert bytes_per_gaussian[(16, 1)] == 8.5
    assert bytes_per_gaussian[(16, 16)] == 16.0
    assert all(len({64 * (int(x) + int(y)) for x, y in zip(b, j)}) == 14 for _ in [0])   # rates are distinct


def _rates(O):
    b, j = O.mode_table()
    return 64 * (b.astype(np.int64) + j.astype(np.int64))


def _random_D(rng, ng):
    # distortions that mostly fall with rate, with noise so the hull is non-trivial
    R = np.array([1, 2, 4, 5, 8, 9, 10, 13, 18, 16, 17, 20, 25, 32], np.float64)
    base = rng.uniform(1e3, 1e7, size=(ng, 1)) * np.exp(-R[None, :] * rng.uniform(0.05, 0.3, size=(ng, 1)))
    return (base * rng.uniform(0.7, 1.3, size=(ng, 14))).astype(np.uint64)


def test_lagrangian_choice_is_on_the_hull(O):
    # exhaustive knapsack over 14^4 assignments: at lambda*, no assignment of no more total
    # rate has lower total distortion
    rng = np.random.default_rng(21)
    R = _rates(O)
    for trial in range(6):
        ng = 4
        D = _random_D(rng, ng)
        budget = int(rng.integers(R.min() * ng, R.max() * ng))
        rc, mode, lam = O.rate_control(D, budget)
        assert rc == 0
        base = O.rate_choose(D, lam)
        r_star = int(R[base].sum())
        d_star = int(D[np.arange(ng), base].sum())
        combos = np.array(list(itertools.product(range(14), repeat=ng)))
        rr = R[combos].sum(axis=1)
        dd = D[np.arange(ng)[None, :], combos].astype(np.float64).sum(axis=1)
        assert dd[rr <= r_star].min() >= d_star - 1e-6 * d_star
        # lambda* is the smallest feasible multiplier
        assert r_star <= budget
        if lam > 0:
            assert int(R[O.rate_choose(D, lam - 1)].sum()) > budget
        # the fill step stays within the budget and only raises rates
        used = int(R[mode].sum())
        assert r_star <= used <= budget
        assert np.all(R[mode] >= R[base])


def test_budget_met_exactly(O):
    # a budget equal to the total rate of some multiplier's choice is met exactly: lambda* is the
    # smallest multiplier whose choice fits (total <= budget), so its total equals the budget
    rng = np.random.default_rng(24)
    R = _rates(O)
    D = _random_D(rng, 12)
    lams = sorted(set(int(x) for x in np.exp(rng.uniform(0, 40, size=40))))
    seen = 0
    for l in lams:
        budget = int(R[O.rate_choose(D, l)].sum())
        rc, mode, lam = O.rate_control(D, budget)
        assert rc == 0
        assert int(R[O.rate_choose(D, lam)].sum()) == budget
        assert lam == 0 or int(R[O.rate_choose(D, lam - 1)].sum()) > budget
        assert int(R[mode].sum()) == budget
        seen += lam > 0
    assert seen > 10


def test_distortion_table_is_dequantised_squared_error(O):
    # Sec. IV-B trades rate against the distortion of the decoded colours. Reading: a group's
    # distortion under a coding is the squared error of the dequantised coefficients it leaves,
    # x' = (q - 128) / 255 * s_k (Sec. V-A): BC7 blocks for the first j coefficients, BC1 blocks up
    # to b, dropped coefficients (x' = 0) after. Checked against block errors computed here from
    # the block coders, up to one positive factor; the table's integer weights round that factor
    # per coefficient, which bounds the slack by one unit of weight per unit of block error.
    sc = S.make_scene(512, 31)
    scl = O.scales(sc.sh)
    q = O.quantise(sc.sh, scl)
    perm = O.plan(sc.pos, q, 256, 1)
    D = O.encode(q, perm, scl, 0, 24, want_dtab=True)["dtab"].astype(np.float64)
    tex = O.stage(q, perm).astype(np.int64)                       # [groups, block k, texel, channel]
    ng = tex.shape[0]
    flat = tex.reshape(-1, 16, 3).astype(np.uint8)
    dec = {f: O.decode_blocks(O.encode_blocks(flat, f)[0], f)[..., :3].reshape(ng, 16, 16, 3).astype(np.int64)
           for f in (1, 7)}
    e1 = ((dec[1] - tex) ** 2).sum(axis=(2, 3))
    e7 = ((dec[7] - tex) ** 2).sum(axis=(2, 3))
    e0 = ((tex - 128) ** 2).sum(axis=(2, 3))
    b, j = O.mode_table()
    k = np.arange(16)
    s2 = scl.astype(np.float64) ** 2
    E = np.zeros_like(D)
    U = np.zeros_like(D)
    for m in range(14):
        e = np.where(k < j[m], e7, np.where(k < b[m], e1, e0))
        E[:, m] = (e * s2).sum(axis=1)
        U[:, m] = e.sum(axis=1)
    c = (D * E).sum() / (E * E).sum()
    assert c > 0
    assert np.all(np.abs(D - c * E) <= U + 1e-9 * D)
    assert (E > 0).mean() > 0.9


def test_rate_monotone_in_lambda(O):
    rng = np.random.default_rng(22)
    R = _rates(O)
    D = _random_D(rng, 200)
    lams = [0] + sorted(set(int(x) for x in np.exp(rng.uniform(0, 60, size=60))))
    tot = [int(R[O.rate_choose(D, l)].sum()) for l in lams]
    assert all(a >= b for a, b in zip(tot, tot[1:]))
    assert int(R[O.rate_choose(D, 1 << 62)].sum()) == 64 * 200      # huge lambda: cheapest mode everywhere


def test_budget_infeasible_and_exact(O):
    rng = np.random.default_rng(23)
    D = _random_D(rng, 10)
    rc, _, _ = O.rate_control(D, 64 * 10 - 1)
    assert rc != 0
    rc, mode, _ = O.rate_control(D, 2048 * 10)
    assert rc == 0 and np.all(mode == 13)               # everything affordable: the all-BC7 mode wins
    # groups whose distortion does not depend on the mode take the cheapest mode
    rc, mode, lam = O.rate_control(np.full((5, 14), 1000, np.uint64), 10_000)
    assert rc == 0 and np.all(mode == 0)


@pytest.mark.parametrize("fmt,bpt", [(1, 4), (7, 8)])
def test_forced_formats_hit_their_rate(O, fmt, bpt):
    sc = S.make_scene(512, 31)
    r = O.full_encode(sc.pos, sc.sh, fmt)
    t = r["table"]
    assert t.used_bits == bpt * 16 * 512
    assert t.total_bytes == (16 if fmt == 7 else 8) * 16 * 512 // 16


@pytest.mark.parametrize("target_x4", [12, 16, 24, 32])
def test_rate_targets_respect_budget(O, target_x4):
    n = 480                                      # 30 groups, not a power of two
    sc = S.make_scene(n, 32)
    r = O.full_encode(sc.pos, sc.sh, 0, target_x4=target_x4)
    t = r["table"]
    budget = target_x4 * 4 * n
    assert t.budget_bits == budget
    assert t.used_bits <= budget
    # within one group's largest upgrade of the budget
    assert t.used_bits > budget - 64 * 32
    # streams: consecutive, by mode id, offsets add up
    off, g = 0, 0
    for i in range(t.n_streams):
        s = t.s[i]
        assert s.first_group == g and s.byte_offset == off
        g += s.n_groups
        off += s.n_groups * (16 * s.bc7_blocks + 8 * (s.bands - s.bc7_blocks))
    assert g == t.n_groups and off == t.total_bytes


def test_rate_path_split_and_threads_change_nothing():
    # coding all groups once (over several threads) and assembling per target gives exactly the
    # single-call serial encode at every target
    import numpy as np
    from oracle import oracle as O
    from paper_2607_14513_gb300 import synthetic as S
    O.lib()
    sc = S.make_scene(1500, 711, heavy_frac=0.1)
    osc = O.scales(sc.sh)
    q = O.quantise(sc.sh, osc)
    perm = O.plan(sc.pos, q, 256, 1)
    targets = (12, 24)
    outs = O.encode_rates(q, perm, osc, targets, threads=4)
    for t4, o in zip(targets, outs):
        r = O.encode(q, perm, osc, 0, t4)
        assert np.array_equal(r["blocks"], o["blocks"]) and np.array_equal(r["perm"], o["perm"])
        assert (r["table"].lambda_, r["table"].used_bits, r["table"].budget_bits) == \
            (o["table"].lambda_, o["table"].used_bits, o["table"].budget_bits)
        assert [r["table"].s[i].n_groups for i in range(14)] == [o["table"].s[i].n_groups for i in range(14)]
