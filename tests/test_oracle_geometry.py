"""Pins of the oracle's geometry streams and chunk hierarchy (Sec. IV-A: position and shape coded
apart from appearance, each parameter quantised to a fixed number of bits in its own bitstream; a
hierarchy lets a view touch only the primitives of what it sees).

The bit allocations are readings (16-bit positions over the chunk box, bfloat16 scales,
smallest-three quaternions with 10-bit components, 8-bit opacity logits over [-8, 8]). Pins: the
quantisers' error bounds and exact cases, sign invariance of the rotation code, chunk boxes that
hold their centres, and the culling rule never dropping a chunk that holds a Gaussian the
renderer would draw (checked against the splat setup over many cameras).
"""
import numpy as np
import pytest

from paper_2607_14513_gb300 import synthetic as S


def _scene(n=300, seed=3, scale=0.01):
    sc = S.make_scene(n, seed)
    geo = S.make_geometry(n, seed + 1, scale)
    ns = (n + 15) // 16 * 16
    perm = np.full(ns, -1, np.int32)
    perm[:n] = np.random.default_rng(seed).permutation(n)
    return sc, geo, perm


def test_position_codes_within_half_a_step_of_the_chunk_box(O):
    sc, geo, perm = _scene()
    g = O.geometry_encode(sc.pos, geo.scale, geo.rot, geo.logit, perm, 64)
    P, _, _, _ = O.geometry_decode(g)
    for s, o in enumerate(perm):
        if o < 0:
            assert np.all(g["qpos"][s] == 0)
            continue
        e = g["chunk"][s // 64]
        ext = e[3:6] - e[0:3]
        assert np.all(e[0:3] <= sc.pos[o]) and np.all(sc.pos[o] <= e[3:6])
        assert np.all(np.abs(P[s] - sc.pos[o]) <= 0.5 * ext / 65535 + 1e-6)
    # the box's extremes are codes 0 and 65535
    for c in range(g["chunk"].shape[0]):
        sl = slice(64 * c, 64 * c + 64)
        live = perm[sl] >= 0
        assert np.all(g["qpos"][sl][live].min(axis=0) == 0) and np.all(g["qpos"][sl][live].max(axis=0) == 65535)


def test_scale_and_opacity_codes(O):
    sc, geo, perm = _scene()
    geo.scale[:4] = [[0.5, 0.0234375, 1.0], [2.0 ** -10, 3.0, 0.75], [0.1, 0.1, 0.1], [1e-3, 2e-3, 3e-3]]
    geo.logit[:4] = [-20.0, 20.0, 0.0, -8.0]
    g = O.geometry_encode(sc.pos, geo.scale, geo.rot, geo.logit, perm, 64)
    _, Sc, _, T = O.geometry_decode(g)
    inv = np.argsort(perm[perm >= 0])            # slot of Gaussian o
    slot = np.nonzero(perm >= 0)[0][inv]
    # bfloat16, round to nearest even: within half a unit in the 8th significant bit, exact where representable
    assert np.all(np.abs(Sc[slot] / geo.scale - 1) <= 2.0 ** -8)
    assert np.array_equal(Sc[slot[0]], [0.5, 0.0234375, 1.0]) and np.array_equal(Sc[slot[1]], [2.0 ** -10, 3.0, 0.75])
    # opacity logit: 8 bits over [-8, 8], clamped
    want = np.clip(geo.logit, -8, 8)
    assert np.all(np.abs(T[slot] - want) <= 8.0 / 255 + 1e-6)
    assert g["qlogit"][slot[0]] == 0 and g["qlogit"][slot[1]] == 255 and T[slot[3]] == -8.0


def test_rotation_smallest_three(O):
    sc, geo, perm = _scene()
    geo.rot[:3] = [[0, 0, 3.0, 0], [0.5, -0.5, 0.5, -0.5], [-1.0, 0, 0, 0]]
    g = O.geometry_encode(sc.pos, geo.scale, geo.rot, geo.logit, perm, 64)
    _, _, Q, _ = O.geometry_decode(g)
    slot = np.nonzero(perm >= 0)[0][np.argsort(perm[perm >= 0])]
    qn = geo.rot / np.linalg.norm(geo.rot, axis=1, keepdims=True)
    dq = Q[slot]
    err = np.minimum(np.abs(dq - qn).max(axis=1), np.abs(dq + qn).max(axis=1))
    # three components within half a 10-bit step of [-1/sqrt2, 1/sqrt2]; the fourth follows from |q| = 1
    assert np.all(err <= 2e-3)
    assert np.array_equal(dq[0], [0, 0, 1, 0]) and np.array_equal(dq[2], [1, 0, 0, 0])
    assert g["qrot"][slot[0]] & 3 == 2                     # the largest component's index
    # q and -q are the same rotation and get the same code
    geo.rot[:] = -geo.rot
    g2 = O.geometry_encode(sc.pos, geo.scale, geo.rot, geo.logit, perm, 64)
    ties = np.abs(np.abs(qn).max(axis=1)[:, None] - np.abs(qn)).min(axis=1) == 0
    same = np.nonzero(perm >= 0)[0]
    assert np.array_equal(g2["qrot"][same], g["qrot"][same]) or ties.any()


def test_chunk_table_and_byte_count(O):
    sc, geo, perm = _scene(n=1000)
    geo.scale[perm[0]] = [0.001, 0.5, 0.002]          # the chunk's first Gaussian holds its largest scale
    g = O.geometry_encode(sc.pos, geo.scale, geo.rot, geo.logit, perm, 256)
    _, Sc, _, _ = O.geometry_decode(g)
    for c in range(g["chunk"].shape[0]):
        sl = slice(256 * c, 256 * c + 256)
        live = perm[sl] >= 0
        assert g["chunk"][c, 6] == Sc[sl][live].max()
    per_slot = (g["qpos"].itemsize * 3 + g["qscale"].itemsize * 3 + g["qrot"].itemsize + g["qlogit"].itemsize)
    assert per_slot == 17


def test_culling_never_drops_a_drawn_gaussian(O):
    # the chunk rule against the renderer's own per-Gaussian decision, for cameras inside, around
    # and looking past the scene
    n = 2000
    sc = S.make_scene(n, 11)
    geo = S.make_geometry(n, 12, 0.03)
    # the planned slot order: spatial (Morton) chunks of 128, so chunk boxes are compact
    perm = O.plan(sc.pos, O.quantise(sc.sh, O.scales(sc.sh)), 128, 1)
    g = O.geometry_encode(sc.pos, geo.scale, geo.rot, geo.logit, perm, 128)
    P, Sc, Q, _ = O.geometry_decode(g)
    rng = np.random.default_rng(13)
    culled_any = 0
    for k in range(40):
        eye = 0.5 + rng.normal(0, 1.2, size=3)
        tgt = 0.5 + rng.normal(0, 0.8, size=3)
        cam = S.look_at(eye, tgt, 96, 64, fov_x_deg=float(rng.uniform(30, 90)))
        for c in range(g["chunk"].shape[0]):
            vis = O.chunk_visible(g["chunk"][c], cam)
            culled_any += not vis
            if vis:
                continue
            for s in range(128 * c, min(128 * c + 128, perm.shape[0])):
                if perm[s] >= 0:
                    assert not O.splat_setup(P[s], Sc[s], Q[s], cam).visible, (k, c, s)
    assert culled_any > 0


def test_culling_keeps_adversarial_chunks(O):
    # the chunk rule against the renderer's own decision on chunks built to sit at its edges, for
    # cameras along every axis and an oblique one: tiny splats a few pixels outside a side (only
    # the pixel band protects them), large splats far outside a side (the box growth must reach
    # the view from the near side), and chunks straddling the camera plane. A chunk that holds a
    # Gaussian the renderer draws is never culled.
    rng = np.random.default_rng(17)
    centre = [0.5, 0.5, 0.5]
    drawn = 0
    for eye in ([0.5, 0.5, -1.5], [0.5, 0.5, 2.5], [-1.5, 0.5, 0.5], [2.5, 0.5, 0.5], [0.5, -1.5, 0.5],
                [2.0, -1.0, 1.8]):
        cam = S.look_at(eye, centre, 96, 64, fov_x_deg=60.0)
        R = np.asarray(cam["R"], np.float64).reshape(3, 3)
        t = np.asarray(cam["t"], np.float64)
        f, cx, cy, W, H = float(cam["fx"]), float(cam["cx"]), float(cam["cy"]), cam["width"], cam["height"]
        for trial in range(3000):
            kind, side, m = trial % 3, rng.integers(4), 4
            if kind < 2:
                if kind == 0:   # tiny splats, 0-5 px outside
                    scale = np.full((m, 3), np.exp(rng.uniform(np.log(1e-5), np.log(1e-3))))
                    off, jit = rng.uniform(0, 5), rng.uniform(0, 1e-3)
                else:           # large splats, 10-250 px outside
                    scale = np.exp(rng.uniform(np.log(0.02), np.log(1.0), size=(m, 3)))
                    off, jit = rng.uniform(10, 250), rng.uniform(0, 0.3)
                z = rng.uniform(0.3, 5.0)
                u = [-off, W + off, rng.uniform(0, W), rng.uniform(0, W)][side]
                v = [rng.uniform(0, H), rng.uniform(0, H), -off, H + off][side]
                camp = np.array([(u - cx) * z / f, (v - cy) * z / f, z])[None, :] + rng.normal(0, jit, size=(m, 3))
            else:               # straddling the camera plane
                scale = np.exp(rng.uniform(np.log(1e-3), np.log(0.3), size=(m, 3)))
                camp = (np.array([rng.uniform(-2, 2), rng.uniform(-1.5, 1.5), rng.uniform(-0.4, 0.6)])[None, :]
                        + rng.normal(0, rng.uniform(0.05, 0.6), size=(m, 3)))
            pos = ((camp - t[None, :]) @ R).astype(np.float32)          # world = R^T (camera - t)
            q = rng.normal(size=(m, 4)).astype(np.float32)
            sc = scale.astype(np.float32)
            if not any(O.splat_setup(pos[i], sc[i], q[i], cam).visible for i in range(m)):
                continue
            drawn += 1
            e = np.zeros(8, np.float32)
            e[0:3], e[3:6], e[6] = pos.min(axis=0), pos.max(axis=0), sc.max()
            assert O.chunk_visible(e, cam), (eye, trial)
    assert drawn > 5000


def test_culling_cases(O):
    e = np.array([0.4, 0.4, 0.4, 0.6, 0.6, 0.6, 0.01, 0], np.float32)
    cam = S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, 0.5], 64, 64)
    assert O.chunk_visible(e, cam)
    behind = S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, -3.0], 64, 64)
    assert not O.chunk_visible(e, behind)
    aside = e.copy()
    aside[[0, 3]] += 5.0                                 # far to one side of the view
    assert not O.chunk_visible(aside, cam)
