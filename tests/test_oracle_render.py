"""Pins of the oracle's splatting renderer (Sec. II: Eq. sigmoid, Eq. covar, Eq. opac, Eq. blend,
Eq. preblend with Eq. premult; Fig. GSRend).

The paper defines the primitive (opacity mu = sigmoid(t), covariance R(q) D(s) D(s)^T R(q)^T,
g(x) = exp(-(x - p)^T Sigma^-1 (x - p) / 2)) and the front-to-back blend; the screen-space form
(EWA projection with a 0.3 px^2 low-pass, 3-sigma tile rectangles of 16 x 16 pixels, pixel
centres at +0.5) is the reading. Pins: closed forms of a head-on isotropic splat and of two
overlapping splats, the transmittance product, Eq. preblend against Eq. blend with the
non-premultiplied colour, the symmetry of a rotated elongated splat, culling and truncation.
"""
import numpy as np
import pytest

from paper_2607_14513_gb300 import synthetic as S

W = H = 64


def _cam():
    # on the z axis, looking at (0.5, 0.5, 0.5) along +z: image x = -world x, image y = -world y
    return S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, 0.5], W, H, fov_x_deg=50.0)


def _sig(t):
    return 1.0 / (1.0 + np.exp(-np.float64(t)))


def test_head_on_isotropic_splat_closed_form(O):
    cam = _cam()
    f = float(cam["fx"])
    s, t, z = 0.05, 0.7, 2.0
    col = np.array([[0.3, -0.2, 0.9]])
    img, tr = O.render([[0.5, 0.5, 0.5]], [[s, s, s]], [[1, 0, 0, 0]], [t], col, cam)
    var = (f * s / z) ** 2 + 0.3                     # projected variance plus the low-pass
    ys, xs = np.mgrid[0:H, 0:W]
    g = np.exp(-((xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2) / (2 * var))
    r = np.ceil(3 * np.sqrt(var + np.sqrt(0.1)))    # 3 sigma of the larger axis (equal axes: floor of 0.1)
    inside = ((np.floor((W / 2 - r) / 16) * 16 <= xs) & (xs < (np.floor((W / 2 + r) / 16) + 1) * 16) &
              (np.floor((H / 2 - r) / 16) * 16 <= ys) & (ys < (np.floor((H / 2 + r) / 16) + 1) * 16))
    want = np.where(inside[..., None], g[..., None] * col[0], 0.0)
    assert np.allclose(img, want, rtol=1e-5, atol=1e-9)
    assert np.allclose(tr, np.where(inside, 1 - _sig(t) * g, 1.0), rtol=1e-6, atol=1e-12)
    assert not inside.all() and inside.any()        # the footprint is truncated to its tiles


def test_two_splats_blend_front_to_back(O):
    cam = _cam()
    s = 0.03
    c1, c2 = np.array([1.0, 0.0, 0.5]), np.array([0.0, 1.0, -0.5])
    t1, t2 = 1.2, -0.3
    pos = np.array([[0.5, 0.5, 0.3], [0.5, 0.5, 0.8]], np.float32)     # depth 1.8 (near) and 2.3 (far)
    img, tr = O.render(pos, [[s] * 3] * 2, [[1, 0, 0, 0]] * 2, [t1, t2], np.stack([c1, c2]), cam)
    f = float(cam["fx"])
    px = W // 2                                     # pixel (32, 32): centre offset 0.5 in x and y
    g = [np.exp(-0.25 / ((f * s / z) ** 2 + 0.3)) for z in (1.8, 2.3)]   # dx = dy = 0.5
    want = g[0] * c1 + (1 - _sig(t1) * g[0]) * g[1] * c2
    assert np.allclose(img[px, px], want, rtol=1e-5)
    assert np.isclose(tr[px, px], (1 - _sig(t1) * g[0]) * (1 - _sig(t2) * g[1]), rtol=1e-6)
    # the error bound the GPU parity tests use: the sum of the blend's absolute terms
    _, _, ab = O.render(pos, [[s] * 3] * 2, [[1, 0, 0, 0]] * 2, [t1, t2], np.stack([c1, c2]), cam, want_abs=True)
    assert np.allclose(ab[px, px], g[0] * np.abs(c1) + (1 - _sig(t1) * g[0]) * g[1] * np.abs(c2), rtol=1e-5)
    # swapping the two positions swaps the order: the far splat is now the first colour
    img2, _ = O.render(pos[::-1].copy(), [[s] * 3] * 2, [[1, 0, 0, 0]] * 2, [t1, t2], np.stack([c1, c2]), cam)
    want2 = g[0] * c2 + (1 - _sig(t2) * g[0]) * g[1] * c1
    assert np.allclose(img2[px, px], want2, rtol=1e-5)


def test_preblend_equals_blend_with_opacity_times_colour(O):
    # Eq. preblend with c~ = mu c (Eq. premult) equals Eq. blend: sum_i alpha_i c_i prod_{j<i} (1 - alpha_j)
    rng = np.random.default_rng(5)
    n = 60
    cam = _cam()
    pos = (0.5 + rng.normal(0, 0.08, size=(n, 3))).astype(np.float32)
    scale = np.exp(rng.normal(np.log(0.03), 0.3, size=(n, 3))).astype(np.float32)
    rot = rng.standard_normal(size=(n, 4)).astype(np.float32)
    logit = rng.normal(0, 1.5, size=n).astype(np.float32)
    c = rng.normal(0, 1, size=(n, 3))
    mu = _sig(logit)
    img, tr = O.render(pos, scale, rot, logit, mu[:, None] * c, cam)
    # Eq. blend, nearest first, with the oracle's footprint of each splat
    sp = [O.splat_setup(pos[i], scale[i], rot[i], cam) for i in range(n)]
    order = sorted([i for i in range(n) if sp[i].visible], key=lambda i: (np.float32(sp[i].depth), i))
    ys, xs = np.mgrid[0:H, 0:W]
    want = np.zeros((H, W, 3))
    T = np.ones((H, W))
    for i in order:
        a, b, cc = float(sp[i].a), float(sp[i].b), float(sp[i].c)
        Sinv = np.linalg.inv(np.array([[a, b], [b, cc]]))
        dx, dy = xs + 0.5 - sp[i].u, ys + 0.5 - sp[i].v
        g = np.exp(-0.5 * (Sinv[0, 0] * dx * dx + 2 * Sinv[0, 1] * dx * dy + Sinv[1, 1] * dy * dy))
        live = (xs // 16 >= sp[i].x0) & (xs // 16 < sp[i].x1) & (ys // 16 >= sp[i].y0) & (ys // 16 < sp[i].y1)
        alpha = np.where(live, mu[i] * g, 0.0)
        want += (alpha * T)[..., None] * c[i]
        T *= 1 - alpha
    assert np.allclose(img, want, rtol=1e-9, atol=1e-12)
    assert np.allclose(tr, T, rtol=1e-12)


def test_rotation_about_the_view_axis_transposes_an_elongated_splat(O):
    cam = _cam()
    s = np.array([[0.09, 0.02, 0.02]], np.float32)          # long along world x = image x
    q90 = [np.cos(np.pi / 4), 0, 0, np.sin(np.pi / 4)]        # 90 degrees about world z, the viewing axis
    col = np.array([[1.0, 1.0, 1.0]])
    a, _ = O.render([[0.5, 0.5, 0.5]], s, [[1, 0, 0, 0]], [2.0], col, cam)
    b, _ = O.render([[0.5, 0.5, 0.5]], s, [q90], [2.0], col, cam)
    assert a[32, :, 0].sum() > 2 * a[:, 32, 0].sum()        # wide in x before the rotation
    assert np.allclose(b[..., 0], a[..., 0].T, rtol=1e-4, atol=1e-7)


def test_oblique_splat_points_along_its_axis(O):
    # a Gaussian long along a world direction u in the image plane's parallel plane, on the optical
    # axis: the rendered image's principal axis (second moments) is the camera's image of u, and its
    # variances are (f s / z)^2 + 0.3 along both axes; at oblique angles a wrong sign anywhere in the
    # rotation or the projected covariance mirrors the axis
    cam = _cam()
    f, z = float(cam["fx"]), 2.0
    Rm = np.asarray(cam["R"], np.float64).reshape(3, 3)
    sc = np.array([[0.09, 0.02, 0.02]], np.float32)
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    for deg in (20, 35, 60, 110, 145):
        th = np.radians(deg)
        q = [np.cos(th / 2), 0.0, 0.0, np.sin(th / 2)]          # th about world z
        u = np.array([np.cos(th), np.sin(th), 0.0])              # where the long axis (world x) goes
        img, _ = O.render([[0.5, 0.5, 0.5]], sc, [q], [2.0], np.array([[1.0, 1.0, 1.0]]), cam)
        w = img[..., 0]
        m = w.sum()
        cx, cy = (w * xs).sum() / m, (w * ys).sum() / m
        mxx, myy = (w * (xs - cx) ** 2).sum() / m, (w * (ys - cy) ** 2).sum() / m
        mxy = (w * (xs - cx) * (ys - cy)).sum() / m
        phi = 0.5 * np.arctan2(2 * mxy, mxx - myy)
        want = np.arctan2(Rm[1] @ u, Rm[0] @ u)
        assert abs((phi - want + np.pi / 2) % np.pi - np.pi / 2) < np.radians(0.05), deg
        ev = np.linalg.eigvalsh([[mxx, mxy], [mxy, myy]])
        var = (f * sc[0, [2, 0]].astype(np.float64) / z) ** 2 + 0.3
        assert np.allclose(ev, var, rtol=1e-2), deg


def test_tile_rectangle_is_three_sigma(O):
    # the footprint is every 16 x 16 tile that the square of half-width ceil(3 sigma) around the
    # centre touches (sigma of the larger axis, isotropic here: variance (f s / z)^2 + 0.3 plus the
    # eigenvalue floor sqrt(0.1)); a head-on splat moved across a tile, inside pixels positive,
    # outside exactly zero
    cam = _cam()
    f, z = float(cam["fx"]), 2.0
    s = 0.05
    var = (f * s / z) ** 2 + 0.3
    r = np.ceil(3 * np.sqrt(var + np.sqrt(0.1)))
    for du in (-11.0, -7.5, -3.0, 0.0, 2.5, 6.5, 9.25):
        x = 0.5 - du * z / f                            # image x = -world x
        img, _ = O.render([[x, 0.5, 0.5]], [[s, s, s]], [[1, 0, 0, 0]], [2.0], np.array([[1.0, 1.0, 1.0]]), cam)
        u = W / 2 + du
        t0, t1 = np.floor((u - r) / 16), np.floor((u + r) / 16) + 1
        v0, v1 = np.floor((H / 2 - r) / 16), np.floor((H / 2 + r) / 16) + 1
        ys, xs = np.mgrid[0:H, 0:W]
        inside = (xs >= 16 * t0) & (xs < 16 * t1) & (ys >= 16 * v0) & (ys < 16 * v1)
        assert np.array_equal(img[..., 0] > 0, inside), du


def test_culling_and_empty_footprints(O):
    cam = _cam()
    col = np.ones((3, 3))
    # behind the camera, in front of it but nearer than the near plane (depth 0.1 < 0.2), far
    # outside the image
    pos = [[0.5, 0.5, -2.0], [0.5, 0.5, -1.4], [9.0, 0.5, 0.5]]
    img, tr = O.render(pos, [[0.05] * 3] * 3, [[1, 0, 0, 0]] * 3, [3.0] * 3, col, cam)
    assert np.all(img == 0) and np.all(tr == 1)
    assert O.splat_setup([0.5, 0.5, -1.2], [0.05] * 3, [1, 0, 0, 0], cam).visible      # depth 0.3


def test_equal_depths_keep_index_order(O):
    cam = _cam()
    pos = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5]], np.float32)
    c = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    img, _ = O.render(pos, [[0.05] * 3] * 2, [[1, 0, 0, 0]] * 2, [1.0, 1.0], c, cam)
    g = img[32, 32, 0]                               # the first splat in full
    assert img[32, 32, 1] < g and np.isclose(img[32, 32, 1], (1 - _sig(1.0) * g) * g, rtol=1e-9)


def test_sampled_tiles_equal_the_full_render(O):
    rng = np.random.default_rng(8)
    n = 300
    cam = _cam()
    pos = (0.5 + rng.normal(0, 0.1, size=(n, 3))).astype(np.float32)
    geo = S.make_geometry(n, 9, scale=0.02)
    col = rng.normal(0, 1, size=(n, 3))
    full, tr = O.render(pos, geo.scale, geo.rot, geo.logit, col, cam)
    tiles = np.array([0, 5, 6, 10, 15], np.int32)
    part, trp = O.render(pos, geo.scale, geo.rot, geo.logit, col, cam, tiles=tiles)
    for t in tiles:
        ty, tx = divmod(int(t), 4)
        sl = (slice(16 * ty, 16 * ty + 16), slice(16 * tx, 16 * tx + 16))
        assert np.array_equal(part[sl], full[sl]) and np.array_equal(trp[sl], tr[sl])
