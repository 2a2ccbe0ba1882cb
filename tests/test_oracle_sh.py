"""Pins of the oracle's SH evaluation (Sec. II: c(f) = H w(f - p), w the vector of SH
factors) and of its dequantisation (Sec. V-A, inverse of the 8-bit mapping).

The paper leaves the basis convention silent. Reading: orthonormal real SH to degree 3,
k = l*l + l + m, Condon-Shortley phase inside the associated Legendre function (the
convention of 3DGS checkpoints). Pins: quadrature orthonormality, scipy's complex SH,
closed-form values at the poles, the addition theorem, and degree 0.
"""
import numpy as np
import pytest


def _dirs(n, seed):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_orthonormal_by_quadrature(O):
    # Gauss-Legendre in cos(theta) x uniform phi integrates products of degree <= 6 exactly
    x, w = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * (2 * np.pi / 32)
    G = np.zeros((16, 16))
    for z, wz in zip(x, w):
        r = np.sqrt(1 - z * z)
        for ph in phis:
            Y = O.sh_basis(r * np.cos(ph), r * np.sin(ph), z)
            G += wz * (2 * np.pi / 32) * np.outer(Y, Y)
    assert np.max(np.abs(G - np.eye(16))) < 1e-10


def test_matches_scipy_complex_sh(O):
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    for d in _dirs(40, 1):
        theta = np.arccos(np.clip(d[2], -1, 1))
        phi = np.arctan2(d[1], d[0])
        Y = O.sh_basis(*d)
        for l in range(4):
            for m in range(-l, l + 1):
                c = sp.sph_harm_y(l, abs(m), theta, phi)     # includes the Condon-Shortley phase
                ref = c.real if m == 0 else (np.sqrt(2) * c.real if m > 0 else np.sqrt(2) * c.imag)
                assert abs(Y[l * l + l + m] - ref) < 1e-12


def test_closed_form_values(O):
    Y = O.sh_basis(0.0, 0.0, 1.0)                       # +z: only m = 0 survives, P_l(1) = 1
    expect = np.zeros(16)
    for l in range(4):
        expect[l * l + l] = np.sqrt((2 * l + 1) / (4 * np.pi))
    assert np.max(np.abs(Y - expect)) < 1e-14
    Y = O.sh_basis(1.0, 0.0, 0.0)                       # +x
    assert abs(Y[0] - 0.5 / np.sqrt(np.pi)) < 1e-15
    assert abs(Y[3] + np.sqrt(3 / (4 * np.pi))) < 1e-14  # l=1, m=1 carries the phase: -sqrt(3/4pi) x
    assert abs(Y[1]) < 1e-15 and abs(Y[2]) < 1e-15
    Y = O.sh_basis(0.0, 1.0, 0.0)                       # +y
    assert abs(Y[1] + np.sqrt(3 / (4 * np.pi))) < 1e-14
    Y = O.sh_basis(0.0, 0.0, -1.0)                      # -z: odd bands flip
    for l in range(4):
        assert abs(Y[l * l + l] - (-1) ** l * np.sqrt((2 * l + 1) / (4 * np.pi))) < 1e-14


def test_addition_theorem(O):
    for d in _dirs(50, 2):
        Y = O.sh_basis(*d)
        for l in range(4):
            assert abs(np.sum(Y[l * l:(l + 1) * (l + 1)] ** 2) - (2 * l + 1) / (4 * np.pi)) < 1e-13


def test_degree_zero_and_dequantisation(O):
    rng = np.random.default_rng(3)
    n = 64
    tex = np.full((n, 16, 3), 128, np.uint8)
    tex[:, 0, :] = rng.integers(0, 256, size=(n, 3))
    sc = rng.uniform(0.1, 2.0, size=16).astype(np.float32)
    dirs = _dirs(5, 4).astype(np.float32)
    out = O.eval_sh(tex, sc, dirs=dirs)
    x0 = (tex[:, 0, :].astype(np.float64) - 128.0) / 255.0 * np.float64(sc[0])
    for v in range(5):
        assert np.max(np.abs(out[v] - x0 / (2 * np.sqrt(np.pi)))) < 1e-15


def test_tolerance_sum_is_the_sum_of_absolute_terms(O):
    # the bound the GPU parity tests scale their tolerance by: sum_k |x'_k Y_k(d)| per channel
    rng = np.random.default_rng(6)
    n = 30
    tex = rng.integers(0, 256, size=(n, 16, 3)).astype(np.uint8)
    sc = rng.uniform(0.1, 2.0, size=16).astype(np.float32)
    dirs = _dirs(4, 9).astype(np.float32)
    out, ab = O.eval_sh(tex, sc, dirs=dirs, want_abs=True)
    x = (tex.astype(np.float64) - 128.0) / 255.0 * sc.astype(np.float64)[None, :, None]
    for v in range(4):
        d = dirs[v].astype(np.float64)
        Y = O.sh_basis(*(d / np.linalg.norm(d)))
        want = np.abs(x * Y[None, :, None]).sum(axis=1)
        assert np.allclose(ab[v], want, rtol=1e-12, atol=0)
        assert np.all(ab[v] >= np.abs(out[v]) - 1e-15)


def test_camera_directions(O):
    rng = np.random.default_rng(5)
    n = 20
    tex = rng.integers(0, 256, size=(n, 16, 3)).astype(np.uint8)
    sc = rng.uniform(0.1, 2.0, size=16).astype(np.float32)
    pos = rng.uniform(0, 1, size=(n, 3)).astype(np.float32)
    cams = np.array([[2.0, 0.5, 0.5], [0.5, -1.0, 0.5]], np.float32)
    out = O.eval_sh(tex, sc, pos=pos, cams=cams)
    x = (tex.astype(np.float64) - 128.0) / 255.0 * sc.astype(np.float64)[None, :, None]
    for v in range(2):
        d = cams[v].astype(np.float64)[None, :] - pos.astype(np.float64)       # f - p
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        for i in range(n):
            Y = O.sh_basis(*d[i])
            assert np.allclose(out[v, i], Y @ x[i], rtol=0, atol=1e-14)
    # the camera on the Gaussian: zero vector -> +z
    pos[0] = cams[0]
    out = O.eval_sh(tex, sc, pos=pos, cams=cams[:1])
    assert np.allclose(out[0, 0], O.sh_basis(0, 0, 1) @ x[0], atol=1e-14)
