"""Pins of the scale-map estimator oracle (structure tensor -> ellipse): checks
that do not reuse its formulas."""
import numpy as np
import pytest

from oracle import structure as st


def test_gaussian_taps_normalised_and_symmetric():
    for rho in (0.7, 2.0, 3.3):
        w, r = st.gaussian_taps(rho)
        assert len(w) == 2 * r + 1 and r >= 3 * rho
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.allclose(w, w[::-1], rtol=0, atol=0)


def test_smoothing_equals_direct_2d_convolution():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((9, 13))
    rho = 1.1
    w, r = st.gaussian_taps(rho)
    H, W = a.shape
    ref = np.zeros_like(a)
    for y in range(H):
        for x in range(W):
            acc = 0.0
            for dy in range(-r, r + 1):
                for dx in range(-r, r + 1):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < H and 0 <= xx < W:
                        acc += w[dy + r] * w[dx + r] * a[yy, xx]
            ref[y, x] = acc
    assert np.allclose(st.smooth(a, rho), ref, rtol=1e-13, atol=1e-13)


def test_constant_image_is_isotropic_inside():
    f = np.full((40, 50), 7.25)
    out = st.ellipse_field(f, rho=2.0, sigma0=3.0, e_max=5.0)
    inner = out[9:-9, 9:-9]
    assert np.all(inner[..., 0] == 3.0)
    assert np.all(inner[..., 1] == 1.0)
    assert np.all(inner[..., 2] == 1.0) and np.all(inner[..., 3] == 0.0)


@pytest.mark.parametrize("a,b", [(1.5, 0.0), (0.0, -2.0), (0.8, 0.6), (-1.0, 3.0)])
def test_linear_ramp_gives_coherent_axis_along_the_level_lines(a, b):
    yy, xx = np.mgrid[0:48, 0:48].astype(np.float64)
    f = a * xx + b * yy
    out = st.ellipse_field(f, rho=1.5, sigma0=4.0, e_max=6.0)
    inner = out[10:-10, 10:-10]
    assert np.allclose(inner[..., 1], 6.0, rtol=0, atol=1e-9)
    t = np.array([-b, a]) / np.hypot(a, b)
    if t[1] < 0 or (t[1] == 0 and t[0] < 0):
        t = -t
    assert np.allclose(inner[..., 2], t[0], atol=1e-9)
    assert np.allclose(inner[..., 3], t[1], atol=1e-9)


def test_axis_is_the_small_eigenvector_and_rotation_equivariant():
    rng = np.random.default_rng(11)
    f = rng.uniform(0, 255, (30, 30))
    out = st.ellipse_field(f, rho=1.3)
    gx, gy = st.gradient(f)
    j11, j12, j22 = (st.smooth(p, 1.3) for p in (gx * gx, gx * gy, gy * gy))
    v = out[..., 2:4]
    assert np.allclose(np.hypot(v[..., 0], v[..., 1]), 1.0, atol=1e-12)
    jv = np.stack([j11 * v[..., 0] + j12 * v[..., 1], j12 * v[..., 0] + j22 * v[..., 1]], axis=-1)
    lam = (jv * v).sum(-1, keepdims=True)
    assert np.allclose(jv, lam * v, atol=1e-8 * float(np.abs(j11).max()))
    tr = j11 + j22
    l2 = 0.5 * (tr - np.sqrt((j11 - j22) ** 2 + 4 * j12 * j12))
    assert np.allclose(lam[..., 0], l2, atol=1e-8 * float(np.abs(tr).max()))
    # rotating the image by 90 degrees rotates every axis by 90 degrees
    fr = np.rot90(f)  # new[y, x] = f[x, W-1-y]
    outr = st.ellipse_field(fr, rho=1.3)
    H, W = f.shape
    for y in range(H):
        for x in range(W):
            a = out[y, x]
            b = outr[W - 1 - x, y]
            assert abs(a[1] - b[1]) < 1e-9
            # (vx, vy) at (y, x) maps to (vy, -vx), up to the sign convention
            assert abs(a[3] * b[2] - a[2] * b[3]) > 1 - 1e-9 or a[1] < 1 + 1e-9
