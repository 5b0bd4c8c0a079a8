"""Pins of oracle.general (N = 2 and the B-spline model phi) against what the
paper and the mathematics fix, independently of the oracle's own algorithm."""
from fractions import Fraction as Fr
import random

import numpy as np
import pytest

from oracle import general, line1d, paper


def test_n2_kernel_is_the_tensor_box_spline():
    """N = 2 (directions c1 v1, c3 v3, each n times): the box spline is the
    product of two 1-D B-splines of degree n - 1 and widths c1, c3 -- Sec. 4:
    rect = beta^2_(1,1) at n = 1; beta_a^{n-1}(x) = beta^{n-1}(x / a) / a."""
    rnd = random.Random(3)
    for n in (2, 3):
        c = (Fr(5, 2), Fr(0), Fr(7, 4), Fr(0))
        B = general.kernel_direct(c, (n, 0, n, 0), None)
        for _ in range(25):
            x, y = Fr(rnd.randint(-80, 80), 16), Fr(rnd.randint(-80, 80), 16)
            want = line1d.bspline_scaled(n - 1, Fr(5, 2), x) * line1d.bspline_scaled(n - 1, Fr(7, 4), y)
            assert B.centred_value(x, y) == want


def test_model_kernel_partition_of_unity():
    """With a model of any degree the kernel holds unit boxes along v1 and v3,
    so its lattice translates sum to 1 at every point (also through the
    parallel pair c1 v1, v1 of the recurrence)."""
    rnd = random.Random(4)
    for r, n1 in (((1, 1, 1, 1), 1), ((2, 0, 2, 0), 0), ((1, 1, 1, 1), 3)):
        c = (Fr(3, 2), Fr(5, 4), Fr(2), Fr(1))
        B = general.kernel_direct(c, r, n1)
        for _ in range(3):
            x, y = Fr(rnd.randint(0, 15), 16), Fr(rnd.randint(0, 15), 16)
            tot = sum(B.centred_value(x - i, y - j) for i in range(-9, 10) for j in range(-9, 10))
            assert tot == 1


def test_model_kernel_integer_steps_is_box_times_bspline():
    """N = 2, unit steps c1 = c3 = 1, order n, model degree n1: the kernel is
    beta^{n-1} * beta^{n1} per axis = beta^{n+n1} (B-splines convolve by
    adding degrees), a tensor product."""
    rnd = random.Random(5)
    for n, n1 in ((2, 1), (2, 3)):
        B = general.kernel_direct((1, 0, 1, 0), (n, 0, n, 0), n1)
        for _ in range(10):
            x, y = Fr(rnd.randint(-60, 60), 16), Fr(rnd.randint(-60, 60), 16)
            assert B.centred_value(x, y) == line1d.bspline(n + n1, x) * line1d.bspline(n + n1, y)


def test_general_method_reduces_to_the_four_direction_oracle():
    """r = (n, n, n, n), phi = delta: the generalised method (its own grid, its
    own kernel tables) gives exactly the s of oracle.paper."""
    rng = np.random.default_rng(61)
    H, W, Q = 6, 7, 2
    f = rng.integers(0, 256, (H, W))
    C = rng.integers(2, 10, (H, W, 4))
    for n in (1, 2):
        S, s = paper.filter_image(f, C, n, Q)
        mesh = paper.Mesh(n, Q)
        pix = [(x, y) for y in range(H) for x in range(W)]
        _, sg = general.filter_pixels(f, (0, 0), C, (n, n, n, n), None, Q, 0, pix)
        for (x, y), v in zip(pix, sg):
            assert v == Fr(S[y, x]) / mesh.denominator(C[y, x], 0)


@pytest.mark.parametrize("r,n1", [((2, 0, 2, 0), None), ((3, 0, 3, 0), None), ((1, 1, 1, 1), 1),
                                  ((2, 0, 2, 0), 1)])
def test_general_method_equals_definition(r, n1):
    """Algorithm (running sums on c, the mesh with interpolation kernel
    phi * beta^N_b, Eq. (NA) and Eq. (mask)) == definition (Sec. 6, s[m] =
    sum_k c[k] (phi * beta_a)(m - k)), exactly, at every pixel of a tiny
    image including its borders; coefficients given on a grid that extends
    beyond the image (as a prefiltered model's do)."""
    rng = np.random.default_rng(62)
    H, W, Q = 5, 6, 1
    cq = rng.integers(-300, 300, (H + 2, W + 2))
    C = rng.integers(2, 7, (H, W, 4))
    pix = [(x, y) for y in range(H) for x in range(W)]
    _, sa = general.filter_pixels(cq, (1, 1), C, r, n1, Q, 0, pix)
    sd = general.filter_direct(cq, (1, 1), C, r, n1, Q, 0, pix)
    assert sa == sd


def test_model_partition_of_unity_constant_coefficients():
    """Constant coefficients (over a region wider than every kernel) give s =
    that constant exactly: the model's kernel reproduces constants."""
    H, W, Q = 4, 5, 2
    cq = np.full((H + 24, W + 24), 77, dtype=object)
    rng = np.random.default_rng(63)
    C = rng.integers(4, 12, (H, W, 4))
    pix = [(x, y) for y in range(H) for x in range(W)]
    for r, n1 in (((1, 1, 1, 1), 1), ((2, 0, 2, 0), 3)):
        _, s = general.filter_pixels(cq, (12, 12), C, r, n1, Q, 0, pix)
        assert all(v == 77 for v in s)


@pytest.mark.parametrize("n1", [2, 3])
def test_prefilter2d_interpolates_the_samples(n1):
    """The model f(x) = sum_k c_q[k] 2^-F phi(x - k) passes within half a grid
    step of every sample (phi >= 0 with unit lattice sum, |c_q - c 2^F| <= 1/2),
    and c_q vanishes beyond the kept tail."""
    rng = np.random.default_rng(64 + n1)
    H, W = 5, 6
    f = rng.integers(0, 255 << 4, (H, W))
    cq, (ox, oy) = general.prefilter2d(f, n1, bits=120)
    for y in range(H):
        for x in range(W):
            acc = Fr(0)
            for i in range(cq.shape[0]):
                wy = line1d.bspline(n1, (y + oy) - i)
                if wy == 0:
                    continue
                for j in range(cq.shape[1]):
                    wx = line1d.bspline(n1, (x + ox) - j)
                    if wx:
                        acc += int(cq[i, j]) * wx * wy
            assert abs(acc - int(f[y, x])) <= Fr(1, 2)


def test_prefilter2d_planted_causal_only_inverse_is_caught():
    """A prefilter that drops the anti-causal half (a plausible slip) misses
    the interpolation condition by far more than half a step."""
    rng = np.random.default_rng(66)
    f = rng.integers(0, 255 << 4, (4, 5))
    h = line1d.inverse_filter(3)
    causal = {k: v for k, v in h.items() if k >= 0}

    def conv1(xs):
        return {k: sum(causal.get(k - i, 0) * x for i, x in enumerate(xs)) for k in range(len(xs))}
    rows = [conv1([int(v) for v in f[y]]) for y in range(4)]
    worst = 0
    for y in range(4):
        for x in range(5):
            acc = sum(rows[y][j] * line1d.bspline(3, x - j) for j in range(5))
            worst = max(worst, abs(acc - int(f[y, x])))
    assert worst > 1


def test_whole_image_evaluation_equals_per_pixel_windows():
    """filter_image (one lattice box) == filter_pixels (a window per pixel)."""
    rng = np.random.default_rng(67)
    cq = rng.integers(-500, 500, (9, 11))
    C = rng.integers(2, 9, (7, 9, 4))
    pix = [(x, y) for y in range(7) for x in range(9)]
    for r, n1 in (((1, 1, 1, 1), 3), ((2, 0, 2, 0), None)):
        S1, s1 = general.filter_image(cq, (1, 1), C, r, n1, 2, 3)
        S2, s2 = general.filter_pixels(cq, (1, 1), C, r, n1, 2, 3, pix)
        assert S1 == S2 and s1 == s2
