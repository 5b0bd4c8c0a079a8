"""Pins of the 1-D oracle (Sec. 3, Proposition "prop") against what the paper
and the mathematics fix, independently of the oracle's own formulas."""
from fractions import Fraction as Fr
from math import comb

import numpy as np
import pytest

from oracle import line1d as o


# ------------------------------------------------------------------ B-splines

def test_bspline_known_values():
    # Sec. 2: beta^0 = rect on (-1/2, 1/2]; textbook values of the linear,
    # quadratic and cubic B-splines at integers and half-integers
    assert [o.bspline(0, x) for x in (Fr(-1, 2), 0, Fr(1, 2), Fr(3, 4))] == [0, 1, 1, 0]
    assert [o.bspline(1, x) for x in (0, Fr(1, 2), 1)] == [1, Fr(1, 2), 0]
    assert [o.bspline(2, x) for x in (0, Fr(1, 2), 1, Fr(3, 2))] == [Fr(3, 4), Fr(1, 2), Fr(1, 8), 0]
    assert [o.bspline(3, x) for x in (0, 1, 2)] == [Fr(2, 3), Fr(1, 6), 0]


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5])
def test_bspline_partition_of_unity_and_symmetry(n):
    for x in (Fr(0), Fr(1, 3), Fr(7, 16), Fr(-5, 9)):
        assert sum(o.bspline(n, x - k) for k in range(-6, 7)) == 1
        if n > 0:
            assert o.bspline(n, x) == o.bspline(n, -x)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_bspline_is_repeated_box_convolution(n):
    # beta^n = beta^{n-1} * beta^0: beta^n(x) = integral of beta^{n-1} over
    # [x - 1/2, x + 1/2], integrated exactly on the integer / half-integer pieces
    for x in (Fr(0), Fr(1, 5), Fr(3, 4), Fr(-7, 6)):
        lo, hi = x - Fr(1, 2), x + Fr(1, 2)
        knots = sorted(set([lo, hi] + [Fr(2 * i - n, 2) for i in range(n + 1) if lo < Fr(2 * i - n, 2) < hi]))
        total = Fr(0)
        for u0, u1 in zip(knots[:-1], knots[1:]):
            p = o._bspline_piece(n - 1, 1, 0, u0, u1)
            total += sum(c * (u1 ** (k + 1) - u0 ** (k + 1)) / (k + 1) for k, c in enumerate(p))
        assert total == o.bspline(n, x)


# ---------------------------------------------------------------- the kernel

@pytest.mark.parametrize("n1,n2", [(0, 0), (0, 2), (1, 1), (1, 3)])
def test_kernel_at_unit_scale_is_a_bspline(n1, n2):
    # beta^{n1} * beta^{n2} = beta^{n1+n2+1}
    for t in (Fr(0), Fr(1, 4), Fr(3, 2), Fr(-9, 8)):
        assert o.kernel(n1, n2, 1, t) == o.bspline(n1 + n2 + 1, t)


def test_kernel_box_against_box_is_overlap_length():
    # n1 = n2 = 0: K(t) = |[-1/2, 1/2] intersected with [t - a/2, t + a/2]| / a
    for a in (Fr(1), Fr(5, 2), Fr(13, 8)):
        for t in (Fr(0), Fr(3, 4), Fr(-6, 5), Fr(2)):
            lo, hi = max(Fr(-1, 2), t - a / 2), min(Fr(1, 2), t + a / 2)
            assert o.kernel(0, 0, a, t) == max(hi - lo, 0) / a


@pytest.mark.parametrize("n1,n2,a", [(0, 1, Fr(7, 4)), (1, 2, Fr(19, 8)), (1, 3, Fr(3))])
def test_kernel_shifts_sum_to_one(n1, n2, a):
    # sum_k K(t - k) = integral of beta_a^{n2} = 1 (integer shifts of beta^{n1}
    # form a partition of unity), and K is even
    for t in (Fr(0), Fr(2, 7)):
        assert sum(o.kernel(n1, n2, a, t - k) for k in range(-12, 13)) == 1
    assert o.kernel(n1, n2, a, Fr(5, 6)) == o.kernel(n1, n2, a, Fr(-5, 6))


# ---------------------------------------------------- algorithm == definition

@pytest.mark.parametrize("n1,n2,q", [(0, 0, 3), (0, 2, 2), (1, 1, 3), (1, 3, 2), (1, 2, 4)])
def test_proposition_equals_definition_exactly(n1, n2, q):
    rng = np.random.default_rng(100 + 10 * n1 + n2)
    f = rng.integers(-50, 200, 23)
    a = rng.uniform(1.0, 5.0, 23)
    A = o.quantise(a, q)
    _, s = o.filter_paper(list(f), A, n1, n2, q)
    ref = o.filter_direct(list(f), A, n2, q, n1)
    assert s == ref


def test_proposition_with_fraction_bits():
    rng = np.random.default_rng(7)
    F = 6
    fi = rng.integers(-3000, 3000, 17)
    A = o.quantise(rng.uniform(1.0, 3.0, 17), 3)
    _, s = o.filter_paper(list(fi), A, 1, 2, 3, frac_bits=F)
    ref = o.filter_direct([Fr(int(v), 1 << F) for v in fi], A, 2, 3, 1)
    assert s == ref


def test_integer_odd_scale_box_is_moving_average():
    # n1 = n2 = 0, a odd integer: s[m] = mean of f[m - (a-1)/2 .. m + (a-1)/2]
    f = [3, 9, -4, 7, 0, 12, 5, 5, 1, -8, 2]
    for a in (1, 3, 5):
        A = o.quantise([float(a)] * len(f), 2)
        _, s = o.filter_paper(f, A, 0, 0, 2)
        h = (a - 1) // 2
        for m in range(len(f)):
            win = [f[k] for k in range(m - h, m + h + 1) if 0 <= k < len(f)]
            assert s[m] == Fr(sum(win), a)


def test_constant_signal_is_reproduced_inside():
    f = [11] * 40
    A = o.quantise(np.full(40, 2.625), 3)
    _, s = o.filter_paper(f, A, 1, 3, 3)
    reach = 1 + 2.625 * 2
    for m in range(40):
        if reach < m < 39 - reach:
            assert s[m] == 11


def test_planted_error_in_fd_weights_is_caught():
    # the same steps with unsigned FD weights (a plausible slip) no longer
    # match the definition pin
    rng = np.random.default_rng(3)
    f = list(rng.integers(0, 100, 12))
    A = o.quantise(rng.uniform(1.0, 3.0, 12), 2)
    _, s = o.filter_paper(f, A, 1, 1, 2)
    ref = o.filter_direct(f, A, 1, 2, 1)
    assert s == ref
    N, P = 3, 3
    D = o.denominator(N, P)
    g = o.running_sums(f, 2, len(f) + o.box_right(1, 1, 2, int(max(A))))
    m, Am = 5, int(A[5])
    tauP = (Am - 4) * 2
    wrong = 0
    for j in range(3):
        Y = (m << P) + tauP - 2 * Am * j
        F = sum(g[k] * o.dbspline_int(N, P, Y - (k << P)) for k in range(max(0, (Y >> P) - 3), (Y >> P) + 4))
        wrong += comb(2, j) * F
    assert Fr(wrong * (1 << 4), D * Am ** 2) != ref[5]


# ------------------------------------ the interpolation prefilter (n1 >= 2)

def _dec(fr):
    from decimal import Decimal
    return Decimal(fr.numerator) / Decimal(fr.denominator)


def test_inverse_filter_matches_the_closed_forms():
    # quadratic and cubic B-spline interpolation: the inverse of
    # (z + 6 + 1/z)/8 is sqrt(2) (2 sqrt(2) - 3)^|k|, the inverse of
    # (z + 4 + 1/z)/6 is sqrt(3) (sqrt(3) - 2)^|k| (one pole each, from the
    # partial fractions of the symbol)
    from decimal import Decimal, getcontext
    getcontext().prec = 80
    r2, r3 = Decimal(2).sqrt(), Decimal(3).sqrt()
    h2, h3 = o.inverse_filter(2), o.inverse_filter(3)
    tol = Decimal(10) ** -50
    for k in range(-30, 31):
        assert abs(_dec(h2[k]) - r2 * (2 * r2 - 3) ** abs(k)) < tol
        assert abs(_dec(h3[k]) - r3 * (r3 - 2) ** abs(k)) < tol


# Poles of the B-spline interpolation filters as published (Unser, "Splines:
# a perfect fit for signal and image processing", IEEE SPM 1999, Table 1).
_POLES = {
    2: [-0.171572875253809902],
    3: [-0.267949192431122706],
    4: [-0.361341225900220177, -0.0137254292973391195],
    5: [-0.430575347099973792, -0.0430962882032647440],
}


@pytest.mark.parametrize("n1", [2, 3, 4, 5])
def test_inverse_filter_decays_with_the_published_poles(n1):
    # for k >= 1 the inverse is a sum of z_p^k: it satisfies the recurrence
    # whose characteristic roots are the poles, h[k+2] = (z1 + z2) h[k+1] - z1 z2 h[k]
    # (one pole: h[k+1] = z1 h[k]); checked relative to |h[k]|
    h = o.inverse_filter(n1)
    z = _POLES[n1]
    for k in range(1, 12):
        if len(z) == 1:
            pred = z[0] * float(h[k])
            got = float(h[k + 1])
        else:
            pred = (z[0] + z[1]) * float(h[k + 1]) - z[0] * z[1] * float(h[k])
            got = float(h[k + 2])
        assert abs(got - pred) <= 1e-14 * abs(float(h[k])), (k, got, pred)
        assert h[k] == h[-k]


@pytest.mark.parametrize("n1", [2, 3, 4, 5])
def test_prefilter_interpolates_the_samples(n1):
    # the model f(x) = sum_j c[j] beta^{n1}(x - j) passes through f[k] at every
    # integer (inside the window the oracle keeps, and zero outside the signal)
    rng = np.random.default_rng(40 + n1)
    F = 6
    x = [int(v) for v in rng.integers(-300 << F, 300 << F, 25)]
    kf, cs = o.prefilter(x, n1)
    c = {kf + i: Fr(v, 1 << (200 + F)) for i, v in enumerate(cs)}
    b = {k: o.bspline(n1, k) for k in range(-3, 4)}
    for k in range(-40, 65):
        val = sum(c.get(k - d, 0) * w for d, w in b.items())
        want = Fr(x[k], 1 << F) if 0 <= k < len(x) else 0
        assert abs(val - want) < Fr(1, 1 << 150), k


def test_prefilter_commutes_with_reversal_and_is_linear():
    rng = np.random.default_rng(8)
    x = [int(v) for v in rng.integers(-1000, 1000, 19)]
    y = [int(v) for v in rng.integers(-1000, 1000, 19)]
    kf, cx = o.prefilter(x, 3)
    _, cr = o.prefilter(x[::-1], 3)
    assert cr == cx[::-1]
    _, cy = o.prefilter(y, 3)
    _, cxy = o.prefilter([a + b for a, b in zip(x, y)], 3)
    assert all(abs(a + b - s) <= 2 for a, b, s in zip(cx, cy, cxy))


@pytest.mark.parametrize("n1,n2", [(2, 0), (2, 2), (3, 1), (4, 1), (5, 0)])
def test_quantised_model_moves_s_by_at_most_half_a_grid_step(n1, n2):
    # the Proposition on c_q = rint(c 2^F) against the definition on the exact c:
    # |s_q - s| <= 2^-(F+1) sum_k K(m - k) = 2^-(F+1) (K >= 0, unit lattice sum)
    rng = np.random.default_rng(70 + 10 * n1 + n2)
    q, F = 3, 5
    x = [int(v) for v in rng.integers(-60 << F, 60 << F, 24)]
    A = o.quantise(rng.uniform(0.5, 4.0, 24), q)
    kf, cs = o.prefilter(x, n1)
    s = o.filter_direct([Fr(v, 1 << (200 + F)) for v in cs], A, n2, q, n1, k_first=kf)
    kq, cq = o.prefilter_quantised(x, n1)
    assert kq == kf
    _, sq = o.filter_paper(cq, A, n1, n2, q, F, k_first=kq)
    assert max(abs(a - b) for a, b in zip(s, sq)) <= Fr(1, 1 << (F + 1))


@pytest.mark.parametrize("n1,n2", [(2, 0), (2, 1), (3, 0), (3, 2)])
def test_kernel_at_unit_scale_is_a_bspline_higher_model_degree(n1, n2):
    for t in (Fr(0), Fr(1, 4), Fr(3, 2), Fr(-9, 8)):
        assert o.kernel(n1, n2, 1, t) == o.bspline(n1 + n2 + 1, t)


def test_planted_causal_only_prefilter_is_caught():
    # dropping the anti-causal half of the inverse breaks interpolation
    h = o.inverse_filter(3)
    half = {k: (v if k >= 0 else Fr(0)) for k, v in h.items()}
    x = [7, -2, 5]
    c = {k: sum(x[j] * half.get(k - j, 0) for j in range(3)) for k in range(-20, 23)}
    b = {k: o.bspline(3, k) for k in (-1, 0, 1)}
    resid = max(abs(sum(c.get(k - d, 0) * w for d, w in b.items()) - (x[k] if 0 <= k < 3 else 0))
                for k in range(-5, 8))
    assert resid > Fr(1, 10)
