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
