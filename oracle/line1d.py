"""The 1-D scale-adaptive B-spline filter of Sec. 3 (Proposition "prop"), in
exact rational / integer arithmetic.  TEST INFRASTRUCTURE ONLY (see the
package header).

What the method computes (Sec. 3): from samples f[k], the continuous model
f(x) = sum_k c[k] beta^{n1}(x - k) with f(k) = f[k], i.e. c = f * (b^{n1})^-1
with b^{n1}[k] = beta^{n1}(k); and the projections

    s[m] = < f, beta_a^{n2}(. - m) >,   m in Z,

with one scale a = a(m) > 0 per output sample.  beta^n is the centred B-spline
of degree n (Sec. 2, Eq. (definition) at a = 1) and beta_a^n(x) =
beta^n(x / a) / a its dilate (the same Fourier definition at scale a).  For
n1 in {0, 1}, b^{n1} is the unit impulse, so c = f and everything is exact.

How the Proposition computes it:
  1. Non-adaptive step: g = u_1^{(n2+1)} * c, n2 + 1 causal running sums.
  2. Adaptive step: s[m] = Delta_a^{n2+1} F(m)
         = a^-(n2+1) sum_{j=0}^{n2+1} (-1)^j binom(n2+1, j) F(m - a j),
     F(x) = sum_k g[k] beta^N(x + tau - k),  N = n1 + n2 + 1,
     tau = (a - 1)(n2 + 1) / 2  (Eq. (link)).

Exact form: with c = f 2^F integers and a = A 2^-Q, every evaluation point
y_j = m + tau - a j lies on the 2^-P grid, P = Q + 1, and D beta^N is an
integer there for D = N! 2^(N P).  The numerator
    S[m] = sum_j (-1)^j binom(n2+1, j) sum_k g[k] D beta^N(y_j - k)
is an integer and s[m] = S[m] 2^(Q (n2+1)) / (D A^(n2+1) 2^F).

Model degree n1 >= 2: the interpolation filter b^{n1} is no longer the unit
impulse and c = f * (b^{n1})^-1 has infinite support and irrational values.
The oracle takes the convolution inverse from its definition (the solution of
b^{n1} * h = delta on a wide window, exact rationals), convolves, and keeps c
to 2^-200.  The exact form rounds c to the 2^-F grid (c_q = rint(c 2^F), ties
to even) and runs the Proposition's two steps on c_q exactly; since the
kernel of s in terms of c has unit lattice sum and is non-negative, that
rounding moves s by at most 2^-(F+1).

Readings: zero signal outside [0, len) (as in 2-D);
beta^0 is 1 on (-1/2, 1/2] (Sec. 2); a_m is rounded to A = rint(a 2^Q), ties
to even, as the 2-D steps are.
"""
from fractions import Fraction as Fr
from math import comb, factorial, floor, ceil

import numpy as np


# ------------------------------------------------------------------ B-splines

def _tp(t, n):
    """Truncated power (t)_+^n, with (t)_+^0 = 1 for t > 0 and 0 for t <= 0
    (this half-open choice gives beta^0 = 1 on (-1/2, 1/2], Sec. 2)."""
    if t <= 0:
        return Fr(0)
    return Fr(t) ** n


def bspline(n, x):
    """beta^n(x): the inverse Fourier transform of Eq. (definition) at a = 1,
    in truncated-power form sum_i (-1)^i binom(n+1, i) (x + (n+1)/2 - i)_+^n / n!."""
    x = Fr(x)
    h = Fr(n + 1, 2)
    return sum((-1) ** i * comb(n + 1, i) * _tp(x + h - i, n) for i in range(n + 2)) / factorial(n)


def bspline_scaled(n, a, x):
    """beta_a^n(x) = beta^n(x / a) / a."""
    a = Fr(a)
    return bspline(n, Fr(x) / a) / a


# Piecewise polynomials: a polynomial is a list of Fraction coefficients
# (constant term first).

def _poly_mul(p, q):
    out = [Fr(0)] * (len(p) + len(q) - 1)
    for i, pi in enumerate(p):
        for j, qj in enumerate(q):
            out[i + j] += pi * qj
    return out


def _poly_affine_power(alpha, beta, n):
    """(alpha u + beta)^n as a polynomial in u."""
    return [Fr(comb(n, k)) * Fr(alpha) ** k * Fr(beta) ** (n - k) for k in range(n + 1)]


def _bspline_piece(n, a, shift, lo, hi):
    """beta_a^n(u - shift) on [lo, hi] (no knot inside) as a polynomial in u:
    the truncated powers that are positive on the interval, expanded."""
    a, shift = Fr(a), Fr(shift)
    mid = (Fr(lo) + Fr(hi)) / 2
    h = Fr(n + 1, 2)
    out = [Fr(0)] * (n + 1)
    for i in range(n + 2):
        # term (v + h - i)_+^n with v = (u - shift) / a
        if (mid - shift) / a + h - i <= 0:
            continue
        if n == 0:
            term = [Fr(1)]
        else:
            term = _poly_affine_power(1 / a, -shift / a + h - i, n)
        c = Fr((-1) ** i * comb(n + 1, i), factorial(n)) / a
        for k, tk in enumerate(term):
            out[k] += c * tk
    return out


def _knots(n, a, shift):
    a, shift = Fr(a), Fr(shift)
    return [shift + a * (Fr(i) - Fr(n + 1, 2)) for i in range(n + 2)]


def kernel(n1, n2, a, t):
    """K(t) = integral of beta^{n1}(u) beta_a^{n2}(u - t) du, exactly: the
    product is a polynomial between consecutive knots of the two factors."""
    a, t = Fr(a), Fr(t)
    k1, k2 = _knots(n1, 1, 0), _knots(n2, a, t)
    lo, hi = max(k1[0], k2[0]), min(k1[-1], k2[-1])
    if lo >= hi:
        return Fr(0)
    cuts = sorted(set([lo, hi] + [k for k in k1 + k2 if lo < k < hi]))
    total = Fr(0)
    for u0, u1 in zip(cuts[:-1], cuts[1:]):
        prod = _poly_mul(_bspline_piece(n1, 1, 0, u0, u1), _bspline_piece(n2, a, t, u0, u1))
        total += sum(c * (u1 ** (k + 1) - u0 ** (k + 1)) / (k + 1) for k, c in enumerate(prod))
    return total


# ---------------------------------------------------------- the definition

def quantise(a, q_bits):
    """A = rint(a 2^Q), ties to even (binary64), as the 2-D steps."""
    return np.rint(np.asarray(a, dtype=np.float64) * float(1 << q_bits)).astype(np.int64)


def filter_direct(c, A, n2, q_bits, n1, k_first=0, ms=None):
    """s[m] = sum_k c[k] K(m - k) for the quantised scales a_m = A_m 2^-Q,
    exact Fractions.  c holds the model coefficients at k = k_first,
    k_first + 1, ... (c = f for n1 in {0, 1}; `prefilter` for n1 >= 2), zero
    elsewhere; the outputs are the samples m of the signal (len(A) of them),
    or the samples ms."""
    c = [Fr(v) for v in c]
    kl, kh = k_first, k_first + len(c) - 1
    out = []
    for m in (range(len(A)) if ms is None else ms):
        m = int(m)
        a = Fr(int(A[m]), 1 << q_bits)
        reach = Fr(n1 + 1, 2) + a * Fr(n2 + 1, 2)
        k0, k1 = max(kl, floor(m - reach)), min(kh, ceil(m + reach))
        out.append(sum(c[k - k_first] * kernel(n1, n2, a, m - k) for k in range(k0, k1 + 1)))
    return out


# ------------------------------------ the interpolation prefilter (n1 >= 2)

def interp_filter(n1):
    """b^{n1}[k] = beta^{n1}(k) on its support |k| <= n1 // 2 (exact)."""
    M = n1 // 2
    return {k: bspline(n1, k) for k in range(-M, M + 1)}


_INVERSE = {}


def inverse_filter(n1, E=160):
    """The convolution inverse (b^{n1})^-1 on [-E, E]: the solution h of
    sum_j b[k - j] h[j] = delta[k] for |k| <= E with h = 0 outside, by banded
    Gaussian elimination in exact rationals (the matrix is symmetric Toeplitz
    and strictly diagonally dominant for n1 >= 2, so no pivoting).  It differs
    from the bounded inverse on Z by O(|z|^(E - |k|)), |z| < 0.44 the largest
    root of the filter's symbol: below 2^-190 at the centre taps used here."""
    key = (n1, E)
    if key in _INVERSE:
        return _INVERSE[key]
    b = interp_filter(n1)
    M = max(b)
    n = 2 * E + 1
    rows = [{j: b[i - j] for j in range(max(0, i - M), min(n, i + M + 1))} for i in range(n)]
    rhs = [Fr(1) if i == E else Fr(0) for i in range(n)]
    for i in range(n):
        piv = rows[i][i]
        for r in range(i + 1, min(n, i + M + 1)):
            if rows[r].get(i, 0) == 0:
                continue
            fct = rows[r][i] / piv
            for j, v in rows[i].items():
                if j >= i:
                    rows[r][j] = rows[r].get(j, Fr(0)) - fct * v
            rhs[r] -= fct * rhs[i]
    h = [Fr(0)] * n
    for i in reversed(range(n)):
        acc = rhs[i] - sum(v * h[j] for j, v in rows[i].items() if j > i)
        h[i] = acc / rows[i][i]
    out = {k: h[k + E] for k in range(-E, E + 1)}
    _INVERSE[key] = out
    return out


def rint_shift(v, bits):
    """rint(v 2^-bits) for an integer v, ties to even."""
    q, r = divmod(v, 1 << bits)
    half = 1 << (bits - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return q


def prefilter(x_int, n1, bits=200):
    """c = f * (b^{n1})^-1 for f zero outside [0, len), f 2^F = x_int:
    returns (k_first, cs) with cs[i] = rint(c[k_first + i] 2^(F + bits)), the
    coefficients for k in [k_first, len - k_first).  Taps of the inverse below
    2^-(bits+1) are dropped; c beyond the returned range is below 2^-bits |x|."""
    h = inverse_filter(n1)
    taps = {k: round(v * (1 << bits)) for k, v in h.items()}  # Fraction rounding: ties to even
    E = max(abs(k) for k, t in taps.items() if t != 0)
    hk = np.array([taps[k] for k in range(-E, E + 1)], dtype=object)
    xs = np.array([int(v) for v in x_int], dtype=object)
    cs = np.convolve(xs, hk)  # index i <-> k = i - E
    return -E, [int(v) for v in cs]


def prefilter_quantised(x_int, n1, bits=200):
    """(k_first, c_q): c_q = rint(c 2^F), ties to even, on the range of
    `prefilter` (the exact form's model coefficients)."""
    k_first, cs = prefilter(x_int, n1, bits)
    return k_first, [rint_shift(v, bits) for v in cs]


# -------------------------------------------------- the Proposition, exact

def p_bits(q_bits):
    """Grid of the evaluation points y_j = m + tau - a j: 2^-(Q+1)."""
    return q_bits + 1


def denominator(N, P):
    """D = N! 2^(N P): D beta^N is an integer on the 2^-P grid."""
    return factorial(N) << (N * P)


def dbspline_int(N, P, X):
    """D beta^N(X 2^-P) as an integer, from the truncated-power form scaled by
    2^(N P) N! (every term is an integer power on the 2^-P grid)."""
    h = (N + 1) << (P - 1)  # (N+1)/2 in units of 2^-P
    tot = 0
    for i in range(N + 2):
        t = X + h - (i << P)
        if t > 0:
            tot += (-1) ** i * comb(N + 1, i) * t ** N
    return tot


def running_sums(c, times, length):
    """g = u_1^{(times)} * c on [0, length): `times` causal running sums, with
    c = 0 outside its support (zero signal outside [0, len)).  Index 0 is the
    first coefficient of c, wherever it sits on the signal axis."""
    g = [int(v) for v in c] + [0] * (length - len(c))
    for _ in range(times):
        acc = 0
        for k in range(length):
            acc += g[k]
            g[k] = acc
    return g


def box_right(n1, n2, q_bits, A_max):
    """Samples beyond the signal end that the adaptive step reads: tau_max +
    (N+1)/2 + 1 (the running sums keep growing there)."""
    N = n1 + n2 + 1
    tau_max = Fr(max(A_max - (1 << q_bits), 0) * (n2 + 1), 1 << (q_bits + 1))
    return int(ceil(tau_max + Fr(N + 1, 2))) + 2


def filter_paper(c_int, A, n1, n2, q_bits, frac_bits=0, k_first=0):
    """The two steps of the Proposition in exact integers: returns the
    numerators S[m] (Python ints) and s[m] (Fractions) for the len(A) samples
    of the signal.  c_int = c 2^F at k = k_first, k_first + 1, ... (c = f for
    n1 in {0, 1}; `prefilter_quantised` for n1 >= 2)."""
    return filter_paper_at(c_int, A, n1, n2, q_bits, frac_bits, range(len(A)), k_first)


def filter_paper_at(c_int, A, n1, n2, q_bits, frac_bits, ms, k_first=0):
    """filter_paper at the samples ms only (the running sums still cover the
    whole signal)."""
    n = len(A)
    N = n1 + n2 + 1
    P = p_bits(q_bits)
    D = denominator(N, P)
    right = box_right(n1, n2, q_bits, int(np.max(A)) if n else 0)
    g = running_sums(c_int[: n + right - k_first], n2 + 1, n + right - k_first)  # g[i] <-> k = k_first + i
    h = Fr(N + 1, 2)
    S_all, s_all = [], []
    for m in ms:
        m = int(m)  # Python integers throughout (numpy scalars would overflow)
        Am = int(A[m])
        tauP = (Am - (1 << q_bits)) * (n2 + 1)          # tau in units of 2^-P
        S = 0
        for j in range(n2 + 2):
            Y = (m << P) + tauP - 2 * Am * j            # y_j in units of 2^-P
            y = Fr(Y, 1 << P)
            k0, k1 = floor(y - h), ceil(y + h)
            F = 0
            for k in range(max(k0, k_first), k1 + 1):
                F += g[k - k_first] * dbspline_int(N, P, Y - (k << P))
            S += (-1) ** j * comb(n2 + 1, j) * F
        S_all.append(S)
        s_all.append(Fr(S * (1 << (q_bits * (n2 + 1))), D * Am ** (n2 + 1) * (1 << frac_bits)))
    return S_all, s_all
