"""Exact box-spline values (test infrastructure only; see package header).

Two evaluators, both built on de Boor's box-spline recurrence:

1. ``BoxSpline`` -- point values of the (uncentred or centred) box spline with an
   arbitrary multiset of 2-D direction vectors.  Used for the direct definition
   of the filter: the kernel beta^4_a of Sec. 4 Eq. (def) (N=4, theta_k =
   (k-1) pi/4), whose k-th direction vector is a_k r_{theta_k}; in lattice
   units that is c_k v_k with v = (1,0), (1,1), (0,1), (-1,1) (Sec. 7).

2. ``zp_piece`` / ``zp_value`` -- the Zwart-Powell element of Sec. 7 (the box
   spline beta^4_b with b = (1, sqrt2, 1, sqrt2), i.e. unit lattice directions
   v1..v4) and its n-fold self-convolution, as exact polynomial pieces on the
   triangles of the four-direction mesh (lines x = i, y = j, x +- y = k).  This
   is the interpolation kernel g_I of Eq. (final_eqn).

Normalisation: every box spline here has integral 1 (the density of
sum_k t_k xi_k with t uniform on [0,1)^N).  Sec. 7 calls 2 beta^4_b the ZP
element; the paper's beta^4_b already has integral 1 (each phi_{a,theta} of
Eq. (generator) has integral 1), which is the kernel used here.

de Boor's recurrence, for x = sum_xi lambda_xi xi and #Xi = N > 2:

    (N - 2) M_Xi(x) = sum_xi [lambda_xi M_{Xi\\xi}(x) + (1 - lambda_xi) M_{Xi\\xi}(x - xi)],

with M of a multiset that does not span R^2 taken as 0, and for N = 2 the
scaled indicator 1/|det| of the half-open parallelogram.  Point values are taken
as limits from the fixed direction PERTURB (not parallel to any direction), so
points on break lines get a definite, consistent value; wherever the spline is
continuous (always, here: N >= 4 pairwise independent directions) that limit
is the value itself.
"""
from fractions import Fraction as Fr
from functools import lru_cache
from math import comb, gcd

# Lattice direction vectors of Sec. 7: theta = 0, pi/4, pi/2, 3pi/4 with
# b = (1, sqrt2, 1, sqrt2), so b_k r_{theta_k} = v_k.
LATTICE_DIRS = ((1, 0), (1, 1), (0, 1), (-1, 1))

# Direction of the one-sided limit used at break lines (not parallel to any v_k).
PERTURB = (3, 1)


# ---------------------------------------------------------------- polynomials
# A bivariate polynomial is a dict {(i, j): coefficient} meaning sum c x^i y^j.

def _padd(acc, p, s=1):
    for k, v in p.items():
        acc[k] = acc.get(k, 0) + s * v


def _pmul_linear(p, a, b):
    """p(x, y) * (a x + b y)."""
    r = {}
    for (i, j), v in p.items():
        if a:
            r[(i + 1, j)] = r.get((i + 1, j), 0) + a * v
        if b:
            r[(i, j + 1)] = r.get((i, j + 1), 0) + b * v
    return r


def _pshift(p, dx, dy):
    """The polynomial x -> p(x - dx, y - dy)."""
    r = {}
    for (i, j), v in p.items():
        for a in range(i + 1):
            ca = comb(i, a) * (-dx) ** (i - a)
            if ca == 0:
                continue
            for b in range(j + 1):
                cb = comb(j, b) * (-dy) ** (j - b)
                if cb == 0:
                    continue
                r[(a, b)] = r.get((a, b), 0) + v * ca * cb
    return {k: v for k, v in r.items() if v != 0}


def poly_eval(p, x, y):
    return sum(v * x ** i * y ** j for (i, j), v in p.items())


# ------------------------------------------------- pointwise general evaluator

def _solve2(a, b, x):
    """Coefficients (u, w) with x = u a + w b (exact)."""
    det = a[0] * b[1] - a[1] * b[0]
    u = Fr(x[0] * b[1] - x[1] * b[0]) / det
    w = Fr(a[0] * x[1] - a[1] * x[0]) / det
    return u, w


def _open_unit(u, pu):
    """Is u + eps*pu in (0, 1) for all small eps > 0?"""
    if 0 < u < 1:
        return True
    if u == 0:
        return pu > 0
    if u == 1:
        return pu < 0
    return False


class BoxSpline:
    """Uncentred box spline M_Xi for Xi = the directions ``dirs`` with
    multiplicities ``counts`` (exact, any rational direction vectors, pairwise
    non-parallel).  ``value(x)`` is lim_{eps->0+} M_Xi(x + eps PERTURB)."""

    def __init__(self, dirs, counts):
        self.dirs = tuple((Fr(d[0]), Fr(d[1])) for d in dirs)
        self.counts = tuple(counts)
        self.memo = {}

    def _m(self, counts, x):
        key = (counts, x)
        hit = self.memo.get(key)
        if hit is not None:
            return hit
        present = [k for k, c in enumerate(counts) if c > 0]
        n_tot = sum(counts)
        val = Fr(0)
        if len(present) >= 2:
            if n_tot == 2:
                a, b = (self.dirs[k] for k in present)
                u, w = _solve2(a, b, x)
                pu, pw = _solve2(a, b, PERTURB)
                if _open_unit(u, pu) and _open_unit(w, pw):
                    val = 1 / abs(Fr(a[0] * b[1] - a[1] * b[0]))
            else:
                ka, kb = present[0], present[1]
                lam_a, lam_b = _solve2(self.dirs[ka], self.dirs[kb], x)
                acc = Fr(0)
                for k in present:
                    sub = list(counts)
                    sub[k] -= 1
                    sub = tuple(sub)
                    d = self.dirs[k]
                    xs = (x[0] - d[0], x[1] - d[1])
                    m_shift = self._m(sub, xs)
                    acc += counts[k] * m_shift
                    if k == ka:
                        acc += lam_a * (self._m(sub, x) - m_shift)
                    elif k == kb:
                        acc += lam_b * (self._m(sub, x) - m_shift)
                val = acc / (n_tot - 2)
        self.memo[key] = val
        return val

    def value(self, x, y):
        return self._m(self.counts, (Fr(x), Fr(y)))

    def centre(self):
        """Half the sum of all direction vectors: M(. + centre) is symmetric."""
        cx = sum(c * d[0] for c, d in zip(self.counts, self.dirs)) / 2
        cy = sum(c * d[1] for c, d in zip(self.counts, self.dirs)) / 2
        return cx, cy

    def centred_value(self, x, y):
        cx, cy = self.centre()
        return self.value(Fr(x) + cx, Fr(y) + cy)


def kernel_B(c, n):
    """The filter kernel for lattice steps c = (c1..c4): the box spline with
    direction vectors c_k v_k, each n times (Sec. 4 Eq. (def) with N = 4, order n
    read as n-fold self-convolution), centred and of integral 1."""
    dirs = [(Fr(ck) * v[0], Fr(ck) * v[1]) for ck, v in zip(c, LATTICE_DIRS)]
    return BoxSpline(dirs, (n, n, n, n))


# ------------------------------------------------- ZP^n as polynomial pieces
# Cells of the four-direction mesh: each unit square [i,i+1]x[j,j+1] is cut by
# its two diagonals into triangles t = 0 (bottom), 1 (right), 2 (top), 3 (left).
# A cell is named (i, j, t); its centroid is an interior point.

_CENTROIDS = ((Fr(1, 2), Fr(1, 6)), (Fr(5, 6), Fr(1, 2)),
              (Fr(1, 2), Fr(5, 6)), (Fr(1, 6), Fr(1, 2)))

_piece_memo = {}


def _in_zonotope(counts, x, y):
    """Is (x, y) strictly inside the support sum_k [0, counts_k] v_k?"""
    c1, c2, c3, c4 = counts
    return (-c4 < x < c1 + c2 and 0 < y < c2 + c3 + c4
            and 0 < x + y < c1 + 2 * c2 + c3 and -c3 - 2 * c4 < x - y < c1)


def _uncentred_piece(counts, rep):
    """Polynomial equal to M_Xi on the open mesh cell containing ``rep``, where
    Xi = the lattice directions with multiplicities ``counts`` (de Boor's
    recurrence carried out on polynomials; every sub-spline is one polynomial
    on a mesh cell because all its break lines are mesh lines)."""
    key = (counts, rep)
    hit = _piece_memo.get(key)
    if hit is not None:
        return hit
    present = [k for k in range(4) if counts[k] > 0]
    n_tot = sum(counts)
    x, y = rep
    res = {}
    if len(present) >= 2 and _in_zonotope(counts, x, y):
        if n_tot == 2:
            a, b = (LATTICE_DIRS[k] for k in present)
            u, w = _solve2(a, b, (x, y))
            if 0 < u < 1 and 0 < w < 1:
                res = {(0, 0): 1 / abs(Fr(a[0] * b[1] - a[1] * b[0]))}
        else:
            ka, kb = present[0], present[1]
            va, vb = LATTICE_DIRS[ka], LATTICE_DIRS[kb]
            det = va[0] * vb[1] - va[1] * vb[0]
            # lambda_a(x) = (x vb_y - y vb_x)/det, lambda_b(x) = (va_x y - va_y x)/det
            lam = {ka: (Fr(vb[1], det), Fr(-vb[0], det)),
                   kb: (Fr(-va[1], det), Fr(va[0], det))}
            acc = {}
            for k in present:
                sub = list(counts)
                sub[k] -= 1
                sub = tuple(sub)
                vk = LATTICE_DIRS[k]
                shifted = _pshift(_uncentred_piece(sub, (x - vk[0], y - vk[1])), vk[0], vk[1])
                _padd(acc, shifted, counts[k])
                if k in lam:
                    diff = dict(_uncentred_piece(sub, rep))
                    _padd(diff, shifted, -1)
                    _padd(acc, _pmul_linear(diff, *lam[k]))
            res = {kk: v / (n_tot - 2) for kk, v in acc.items() if v != 0}
    _piece_memo[key] = res
    return res


@lru_cache(maxsize=None)
def zp_pieces(n):
    """All non-zero polynomial pieces of the uncentred ZP^{*n}
    (directions v1..v4, each n times), keyed by cell (i, j, t)."""
    counts = (n, n, n, n)
    out = {}
    for i in range(-n - 1, 2 * n + 1):
        for j in range(-1, 3 * n + 1):
            for t, (cx, cy) in enumerate(_CENTROIDS):
                p = _uncentred_piece(counts, (i + cx, j + cy))
                if p:
                    out[(i, j, t)] = p
    return out


def _cell_of(x, y):
    """Mesh cell whose closure holds (x, y), chosen as the cell entered by
    (x, y) + eps PERTURB (any closure cell gives the same value: ZP^{*n} is
    continuous)."""
    i = x.numerator // x.denominator
    j = y.numerator // y.denominator
    fx, fy = x - i, y - j
    below_main = fy <= fx          # ties go below: PERTURB has py < px
    above_anti = fx + fy >= 1      # ties go above: px + py > 0
    if below_main:
        t = 1 if above_anti else 0
    else:
        t = 2 if above_anti else 3
    return i, j, t


def zp_shift(n):
    """Centre of the uncentred ZP^{*n}: n (1/2, 3/2) = half the sum of v1..v4, n times."""
    return Fr(n, 2), Fr(3 * n, 2)


def zp_value_uncentred(n, x, y):
    x, y = Fr(x), Fr(y)
    p = zp_pieces(n).get(_cell_of(x, y))
    return poly_eval(p, x, y) if p else Fr(0)


def zp_value(n, x, y):
    """Centred ZP^{*n}(x, y): the interpolation kernel g_I of Eq. (final_eqn)
    for n = 1, its n-fold self-convolution for order n."""
    sx, sy = zp_shift(n)
    return zp_value_uncentred(n, Fr(x) + sx, Fr(y) + sy)


@lru_cache(maxsize=None)
def zp_integer_denominator(n):
    """LCD of the values of the uncentred ZP^{*n} at the integer points."""
    d = 1
    for i in range(-n, 2 * n + 1):
        for j in range(0, 3 * n + 1):
            v = zp_value_uncentred(n, i, j)
            d = d * v.denominator // gcd(d, v.denominator)
    return d


def zp_denominator(n, p_bits):
    """Common denominator D = D0 * 2^((4n-2) P) of ZP^{*n} on the centred
    2^-P grid (P >= 1), D0 = zp_integer_denominator(n).  The refinement
    equation of a box spline with 4n unit directions multiplies denominators by
    at most 2^(4n-2) per halving of the grid, and for odd n the centred grid
    sits on the half-integer points of the uncentred one."""
    return zp_integer_denominator(n) << ((4 * n - 2) * p_bits)


class ZPIntegerWeights:
    """Integer interpolation weights D * ZP^{*n}(r - d) for the 3n x 3n lattice
    neighbours d of a point y = p + r on the 2^-P grid (memoised per offset).

    Conventions (restated independently in the CUDA path):
      n even: p = floor(y), r in [0, 1),            d in {-3n/2+1, ..., 3n/2}
      n odd:  p = floor(y + 1/2), r in [-1/2, 1/2), d in {-(3n-1)/2, ..., (3n-1)/2}
    These d cover every lattice point k = p + d with y - k inside the open
    support |x|, |y| < 3n/2 of the centred kernel.

    Each polynomial piece is rewritten once in integer grid coordinates
    (x = X 2^-P): D p(X 2^-P, Y 2^-P) = (sum A_ij X^i Y^j) / K with integers
    A_ij, K, so a weight costs a few integer operations and one exact division.
    """

    def __init__(self, n, p_bits):
        self.n, self.P = n, p_bits
        self.D = zp_denominator(n, p_bits)
        self.dmin = -(3 * n) // 2 + 1 if n % 2 == 0 else -(3 * n - 1) // 2
        self.cache = {}
        sx, sy = zp_shift(n)
        self.SX, self.SY = int(sx * (1 << p_bits)), int(sy * (1 << p_bits))
        self.pieces = {}
        for cell, poly in zp_pieces(n).items():
            terms = {}
            for (i, j), v in poly.items():
                terms[(i, j)] = v * self.D / (1 << (p_bits * (i + j)))
            k = 1
            for v in terms.values():
                k = k * v.denominator // gcd(k, v.denominator)
            self.pieces[cell] = ([(i, j, int(v * k)) for (i, j), v in terms.items()], k)

    def split(self, yq):
        """yq = y * 2^P (an integer) -> (p, ridx) with y = p + r, ridx in [0, 2^P)."""
        one = 1 << self.P
        if self.n % 2 == 0:
            p = yq >> self.P
            return p, yq - (p << self.P)
        p = (yq + (one >> 1)) >> self.P
        return p, yq - (p << self.P) + (one >> 1)

    def uncentred_grid_value(self, X, Y):
        """D * (uncentred ZP^{*n})(X 2^-P, Y 2^-P), exact integer."""
        P = self.P
        i, j = X >> P, Y >> P
        fx, fy = X - (i << P), Y - (j << P)
        below_main = fy <= fx
        above_anti = fx + fy >= (1 << P)
        t = (1 if above_anti else 0) if below_main else (2 if above_anti else 3)
        piece = self.pieces.get((i, j, t))
        if piece is None:
            return 0
        terms, k = piece
        num = 0
        for a, b, coef in terms:
            num += coef * X ** a * Y ** b
        q, rem = divmod(num, k)
        assert rem == 0, "ZP weight not integral on the 2^-P grid"
        return q

    def row(self, rx, ry):
        """Weights for offset indices (rx, ry) in [0, 2^P)^2 as a (3n) x (3n)
        nested list indexed [dy - dmin][dx - dmin]."""
        key = (rx, ry)
        hit = self.cache.get(key)
        if hit is not None:
            return hit
        n, P = self.n, self.P
        half = (1 << (P - 1)) if n % 2 else 0
        out = []
        for iy in range(3 * n):
            dy = self.dmin + iy
            Y = ry - half - (dy << P) + self.SY
            out.append([self.uncentred_grid_value(rx - half - ((self.dmin + ix) << P) + self.SX, Y)
                        for ix in range(3 * n)])
        self.cache[key] = out
        return out
