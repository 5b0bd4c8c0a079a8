"""Two further members of the paper's method, exact (test infrastructure only;
see package header).  oracle.paper holds the four-direction algorithm of
Sec. 7 with phi = delta; this module keeps that code as it is and restates the
method for

(a) directional order N = 2.  Sec. 4 Eq. (def) takes the directions
    theta_k = (k-1) pi / N; the RS filters of Eq. (RS_filter) exist only when
    b cos theta_k and b sin theta_k are integers for some b, which among
    N >= 2 holds for N = 2 (theta = 0, pi/2; b = (1, 1)) and N = 4 (Sec. 7):
    for any other N, tan(pi / N) is irrational (a rational multiple of pi
    has a rational tangent only at 0 and +-pi/4).  N = 2 gives the tensor box
    splines (Sec. 4: rect = beta^2_(1,1)), built here from the directions
    v1 = (1, 0) and v3 = (0, 1) alone.

(b) the interpolation model of Sec. 6, f(x) = sum_k c[k] phi(x - k) with
    c = f * (b^n)^-1, b^n[k] = phi(k), phi the tensor B-spline
    beta^{n1}(x1) beta^{n1}(x2) (a reading: Sec. 6 leaves phi open; Sec. 3
    uses B-splines).  Eq. (NA) without interpolation runs the running sums on
    c, and Eq. (mask) interpolates with phi * beta^N_b: the box spline whose
    directions are the FD/RS directions plus n1 + 1 further copies of v1 and
    of v3 (beta^{n1} is n1 + 1 unit boxes).  c is irrational for n1 >= 2; as
    in the 1-D filter it is rounded to the 2^-F grid, c_q = rint(c 2^F), and
    the method runs exactly on c_q.

A problem is given by the counts r = (r1, r2, r3, r4) of the FD / RS
directions (r = (n, n, n, n) for N = 4 at order n, (n, 0, n, 0) for N = 2)
and the model degree n1 (None for phi = delta).  Then

    g     = U_{v1}^{r1} U_{v2}^{r2} U_{v3}^{r3} U_{v4}^{r4} c          (Eq. (RS), unit weights)
    tau   = (1/2) sum_k r_k (c_k - 1) v_k                              (Sec. 5, Eq. (factor))
    S[m]  = D sum_j w_j g_I(m + tau - sum_k j_k c_k v_k),  j_k in {0..r_k},
            w_j = prod_k (-1)^{j_k} binom(r_k, j_k)                    (Eq. (FD), Eq. (mask))
    g_I(y) = sum_k g[k] M(y - k),  M = the centred box spline with v_k r_k times
            and, for a model, v1 and v3 n1 + 1 more times each
    s[m]  = S[m] / (D prod_k c_k^{r_k} 2^F)

and, from the definition (Sec. 6), s[m] = sum_k c_q[k] 2^-F B(m - k) with B
the centred box spline with directions c_k v_k (r_k times each) and unit
v1, v3 (n1 + 1 times each).
"""
from fractions import Fraction as Fr
from itertools import product
from math import comb, gcd

import numpy as np

from .boxspline import LATTICE_DIRS, BoxSpline, PERTURB, _uncentred_piece, _cell_of, poly_eval, _solve2, _open_unit
from . import line1d


def interp_counts(r, n1):
    """Direction counts of the interpolation kernel M of Eq. (mask)."""
    m = list(r)
    if n1 is not None:
        m[0] += n1 + 1
        m[2] += n1 + 1
    return tuple(m)


# --------------------------------------------------------- kernels, exact

class SpanBoxSpline(BoxSpline):
    """BoxSpline for direction multisets that may hold parallel vectors (c1 v1
    and v1): de Boor's recurrence with its coordinate pair taken from two
    non-parallel present directions; a multiset that does not span R^2 gives 0
    (its box spline is not a function of the plane)."""

    def _m(self, counts, x):
        key = (counts, x)
        hit = self.memo.get(key)
        if hit is not None:
            return hit
        present = [k for k, c in enumerate(counts) if c > 0]
        pair = None
        for i in range(len(present)):
            for j in range(i + 1, len(present)):
                a, b = self.dirs[present[i]], self.dirs[present[j]]
                if a[0] * b[1] - a[1] * b[0] != 0:
                    pair = (present[i], present[j])
                    break
            if pair:
                break
        n_tot = sum(counts)
        val = Fr(0)
        if pair is not None:
            ka, kb = pair
            if n_tot == 2:
                a, b = self.dirs[ka], self.dirs[kb]
                u, w = _solve2(a, b, x)
                pu, pw = _solve2(a, b, PERTURB)
                if _open_unit(u, pu) and _open_unit(w, pw):
                    val = 1 / abs(Fr(a[0] * b[1] - a[1] * b[0]))
            else:
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


def kernel_direct(c, r, n1):
    """The filter kernel B of the definition: directions c_k v_k (r_k times)
    and, for a model of degree n1, unit v1 and v3 (n1 + 1 times each);
    integral 1; evaluate with centred_value."""
    dirs, counts = [], []
    for ck, v, rk in zip(c, LATTICE_DIRS, r):
        if rk:
            dirs.append((Fr(ck) * v[0], Fr(ck) * v[1]))
            counts.append(rk)
    if n1 is not None:
        dirs += [(Fr(1), Fr(0)), (Fr(0), Fr(1))]
        counts += [n1 + 1, n1 + 1]
    return SpanBoxSpline(dirs, counts)


def _in_support(m, x, y):
    c1, c2, c3, c4 = m
    return (-c4 < x < c1 + c2 and 0 < y < c2 + c3 + c4
            and 0 < x + y < c1 + 2 * c2 + c3 and -c3 - 2 * c4 < x - y < c1)


_PIECES = {}


def mesh_pieces(m):
    """Polynomial pieces of the uncentred box spline with the lattice
    directions v1..v4 taken m = (m1..m4) times, on the cells of the
    four-direction mesh (every break line is a mesh line)."""
    if m in _PIECES:
        return _PIECES[m]
    from .boxspline import _CENTROIDS
    out = {}
    for i in range(-m[3] - 1, m[0] + m[1] + 1):
        for j in range(-1, m[1] + m[2] + m[3] + 1):
            for t, (cx, cy) in enumerate(_CENTROIDS):
                x, y = i + cx, j + cy
                if not _in_support(m, x, y):
                    continue
                p = _uncentred_piece(m, (x, y))
                if p:
                    out[(i, j, t)] = p
    _PIECES[m] = out
    return out


def centre(m):
    """Half the sum of the directions: the uncentred kernel's centre."""
    return (Fr(m[0] + m[1] - m[3], 2), Fr(m[1] + m[2] + m[3], 2))


def integer_denominator(m):
    """Least common denominator D0 of the uncentred kernel at integer points."""
    d = 1
    for i in range(-m[3], m[0] + m[1] + 1):
        for j in range(0, m[1] + m[2] + m[3] + 1):
            p = mesh_pieces(m).get(_cell_of(Fr(i), Fr(j)))
            if p:
                v = poly_eval(p, Fr(i), Fr(j))
                d = d * v.denominator // gcd(d, v.denominator)
    return d


class MeshWeights:
    """Integer weights D M(y - k) for a point y on the 2^-P grid and its
    lattice neighbours k = p + d, p = floor(y), d in [dmin, dmin + width)^2,
    with D = D0 2^((sum m - 2) P) (the refinement equation of a box spline
    with sum m unit directions multiplies denominators by 2^(sum m - 2) per
    halving of the grid).  Points are handled in integer grid units."""

    def __init__(self, m, p_bits):
        self.m, self.P = tuple(m), p_bits
        self.D = integer_denominator(self.m) << ((sum(self.m) - 2) * p_bits)
        cx, cy = centre(self.m)
        self.CX, self.CY = int(cx * (1 << p_bits)), int(cy * (1 << p_bits))
        # centred support |x| < hx, |y| < hy: neighbours k with y - k inside
        hx = Fr(self.m[0] + self.m[1] + self.m[3], 2)
        hy = Fr(self.m[1] + self.m[2] + self.m[3], 2)
        self.dminx = -int(hx) - 1
        self.dminy = -int(hy) - 1
        self.wx = 2 * int(hx) + 3
        self.wy = 2 * int(hy) + 3
        self.pieces = {}
        for cell, poly in mesh_pieces(self.m).items():
            terms = {}
            for (i, j), v in poly.items():
                terms[(i, j)] = v * self.D / (1 << (p_bits * (i + j)))
            k = 1
            for v in terms.values():
                k = k * v.denominator // gcd(k, v.denominator)
            self.pieces[cell] = ([(i, j, int(v * k)) for (i, j), v in terms.items()], k)
        self.cache = {}

    def uncentred(self, X, Y):
        """D M_uncentred(X 2^-P, Y 2^-P), an exact integer."""
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
        num = sum(coef * X ** a * Y ** b for a, b, coef in terms)
        q, rem = divmod(num, k)
        assert rem == 0, "kernel weight not integral on the 2^-P grid"
        return q

    def value(self, Xq, Yq):
        """D M(x, y) (centred) at (Xq, Yq) 2^-P."""
        return self.uncentred(Xq + self.CX, Yq + self.CY)

    def row(self, rx, ry):
        """Weights of a point p + r, r = (rx, ry) 2^-P in [0, 1)^2, for the
        neighbours p + d, d in [dminx, dminx + wx) x [dminy, dminy + wy), as a
        list indexed [iy][ix] (memoised per offset)."""
        key = (rx, ry)
        hit = self.cache.get(key)
        if hit is None:
            P = self.P
            hit = [[self.value(rx - ((self.dminx + ix) << P), ry - ((self.dminy + iy) << P))
                    for ix in range(self.wx)] for iy in range(self.wy)]
            self.cache[key] = hit
        return hit


# ------------------------------------------------------------ the method

def p_bits(q_bits):
    """Grid of every tap offset and of the kernel's centre: 2^-(Q+1)."""
    return q_bits + 1


def taps(r):
    """[(j, w_j)] over j_k in {0..r_k}."""
    out = []
    for j in product(*[range(rk + 1) for rk in r]):
        w = 1
        for jk, rk in zip(j, r):
            w *= (-1) ** jk * comb(rk, jk)
        out.append((j, w))
    return out


def tau(c, r):
    tx = sum(Fr(rk, 2) * (Fr(ck) - 1) * v[0] for ck, v, rk in zip(c, LATTICE_DIRS, r))
    ty = sum(Fr(rk, 2) * (Fr(ck) - 1) * v[1] for ck, v, rk in zip(c, LATTICE_DIRS, r))
    return tx, ty


def integrate(c_int, r, x0, x1, y0, y1):
    """g on the lattice box [x0, x1) x [y0, y1) (coordinates of c_int's
    array, c = 0 outside it): r1 running sums along v1, then r2 along v2, r3
    along v3, r4 along v4 (the paper's order), exact; rows carried out far
    enough to the right that the 3pi/4 sums are exact on the box."""
    c_int = np.asarray(c_int, dtype=object)
    H, W = c_int.shape
    rows, cols = y1 - y0, x1 - x0
    width = cols + rows
    prev = [[0] * width for _ in range(r[1] + r[2] + r[3])]
    out = np.zeros((rows, cols), dtype=object)
    for yi in range(rows):
        y = y0 + yi
        row = [0] * width
        if 0 <= y < H:
            for x in range(W):
                xi = x - x0
                if 0 <= xi < width:
                    row[xi] = int(c_int[y, x])
        for _ in range(r[0]):
            acc = 0
            for i in range(width):
                acc += row[i]
                row[i] = acc
        s = 0
        for _ in range(r[1]):
            cur = [row[i] + (prev[s][i - 1] if i else 0) for i in range(width)]
            prev[s] = cur
            row = cur
            s += 1
        for _ in range(r[2]):
            cur = [row[i] + prev[s][i] for i in range(width)]
            prev[s] = cur
            row = cur
            s += 1
        for _ in range(r[3]):
            cur = [row[i] + (prev[s][i + 1] if i + 1 < width else 0) for i in range(width)]
            prev[s] = cur
            row = cur
            s += 1
        out[yi] = row[:cols]
    return out


class Method:
    """The adaptive step with direction counts r and model degree n1, exact."""

    def __init__(self, r, n1, q_bits):
        self.r, self.n1, self.Q = tuple(r), n1, q_bits
        self.P = p_bits(q_bits)
        self.mw = MeshWeights(interp_counts(self.r, n1), self.P)
        self.D = self.mw.D
        self.verts = taps(self.r)

    def reach(self, C):
        """Lattice margins (left, right, below, above) that a pixel's taps and
        their kernel support cover."""
        c = [Fr(int(v), 1 << self.Q) for v in C]
        tx, ty = tau(c, self.r)
        xs, ys = [], []
        for j, _ in self.verts:
            xs.append(tx - sum(jk * ck * v[0] for jk, ck, v in zip(j, c, LATTICE_DIRS)))
            ys.append(ty - sum(jk * ck * v[1] for jk, ck, v in zip(j, c, LATTICE_DIRS)))
        mw = self.mw
        left = -int(np.floor(float(min(xs)))) - mw.dminx + 2
        right = int(np.ceil(float(max(xs)))) + mw.dminx + mw.wx + 2
        below = -int(np.floor(float(min(ys)))) - mw.dminy + 2
        above = int(np.ceil(float(max(ys)))) + mw.dminy + mw.wy + 2
        return left, right, below, above

    def numerator(self, gget, m1, m2, C):
        c = [Fr(int(v), 1 << self.Q) for v in C]
        tx, ty = tau(c, self.r)
        one = 1 << self.P
        mw = self.mw
        S = 0
        for j, w in self.verts:
            yx = (m1 + tx - sum(jk * ck * v[0] for jk, ck, v in zip(j, c, LATTICE_DIRS))) * one
            yy = (m2 + ty - sum(jk * ck * v[1] for jk, ck, v in zip(j, c, LATTICE_DIRS))) * one
            assert yx.denominator == 1 and yy.denominator == 1
            X, Y = int(yx), int(yy)
            px, py = X >> self.P, Y >> self.P
            wrow = mw.row(X - (px << self.P), Y - (py << self.P))
            acc = 0
            for iy in range(mw.wy):
                k2 = py + mw.dminy + iy
                line = wrow[iy]
                for ix in range(mw.wx):
                    wt = line[ix]
                    if wt:
                        acc += int(gget(px + mw.dminx + ix, k2)) * wt
            S += w * acc
        return S

    def denominator(self, C, f_bits):
        prod = Fr(1)
        for ck, rk in zip(C, self.r):
            prod *= Fr(int(ck), 1 << self.Q) ** rk
        return self.D * prod * (1 << f_bits)


def filter_pixels(c_int, origin, C, r, n1, q_bits, f_bits, pixels):
    """s at the given image pixels m = (m1, m2) from the integer coefficients
    c_int (c 2^F), whose element [i, j] sits at image point (j - ox, i - oy),
    origin = (ox, oy) (c = 0 elsewhere).  Each pixel integrates its own
    window (the lattice box its mesh reads), as oracle.paper does."""
    c_int = np.asarray(c_int, dtype=object)
    ox, oy = origin
    meth = Method(r, n1, q_bits)
    S_out, s_out = [], []
    for (m1, m2) in pixels:
        Cm = C[m2, m1]
        left, right, below, above = meth.reach(Cm)
        x0, x1, y0, y1 = m1 - left, m1 + right + 1, m2 - below, m2 + above + 1
        local = np.zeros((y1 - y0, x1 - x0), dtype=object)
        local[:, :] = 0
        for yy in range(y0, y1):
            i = yy + oy
            if 0 <= i < c_int.shape[0]:
                for xx in range(x0, x1):
                    jx = xx + ox
                    if 0 <= jx < c_int.shape[1]:
                        local[yy - y0, xx - x0] = c_int[i, jx]
        g = integrate(local, meth.r, 0, x1 - x0, 0, y1 - y0)

        def gget(k1, k2, g=g, x0=x0, y0=y0):
            return g[k2 - y0, k1 - x0]

        Sm = meth.numerator(gget, m1, m2, Cm)
        S_out.append(Sm)
        s_out.append(Fr(Sm) / meth.denominator(Cm, f_bits))
    return S_out, s_out


def filter_image(c_int, origin, C, r, n1, q_bits, f_bits):
    """Every pixel of an H x W image (C: H x W x 4 integer steps), with one
    lattice box for all of them: returns (S, s) as lists in row-major order."""
    c_int = np.asarray(c_int, dtype=object)
    ox, oy = origin
    C = np.asarray(C)
    H, W = C.shape[:2]
    meth = Method(r, n1, q_bits)
    cm = [int(C[..., k].max()) for k in range(4)]
    left, right, below, above = meth.reach(cm)
    x0, x1 = -left - ox, W + right + c_int.shape[1]
    y0, y1 = -below - oy, H + above + c_int.shape[0]
    # c on the box, in box coordinates: element [i, j] of c_int is image point (j - ox, i - oy)
    local = np.zeros((y1 - y0, x1 - x0), dtype=object)
    local[:, :] = 0
    local[-oy - y0:-oy - y0 + c_int.shape[0], -ox - x0:-ox - x0 + c_int.shape[1]] = c_int
    g = integrate(local, meth.r, 0, x1 - x0, 0, y1 - y0)

    def gget(k1, k2):
        return g[k2 - y0, k1 - x0]

    S_out, s_out = [], []
    for m2 in range(H):
        for m1 in range(W):
            Sm = meth.numerator(gget, m1, m2, C[m2, m1])
            S_out.append(Sm)
            s_out.append(Fr(Sm) / meth.denominator(C[m2, m1], f_bits))
    return S_out, s_out


def filter_direct(c_int, origin, C, r, n1, q_bits, f_bits, pixels):
    """s[m] = sum_k c[k] B(m - k) from the definition (exact Fractions)."""
    c_int = np.asarray(c_int, dtype=object)
    ox, oy = origin
    out = []
    kernels = {}
    for (m1, m2) in pixels:
        key = tuple(int(v) for v in C[m2, m1])
        c = [Fr(v, 1 << q_bits) for v in key]
        kb = kernels.get(key)
        if kb is None:
            kb = kernels[key] = kernel_direct(c, r, n1)
        # the centred kernel vanishes beyond half the sum of |direction components|
        hx = sum(abs(d[0]) * k for d, k in zip(kb.dirs, kb.counts)) / 2
        hy = sum(abs(d[1]) * k for d, k in zip(kb.dirs, kb.counts)) / 2
        acc = Fr(0)
        for i in range(c_int.shape[0]):
            if abs(m2 - (i - oy)) >= hy:
                continue
            for j in range(c_int.shape[1]):
                if abs(m1 - (j - ox)) >= hx:
                    continue
                v = int(c_int[i, j])
                if v:
                    acc += v * kb.centred_value(m1 - (j - ox), m2 - (i - oy))
        out.append(acc / (1 << f_bits))
    return out


# ------------------------------------------------------------- the model

def prefilter2d(f_int, n1, bits=200):
    """c = f * (b^{n1} (x) b^{n1})^-1, separably (rows, then columns), with
    f 2^F = f_int zero outside the image, each pass the 1-D inverse filter
    of oracle.line1d; c_q = rint(c 2^F), ties to even.  Returns (c_q, origin):
    c_q[i, j] sits at image point (j - T, i - T) with T the tail kept on each
    side (c_q = 0 beyond it)."""
    f_int = np.asarray(f_int)
    H, W = f_int.shape
    rows = []
    first = None
    for y in range(H):
        k0, cs = line1d.prefilter([int(v) for v in f_int[y]], n1, bits)
        first = k0
        rows.append(cs)
    wide = len(rows[0])
    inter = np.array(rows, dtype=object)           # H x wide, scale 2^(F + bits)
    cols = []
    for x in range(wide):
        k0y, cs = line1d.prefilter([int(v) for v in inter[:, x]], n1, bits)
        cols.append(cs)
    full = np.array(cols, dtype=object).T           # (H + 2E) x wide, scale 2^(F + 2 bits)
    q = np.vectorize(lambda v: line1d.rint_shift(int(v), 2 * bits), otypes=[object])(full)
    # trim all-zero border rows and columns symmetrically to the tail T
    E = -first
    nz = np.argwhere(q != 0)
    if nz.size == 0:
        T = 0
    else:
        T = max(E - int(nz[:, 0].min()), int(nz[:, 0].max()) - (H - 1 + E),
                E - int(nz[:, 1].min()), int(nz[:, 1].max()) - (W - 1 + E), 0)
    out = q[E - T:E + H + T, E - T:E + W + T]
    return out, (T, T)
