"""The paper's fast algorithm in exact integer arithmetic (test infrastructure
only; see package header).

Sec. 7 of the paper, restated in lattice units (see ``oracle.scales``):

(1) Non-adaptive step, Eq. (RS) with phi = delta (so c = f).  Four recursions,
    in the paper's order:
        F0[k1,k2]    = f[k1,k2]  + F0[k1-1,k2]          (0)
        Fq[k1,k2]    = F0[k1,k2] + Fq[k1-1,k2-1]        (pi/4)
        Fh[k1,k2]    = Fq[k1,k2] + Fh[k1,k2-1]          (pi/2)
        g[k1,k2]     = Fh[k1,k2] + g[k1+1,k2-1]         (3pi/4)
    The paper's diagonal recursions carry a factor sqrt2 each; they are folded
    out here (unit weights), so the paper's g_b equals 2 g (2^n g at order n),
    and its alpha = (a1 a2 a3 a4)^-1 = (2 c1 c2 c3 c4)^-1.  Order n applies each
    recursion n times (the n-fold running sum Delta_b^{-n} of Sec. 2).

(2) Adaptive step, Eq. (final_eqn):
        s[m] = alpha sum_i h[i] g_I(m + tau - x_i)
    with the vertices x_i = sum_k eps_k c_k v_k, eps in {0,1}^4, signs
    (-1)^{|eps|} (Table "Mesh Vertices"), tau from Sec. 7, and g_I the ZP
    interpolation of g.  At order n the vertices are sum_k j_k c_k v_k,
    j in {0..n}^4, with weights prod_k (-1)^{j_k} binom(n, j_k) (the FD filter
    d^n_a of Eq. (FD) along each direction), tau_n = n tau (from the link
    Eq. (link), tau = (a-1)(n+1)/2 in 1-D), and g_I uses ZP^{*n}.

Exactness: with f an integer image (or f 2^F integer) and C_k = c_k 2^Q
integers, every tap lies on the 2^-P grid (P = Q for even n, Q+1 for odd n) and
D ZP^{*n} is integral there, so the numerator

    S[m] = D sum_j w_j g_I(y_j)

is an integer and s[m] = S[m] 2^{4Qn} / (D (prod_k C_k)^n 2^F), a rational
number rounded once to binary64.
"""
from fractions import Fraction as Fr
from itertools import product
from math import comb, ceil

import numpy as np

from .boxspline import LATTICE_DIRS, ZPIntegerWeights


def p_bits(n, q_bits):
    """Grid of the tap positions: tau_n = (n/2) sum (c_k - 1) v_k lies on the
    2^-Q grid for even n and on the 2^-(Q+1) grid for odd n."""
    return q_bits if n % 2 == 0 else q_bits + 1


def mesh_vertices(n):
    """[(j, weight)] for j in {0..n}^4: vertex sum_k j_k c_k v_k with weight
    prod_k (-1)^{j_k} binom(n, j_k).  For n = 1 these are the 16 vertices of
    Table "Mesh Vertices" with h[i] / alpha = (-1)^{i+1}."""
    out = []
    for j in product(range(n + 1), repeat=4):
        w = 1
        for jk in j:
            w *= (-1) ** jk * comb(n, jk)
        out.append((j, w))
    return out


def tau(c, n):
    """Shift vector of Sec. 7 at order n, lattice units: (n/2) sum_k (c_k - 1) v_k."""
    tx = Fr(n, 2) * sum((Fr(ck) - 1) * v[0] for ck, v in zip(c, LATTICE_DIRS))
    ty = Fr(n, 2) * sum((Fr(ck) - 1) * v[1] for ck, v in zip(c, LATTICE_DIRS))
    return tx, ty


def reach(c, n):
    """Lattice margins (left, right, below, above) around a pixel that its
    mesh reads: taps span m + tau - sum_k j_k c_k v_k, the ZP^{*n} stencil adds
    3n/2 on each side.  With E_x = (n/2)(c1+c2+c4), E_y = (n/2)(c2+c3+c4):
    x in [m1 - E_x - 2n, m1 + E_x + n], y in [m2 - E_y - 3n, m2 + E_y]."""
    ex = Fr(n, 2) * (Fr(c[0]) + Fr(c[1]) + Fr(c[3]))
    ey = Fr(n, 2) * (Fr(c[1]) + Fr(c[2]) + Fr(c[3]))
    return ceil(ex + 2 * n), ceil(ex + n), ceil(ey + 3 * n), ceil(ey)


# ------------------------------------------------------------ integration

def integrate(f_int, n, x0, x1, y0, y1, exact=True):
    """g = the paper's four recursions (unit weights), each applied n times,
    on the lattice box [x0, x1) x [y0, y1) in image coordinates, with f = 0
    outside the image (zero padding).  Requires x0 <= 0, y0 <= 0.

    Rows are produced in increasing k2; every recursion reads only the current
    and the previous row, so each stage keeps its previous row.  The 3pi/4
    recursion reads g[k1+1, k2-1]: to be exact on [x0, x1) every row is carried
    out to x1 + (y1 - y0), beyond which the values never reach the box
    (the anti-diagonal through (x, y) meets row y0 at x + y - y0 < x1 + y1 - y0).

    exact=True: Python integers (object arrays).  exact=False: numpy uint64,
    i.e. g mod 2^64 (two's complement wrap-around; exact modulo 2^64).
    """
    f_int = np.asarray(f_int)
    H, W = f_int.shape
    assert x0 <= 0 and y0 <= 0 and x1 >= W and y1 >= H
    rows, cols = y1 - y0, x1 - x0
    width = cols + rows
    dt = object if exact else np.uint64

    def zeros():
        z = np.zeros(width, dtype=dt)
        if exact:
            z[:] = 0
        return z

    prev = [zeros() for _ in range(3 * n)]
    out = np.zeros((rows, cols), dtype=dt)
    for yi in range(rows):
        y = y0 + yi
        row = zeros()
        if 0 <= y < H:
            src = f_int[y]
            if exact:
                row[-x0:-x0 + W] = [int(v) for v in src]
            else:
                row[-x0:-x0 + W] = src.astype(np.int64).astype(np.uint64)
        # F0: running sum along 0 (n times)
        for _ in range(n):
            row = np.cumsum(row, dtype=dt)
        # F_{pi/4}: cur[x] = in[x] + prev[x-1]
        for s in range(n):
            cur = row.copy()
            cur[1:] += prev[s][:-1]
            prev[s] = cur
            row = cur
        # F_{pi/2}: cur[x] = in[x] + prev[x]
        for s in range(n, 2 * n):
            cur = row + prev[s]
            prev[s] = cur
            row = cur
        # g: cur[x] = in[x] + prev[x+1]
        for s in range(2 * n, 3 * n):
            cur = row.copy()
            cur[:-1] += prev[s][1:]
            prev[s] = cur
            row = cur
        out[yi] = row[:cols]
    return out


def domain_for(shape, c_max4, n):
    """Lattice box [x0, x1) x [y0, y1) that holds every mesh read of every
    pixel of an H x W image whose steps are bounded by c_max4 (per direction)."""
    H, W = shape
    left, right, below, above = reach(c_max4, n)
    return -left, W + right, -below, H + above


# ------------------------------------------------------------------- mesh

class Mesh:
    """The adaptive step of Eq. (final_eqn) at order n, exact."""

    def __init__(self, n, q_bits):
        self.n, self.Q = n, q_bits
        self.P = p_bits(n, q_bits)
        self.zw = ZPIntegerWeights(n, self.P)
        self.D = self.zw.D
        self.verts = mesh_vertices(n)

    def taps(self, m1, m2, C):
        """[(w_j, Yx, Yy)]: tap positions y_j = m + tau - sum_k j_k c_k v_k in
        units of 2^-P (integers), c_k = C_k 2^-Q."""
        c = [Fr(int(ck), 1 << self.Q) for ck in C]
        tx, ty = tau(c, self.n)
        one = 1 << self.P
        out = []
        for j, w in self.verts:
            yx = m1 + tx - sum(jk * ck * v[0] for jk, ck, v in zip(j, c, LATTICE_DIRS))
            yy = m2 + ty - sum(jk * ck * v[1] for jk, ck, v in zip(j, c, LATTICE_DIRS))
            yx, yy = yx * one, yy * one
            assert yx.denominator == 1 and yy.denominator == 1
            out.append((w, int(yx), int(yy)))
        return out

    def numerator(self, gget, m1, m2, C):
        """S = D sum_j w_j g_I(y_j), with g_I(y) = sum_k g[k] ZP^{*n}(y - k);
        gget(k1, k2) returns the (integer) pre-integrated image."""
        zw, dmin, n3 = self.zw, self.zw.dmin, 3 * self.n
        S = 0
        for w, yx, yy in self.taps(m1, m2, C):
            px, rx = zw.split(yx)
            py, ry = zw.split(yy)
            wrow = zw.row(rx, ry)
            acc = 0
            for iy in range(n3):
                k2 = py + dmin + iy
                line = wrow[iy]
                for ix in range(n3):
                    wt = line[ix]
                    if wt:
                        acc += int(gget(px + dmin + ix, k2)) * wt
            S += w * acc
        return S

    def denominator(self, C, f_bits):
        """s = S / Den with Den = D (prod_k c_k)^n 2^F (exact rational)."""
        prod = Fr(1)
        for ck in C:
            prod *= Fr(int(ck), 1 << self.Q)
        return self.D * prod ** self.n * (1 << f_bits)


def _signed(v, bits):
    v = int(v) % (1 << bits)
    return v - (1 << bits) if v >= 1 << (bits - 1) else v


def filter_image(f_int, C, n, q_bits, f_bits=0, exact_g=True):
    """All pixels of a (small) image.  Returns (S, s): S the exact integer
    numerators (object array), s = S / Den rounded once to binary64."""
    f_int = np.asarray(f_int)
    C = np.asarray(C)
    H, W = f_int.shape
    cmax = [Fr(int(C[..., k].max()), 1 << q_bits) for k in range(4)]
    x0, x1, y0, y1 = domain_for((H, W), cmax, n)
    g = integrate(f_int, n, x0, x1, y0, y1, exact=exact_g)
    mesh = Mesh(n, q_bits)

    def gget(k1, k2):
        return g[k2 - y0, k1 - x0]

    S = np.empty((H, W), dtype=object)
    s = np.empty((H, W), dtype=np.float64)
    for m2 in range(H):
        for m1 in range(W):
            Sm = mesh.numerator(gget, m1, m2, C[m2, m1])
            if not exact_g:
                Sm = _signed(Sm, 64)
            S[m2, m1] = Sm
            s[m2, m1] = float(Fr(Sm) / mesh.denominator(C[m2, m1], f_bits))
    return S, s


def filter_pixels(f_int, C, n, q_bits, f_bits, pixels):
    """Selected pixels of a (large) image, exact.  Each pixel m uses its own
    window: the input restricted to the lattice box its mesh reads.  That box
    holds the support of the kernel B_c(m - .), so the result is unchanged (the
    filter is linear and the kernel has compact support)."""
    f_int = np.asarray(f_int)
    C = np.asarray(C)
    H, W = f_int.shape
    mesh = Mesh(n, q_bits)
    S_out, s_out = [], []
    for (m1, m2) in pixels:
        Cm = C[m2, m1]
        c = [Fr(int(v), 1 << q_bits) for v in Cm]
        left, right, below, above = reach(c, n)
        wx0, wx1, wy0, wy1 = m1 - left, m1 + right + 1, m2 - below, m2 + above + 1
        local = np.zeros((wy1 - wy0, wx1 - wx0), dtype=object)
        local[:, :] = 0
        lx0, ly0, lx1, ly1 = max(wx0, 0), max(wy0, 0), min(wx1, W), min(wy1, H)
        if lx1 > lx0 and ly1 > ly0:
            local[ly0 - wy0:ly1 - wy0, lx0 - wx0:lx1 - wx0] = f_int[ly0:ly1, lx0:lx1]
        g = integrate(local, n, 0, wx1 - wx0, 0, wy1 - wy0, exact=True)

        def gget(k1, k2, g=g, wx0=wx0, wy0=wy0):
            return g[k2 - wy0, k1 - wx0]

        Sm = mesh.numerator(gget, m1, m2, Cm)
        S_out.append(Sm)
        s_out.append(float(Fr(Sm) / mesh.denominator(Cm, f_bits)))
    return S_out, np.array(s_out)
