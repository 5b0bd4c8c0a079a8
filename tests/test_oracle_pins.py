"""Pins of the exact oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed table and shift vector, a closed-form polygon-area evaluation of the
four-direction box spline (n = 1), brute-force lattice path counts, moving
averages, exact spectral zeros, symmetries, and the direct definition of the
filter.  A plausible slip in the oracle (a dropped term, a wrong sign, a
transposed direction, a wrong shift) fails at least one of them.
"""
import math
import os
import random
from fractions import Fraction as Fr
from itertools import product

import numpy as np
import pytest

from oracle import boxspline as bs
from oracle import paper, direct, scales

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
V = ((1, 0), (1, 1), (0, 1), (-1, 1))


# ------------------------------------------------------------ helpers (test-side)

def _clip(poly, a, b, c):
    """Sutherland-Hodgman: keep the part of polygon ``poly`` with a x + b y <= c."""
    out = []
    for i in range(len(poly)):
        p, q = poly[i], poly[(i + 1) % len(poly)]
        fp, fq = a * p[0] + b * p[1] - c, a * q[0] + b * q[1] - c
        if fp <= 0:
            out.append(p)
        if (fp < 0 < fq) or (fq < 0 < fp):
            t = fp / (fp - fq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    return out


def _area(poly):
    s = Fr(0)
    for i in range(len(poly)):
        p, q = poly[i], poly[(i + 1) % len(poly)]
        s += p[0] * q[1] - q[0] * p[1]
    return abs(s) / 2


def box_spline_polygon(c, x, y):
    """n = 1 kernel B_c(x) = area(R1 cap (x + R2)) / (c1 c3 * 2 c2 c4), with
    R1 = [-c1/2, c1/2] x [-c3/2, c3/2] (axis boxes) and
    R2 = {|u + w| <= c2, |w - u| <= c4} (the two diagonal boxes); an
    independent closed form of Sec. 4 Eq. (def) for N = 4."""
    c1, c2, c3, c4 = (Fr(v) for v in c)
    x, y = Fr(x), Fr(y)
    poly = [(-c1 / 2, -c3 / 2), (c1 / 2, -c3 / 2), (c1 / 2, c3 / 2), (-c1 / 2, c3 / 2)]
    # (u, w) in x + R2  <=>  |(u - x) + (w - y)| <= c2 and |(w - y) - (u - x)| <= c4
    for a, b, cc in ((1, 1, c2 + x + y), (-1, -1, c2 - x - y),
                     (-1, 1, c4 + y - x), (1, -1, c4 - y + x)):
        poly = _clip(poly, a, b, cc)
        if not poly:
            return Fr(0)
    return _area(poly) / (c1 * c3 * 2 * c2 * c4)


def _eval_expr(expr, env):
    expr = expr.replace("-", "+-")
    tot = Fr(0)
    for tok in expr.split("+"):
        tok = tok.strip()
        if not tok:
            continue
        sign = -1 if tok.startswith("-") else 1
        tok = tok.lstrip("-")
        tot += sign * (Fr(0) if tok == "0" else env[tok])
    return tot


# --------------------------------------------------------------- mesh geometry

def test_mesh_vertices_match_paper_table():
    """Table "Mesh Vertices" and the weights h[i] = (-1)^(i+1) alpha of
    Eq. (final_eqn) are the oracle's n = 1 mesh (positions and signs)."""
    rows = []
    with open(os.path.join(GOLDEN, "mesh_vertices.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                i, ex, ey = line.split()
                rows.append((int(i), ex, ey))
    assert len(rows) == 16
    rnd = random.Random(5)
    for _ in range(5):
        c = [Fr(rnd.randint(1, 400), 37) for _ in range(4)]
        env = {"a1": c[0], "a2p": c[1], "a3": c[2], "a4p": c[3]}
        table = sorted(((_eval_expr(ex, env), _eval_expr(ey, env)), (-1) ** (i + 1))
                       for i, ex, ey in rows)
        ours = sorted(((sum(jk * ck * v[0] for jk, ck, v in zip(j, c, V)),
                        sum(jk * ck * v[1] for jk, ck, v in zip(j, c, V))), w)
                      for j, w in paper.mesh_vertices(1))
        assert table == ours


def test_shift_vector_matches_paper_formula():
    """tau of Sec. 7 (printed in the paper's a-scales, with sqrt2) equals the
    oracle's tau = (1/2) sum_k (c_k - 1) v_k with c2 = a2/sqrt2, c4 = a4/sqrt2."""
    lines = [l.split("=", 1)[1] for l in open(os.path.join(GOLDEN, "shift_vector.txt"))
             if l.startswith("tau")]
    rnd = random.Random(3)
    for _ in range(20):
        a = [rnd.uniform(1, 40) for _ in range(4)]
        env = {"a1": a[0], "a2": a[1], "a3": a[2], "a4": a[3], "sqrt2": math.sqrt(2)}
        t_paper = [eval(e, {}, env) for e in lines]
        c = [Fr(a[0]), Fr(a[1] / math.sqrt(2)), Fr(a[2]), Fr(a[3] / math.sqrt(2))]
        t_or = paper.tau(c, 1)
        assert abs(float(t_or[0]) - t_paper[0]) < 1e-12 * (1 + abs(t_paper[0]))
        assert abs(float(t_or[1]) - t_paper[1]) < 1e-12 * (1 + abs(t_paper[1]))


# ---------------------------------------------------------- box-spline values

def test_zp_values_match_polygon_area():
    """ZP element (n = 1, unit steps) from de Boor's recurrence equals the
    polygon-area closed form at integer, half-integer and random dyadic points;
    and the special values 1/2, 1/8, 0, 3/8."""
    assert bs.zp_value(1, 0, 0) == Fr(1, 2)
    assert bs.zp_value(1, 1, 0) == Fr(1, 8) == bs.zp_value(1, 0, -1)
    assert bs.zp_value(1, 1, 1) == 0
    assert bs.zp_value(1, Fr(1, 2), 0) == Fr(3, 8)
    rnd = random.Random(11)
    pts = [(Fr(i, 2), Fr(j, 2)) for i in range(-4, 5) for j in range(-4, 5)]
    pts += [(Fr(rnd.randint(-96, 96), 64), Fr(rnd.randint(-96, 96), 64)) for _ in range(300)]
    for x, y in pts:
        assert bs.zp_value(1, x, y) == box_spline_polygon((1, 1, 1, 1), x, y), (x, y)


def test_general_box_spline_matches_polygon_area():
    """de Boor point evaluation with directions c_k v_k (used by the direct
    filter) equals the polygon-area kernel for random dyadic steps (n = 1)."""
    rnd = random.Random(7)
    for _ in range(6):
        c = [Fr(rnd.randint(4, 40), 8) for _ in range(4)]
        kb = bs.kernel_B(c, 1)
        for _ in range(40):
            x, y = Fr(rnd.randint(-200, 200), 32), Fr(rnd.randint(-200, 200), 32)
            assert kb.centred_value(x, y) == box_spline_polygon(c, x, y)


@pytest.mark.parametrize("n", [1, 2])
def test_zp_partition_of_unity_and_symmetry(n):
    """sum_j ZP^{*n}(x - j) = 1 (integer directions); ZP^{*n} is invariant
    under x -> -x and under swapping the axes (dihedral symmetry of v1..v4)."""
    rnd = random.Random(n)
    for _ in range(20):
        x, y = Fr(rnd.randint(0, 255), 256), Fr(rnd.randint(0, 255), 256)
        tot = sum(bs.zp_value(n, x - i, y - j) for i in range(-2 * n, 2 * n + 1)
                  for j in range(-2 * n, 2 * n + 1))
        assert tot == 1
        a, b = Fr(rnd.randint(-400, 400), 128), Fr(rnd.randint(-400, 400), 128)
        v = bs.zp_value(n, a, b)
        assert v == bs.zp_value(n, -a, b) == bs.zp_value(n, b, a) == bs.zp_value(n, -b, -a)


@pytest.mark.slow
def test_zp3_partition_of_unity():
    rnd = random.Random(3)
    for _ in range(4):
        x, y = Fr(rnd.randint(0, 511), 512), Fr(rnd.randint(0, 511), 512)
        tot = sum(bs.zp_value(3, x - i, y - j) for i in range(-6, 7) for j in range(-6, 7))
        assert tot == 1


@pytest.mark.parametrize("n,P", [(1, 3), (2, 3)])
def test_integer_weight_rows_sum_to_denominator(n, P):
    """Every weight row D ZP^{*n}(r - d) is integral, non-negative and sums to
    D (partition of unity on the 2^-P grid)."""
    zw = bs.ZPIntegerWeights(n, P)
    for rx in range(1 << P):
        for ry in range(1 << P):
            row = zw.row(rx, ry)
            assert sum(map(sum, row)) == zw.D
            assert min(map(min, row)) >= 0


# ---------------------------------------------------------------- integration

def _path_count_g(f, n, x0, x1, y0, y1):
    """g[k] = sum_j f[j] N(k - j), N(d) = number of ways to write d as a sum of
    n copies of each of v1..v4 with non-negative integer multiples, counted
    with the multiplicities of the n-fold running sum (the filter u^4_b of
    Eq. (RS), unit weights)."""
    H, W = f.shape
    # 1-D n-fold running-sum filter: binom(t + n - 1, n - 1) at step t >= 0
    def u(t):
        return math.comb(t + n - 1, n - 1) if t >= 0 else 0
    out = np.zeros((y1 - y0, x1 - x0), dtype=object)
    out[:, :] = 0
    span = (y1 - y0) + (x1 - x0) + H + W
    for ky in range(y0, y1):
        for kx in range(x0, x1):
            tot = 0
            for jy in range(H):
                for jx in range(W):
                    if not f[jy, jx]:
                        continue
                    dx, dy = kx - jx, ky - jy
                    if dy < 0:
                        continue
                    # d = t1 v1 + t2 v2 + t3 v3 + t4 v4: choose t2, t4
                    cnt = 0
                    for t2 in range(0, dy + 1):
                        for t4 in range(0, dy - t2 + 1):
                            t3 = dy - t2 - t4
                            t1 = dx - t2 + t4
                            if t1 < 0:
                                continue
                            cnt += u(t1) * u(t2) * u(t3) * u(t4)
                    tot += f[jy, jx] * cnt
            out[ky - y0, kx - x0] = tot
    return out


@pytest.mark.parametrize("n", [1, 2])
def test_integrate_matches_path_counts(n):
    """The four recursions of Sec. 7 (1) equal the convolution with the
    four-direction running-sum filter u^4_b of Eq. (RS) (brute force)."""
    rng = np.random.default_rng(n)
    f = rng.integers(-5, 9, (3, 4))
    x0, x1, y0, y1 = -3, 7, -2, 6
    g = paper.integrate(f, n, x0, x1, y0, y1, exact=True)
    ref = _path_count_g(f, n, x0, x1, y0, y1)
    assert (g == ref).all()
    g64 = paper.integrate(f, n, x0, x1, y0, y1, exact=False)
    assert all(int(a) == int(b) % (1 << 64) for a, b in zip(g64.ravel(), ref.ravel()))


# ----------------------------------------------------------- filter invariants

def _const_C(H, W, C):
    return np.broadcast_to(np.array(C, dtype=np.int64), (H, W, 4)).copy()


def _interior(H, W, C, n, Q):
    c = [Fr(v, 1 << Q) for v in C]
    ex = math.ceil(Fr(n, 2) * (c[0] + c[1] + c[3]))
    ey = math.ceil(Fr(n, 2) * (c[1] + c[2] + c[3]))
    return [(x, y) for y in range(ey, H - ey) for x in range(ex, W - ex)]


def test_zp_special_case_is_closed_form_stencil():
    """n = 1, a = b (c = 1): the filter is the ZP element itself, i.e. the
    3x3 stencil [0 1/8 0; 1/8 1/2 1/8; 0 1/8 0] (Sec. 7)."""
    rng = np.random.default_rng(0)
    f = rng.integers(0, 256, (9, 11))
    Q = 3
    C = _const_C(9, 11, [1 << Q] * 4)
    S, s = paper.filter_image(f, C, 1, Q)
    fp = np.pad(f.astype(object), 1)
    ref = (Fr(1, 2) * fp[1:-1, 1:-1] + Fr(1, 8) * (fp[:-2, 1:-1] + fp[2:, 1:-1]
                                                    + fp[1:-1, :-2] + fp[1:-1, 2:]))
    mesh = paper.Mesh(1, Q)
    for y in range(9):
        for x in range(11):
            assert Fr(S[y, x]) / mesh.denominator(C[y, x], 0) == ref[y, x]


@pytest.mark.parametrize("n,C", [(1, [24, 13, 16, 29]), (1, [19, 8, 27, 8]), (2, [16, 11, 8, 13])])
def test_partition_of_unity(n, C):
    """Constant image: s = const exactly in the interior when c1, c3 are
    integers or when c2, c4 are integers (the lattice sums of the axis, resp.
    diagonal, boxes are 1); Q = 3 here, so C = 8 k is an integer step."""
    Q = 3
    H, W = 20, 22
    f = np.full((H, W), 7)
    S, s = paper.filter_image(f, _const_C(H, W, C), n, Q)
    for x, y in _interior(H, W, C, n, Q):
        assert s[y, x] == 7.0


def test_constant_image_generic_steps_is_lattice_sum():
    """Generic steps: s = 7 * sum_i B_c(i) at every interior pixel (the
    projection of Sec. 6 has no normalisation), with sum_i B_c(i) from the
    polygon closed form."""
    Q = 3
    C = [13, 11, 10, 9]
    c = [Fr(v, 8) for v in C]
    H, W = 18, 18
    S, s = paper.filter_image(np.full((H, W), 7), _const_C(H, W, C), 1, Q)
    kappa = sum(box_spline_polygon(c, i, j) for i in range(-6, 7) for j in range(-6, 7))
    mesh = paper.Mesh(1, Q)
    for x, y in _interior(H, W, C, 1, Q):
        assert Fr(S[y, x]) / mesh.denominator(C, 0) == 7 * kappa
    assert kappa != 1


@pytest.mark.parametrize("n", [1, 2])
def test_linear_reproduction(n):
    """f = 3 k1 - 2 k2 + 5 is reproduced exactly in the interior (symmetric
    kernel, unit lattice sum) -- pins the sign and size of tau."""
    Q = 2
    C = [8, 6, 4, 5] if n == 1 else [4, 7, 8, 5]
    H, W = 18, 20
    yy, xx = np.mgrid[0:H, 0:W]
    f = 3 * xx - 2 * yy + 5
    S, s = paper.filter_image(f, _const_C(H, W, C), n, Q)
    for x, y in _interior(H, W, C, n, Q):
        assert s[y, x] == f[y, x]


def _moving_sums(f, n, steps, pad):
    """n-fold backward moving sums of integer lengths steps[k] along v_k."""
    H, W = f.shape
    h = np.zeros((H + 2 * pad, W + 2 * pad), dtype=object)
    h[:, :] = 0
    h[pad:pad + H, pad:pad + W] = f
    for k, (vx, vy) in enumerate(V):
        for _ in range(n):
            acc = np.zeros_like(h)
            acc[:, :] = 0
            for i in range(steps[k]):
                sh = np.zeros_like(h)
                sh[:, :] = 0
                dx, dy = i * vx, i * vy
                ys, xs = slice(max(dy, 0), h.shape[0]), slice(max(dx, 0), h.shape[1] + min(dx, 0))
                ysrc = slice(0, h.shape[0] - max(dy, 0))
                xsrc = slice(max(-dx, 0), h.shape[1] - max(dx, 0))
                sh[ys, xs] = h[ysrc, xsrc]
                acc = acc + sh
            h = acc
    return h


@pytest.mark.parametrize("n,steps", [(1, [3, 2, 4, 1]), (2, [2, 1, 3, 2])])
def test_integer_steps_equal_moving_averages(n, steps):
    """Integer steps c_k: seg_{c v} = seg_v * (average of c unit shifts), so
    s[m] = (prod c_k)^-n sum_l h[l] ZP^{*n}(m + tau - l) with h the n-fold
    backward moving sums of length c_k along each v_k -- no running sums."""
    Q = 1
    rng = np.random.default_rng(4 + n)
    H, W = 9, 10
    f = rng.integers(0, 50, (H, W))
    C = [s * 2 for s in steps]
    S, s = paper.filter_image(f, _const_C(H, W, C), n, Q)
    pad = 12
    h = _moving_sums(f, n, steps, pad)
    tx, ty = paper.tau([Fr(v) for v in steps], n)
    prod = math.prod(steps) ** n
    mesh = paper.Mesh(n, Q)
    for y in range(H):
        for x in range(W):
            ref = Fr(0)
            for ly in range(h.shape[0]):
                for lx in range(h.shape[1]):
                    if h[ly, lx]:
                        ref += h[ly, lx] * bs.zp_value(n, x + tx - (lx - pad), y + ty - (ly - pad))
            assert Fr(S[y, x]) / mesh.denominator(C, 0) == ref / prod


@pytest.mark.parametrize("n,C,kind", [(1, [4, 7, 5, 9], "x"), (1, [7, 4, 9, 5], "diag"),
                                      (1, [5, 7, 4, 3], "y"), (1, [6, 3, 5, 4], "anti"),
                                      (2, [4, 3, 5, 6], "x")])
def test_spectral_zeros(n, C, kind):
    """The kernel's spectrum is prod_k sinc^n(c_k v_k . w / 2) (Sec. 4
    Eq. (def)); sampled on the lattice it still vanishes at v_k . w = 2 pi / c_k
    for integer c_k (every alias term vanishes).  With c_k = 2 (Q = 1, C_k = 4)
    along the chosen direction the integer test patterns below are filtered to 0
    in the interior."""
    Q = 1
    H, W = 20, 22
    yy, xx = np.mgrid[0:H, 0:W]
    if kind == "x":
        f = (-1) ** xx                      # w = (pi, 0): w.v1 = pi = 2pi/2
    elif kind == "y":
        f = (-1) ** yy                      # w = (0, pi)
    elif kind == "diag":
        f = np.rint(np.cos(np.pi * (xx + yy) / 2)).astype(int)   # w.v2 = pi
    else:
        f = np.rint(np.cos(np.pi * (yy - xx) / 2)).astype(int)   # w.v4 = pi
    S, s = paper.filter_image(f, _const_C(H, W, C), n, Q)
    for x, y in _interior(H, W, C, n, Q):
        assert S[y, x] == 0


def test_symmetries():
    """Transposing the image swaps c1 and c3; mirroring k1 swaps c2 and c4
    (v2 = (1,1) mirrors to (-1,1) = v4).  Exact equality, all pixels."""
    rng = np.random.default_rng(8)
    H, W = 8, 9
    Q = 2
    f = rng.integers(0, 100, (H, W))
    C = rng.integers(3, 13, (H, W, 4))
    S, s = paper.filter_image(f, C, 1, Q)
    Ct = C.transpose(1, 0, 2)[..., [2, 1, 0, 3]]
    St, st = paper.filter_image(f.T, Ct, 1, Q)
    assert (st == s.T).all()
    Cm = C[:, ::-1][..., [0, 3, 2, 1]]
    Sm, sm = paper.filter_image(f[:, ::-1], Cm, 1, Q)
    assert (sm == s[:, ::-1]).all()


# ------------------------------------------------------------ brute force

def test_paper_equals_direct_definition_n1():
    """The algorithm of Sec. 7 (global running sums + 16-vertex mesh + ZP
    interpolation) equals s[m] = sum_j f[j] B_c(m - j) (Sec. 6, phi = delta)
    exactly at every pixel, borders included; per-pixel random steps."""
    rng = np.random.default_rng(21)
    H, W = 7, 8
    Q = 2
    f = rng.integers(0, 256, (H, W))
    C = rng.integers(2, 14, (H, W, 4))
    S, s = paper.filter_image(f, C, 1, Q)
    exact, sd = direct.filter_direct(f, C, 1, Q)
    mesh = paper.Mesh(1, Q)
    for y in range(H):
        for x in range(W):
            assert Fr(S[y, x]) / mesh.denominator(C[y, x], 0) == exact[y, x]


def test_paper_equals_direct_definition_n2():
    """Order 2 (the n-fold reading of the paper): algorithm == definition
    exactly; a few distinct scale vectors spread over the image."""
    rng = np.random.default_rng(22)
    H, W = 6, 7
    Q = 1
    f = rng.integers(0, 256, (H, W))
    choices = np.array([[2, 3, 2, 2], [3, 2, 2, 3]])
    C = choices[rng.integers(0, 2, (H, W))]
    S, s = paper.filter_image(f, C, 2, Q)
    exact, sd = direct.filter_direct(f, C, 2, Q)
    mesh = paper.Mesh(2, Q)
    for y in range(H):
        for x in range(W):
            assert Fr(S[y, x]) / mesh.denominator(C[y, x], 0) == exact[y, x]


@pytest.mark.slow
def test_paper_equals_direct_definition_n3():
    """Order 3: algorithm == definition exactly at every pixel of a tiny image,
    borders included, two scale vectors spread over it (the n-fold reading:
    256 vertices, weights prod (-1)^j binom(3, j), ZP^{*3} interpolation)."""
    rng = np.random.default_rng(31)
    H, W = 5, 6
    Q = 1
    f = rng.integers(0, 256, (H, W))
    choices = np.array([[2, 3, 2, 2], [3, 2, 2, 3]])
    C = choices[rng.integers(0, 2, (H, W))]
    S, s = paper.filter_image(f, C, 3, Q)
    exact, sd = direct.filter_direct(f, C, 3, Q)
    mesh = paper.Mesh(3, Q)
    for y in range(H):
        for x in range(W):
            assert Fr(S[y, x]) / mesh.denominator(C[y, x], 0) == exact[y, x]


def test_windowed_pixels_equal_global():
    """Per-pixel windows (used at large sizes) give the same exact numerators."""
    rng = np.random.default_rng(23)
    H, W = 10, 12
    Q = 3
    f = rng.integers(0, 256, (H, W))
    C = rng.integers(8, 40, (H, W, 4))
    for n in (1, 2):
        S, s = paper.filter_image(f, C, n, Q)
        pix = [(0, 0), (W - 1, H - 1), (5, 4), (11, 0), (0, 9)]
        Sp, sp = paper.filter_pixels(f, C, n, Q, 0, pix)
        assert [S[y, x] for x, y in pix] == Sp


def test_mod64_integration_gives_same_numerator():
    """g mod 2^64 (wrap-around) yields the same numerator modulo 2^64."""
    rng = np.random.default_rng(24)
    H, W = 8, 9
    f = rng.integers(0, 256, (H, W))
    C = rng.integers(8, 40, (H, W, 4))
    S, _ = paper.filter_image(f, C, 1, 3, exact_g=True)
    S64, _ = paper.filter_image(f, C, 1, 3, exact_g=False)
    assert all(int(a) == int(b) for a, b in zip(S.ravel(), S64.ravel()))


# ----------------------------------------------------------------- scales

def test_ellipse_rule_isotropic_is_convergence_theorem():
    """sigma^2 I gives every paper scale a_k = sigma sqrt(6/n); for n = 1 that
    is Theorem (convergence), a_k = sigma sqrt(24/N) with N = 4."""
    for n in (1, 2, 3):
        for sigma in (1.5, 3.0, 10.0):
            c = scales.c_from_ellipse_scalar(sigma, 1.0, 1.0, 0.0, n, 1e9)
            a = [c[0], c[1] * math.sqrt(2), c[2], c[3] * math.sqrt(2)]
            for ak in a:
                assert abs(ak - sigma * math.sqrt(6.0 / n)) < 1e-12 * sigma


def test_ellipse_rule_matches_covariance():
    """Feasible, unclamped ellipses: sum_k (n c_k^2 / 12) v_k v_k^T equals
    R diag(sigma^2 e, sigma^2 / e) R^T."""
    rnd = random.Random(9)
    for _ in range(200):
        n = rnd.randint(1, 3)
        s, e, th = rnd.uniform(2, 20), rnd.uniform(1, 2.5), rnd.uniform(0, math.pi)
        ct, st = math.cos(th), math.sin(th)
        c = scales.c_from_ellipse_scalar(s, e, ct, st, n, 1e9)
        cov = np.zeros((2, 2))
        for ck, v in zip(c, V):
            cov += n * ck * ck / 12.0 * np.outer(v, v)
        R = np.array([[ct, -st], [st, ct]])
        ref = R @ np.diag([s * s * e, s * s / e]) @ R.T
        if min(c) > 1.0:
            assert np.allclose(cov, ref, rtol=1e-10, atol=1e-9)


# Ellipses the four directions cannot represent (|C12| > min(C11, C22)): the
# rule takes t = min(C11, C22) / 2 and sets negative u to 0.  Worked by hand
# for sigma = 2, elongation 4 (eigenvalues 16 and 1) and the unit axis
# (0.6, 0.8) or its reflections: cc = 0.36, ss = 0.64, cs = +-0.48, so
# {C11, C22} = {6.4, 10.6}, |C12| = 7.2 > 6.4, t = 3.2, h = C12 / 2 = +-3.6 and
# u = (C11 - 2t, t + h, C22 - 2t, t - h); every u <= 0 gives the clamp c = 1,
# the others c = sqrt(12 u / n).
_INFEASIBLE = [
    # (cos, sin, u1, u2, u3, u4) before the clamp
    (0.6, 0.8, 0.0, 6.8, 4.2, -0.4),
    (0.8, 0.6, 4.2, 6.8, 0.0, -0.4),
    (-0.6, 0.8, 0.0, -0.4, 4.2, 6.8),
]


@pytest.mark.parametrize("case", _INFEASIBLE)
@pytest.mark.parametrize("n", [1, 2, 3])
def test_ellipse_rule_infeasible_branch_by_hand(case, n):
    ct, st, *u = case
    c = scales.c_from_ellipse_scalar(2.0, 4.0, ct, st, n, 1e9)
    want = [1.0 if uk <= 0 else math.sqrt(12.0 * uk / n) for uk in u]
    assert np.allclose(c, want, rtol=1e-12, atol=0)
    # the hand values solve the moment equations exactly before the clamp
    C11 = 16 * ct * ct + st * st
    C22 = 16 * st * st + ct * ct
    C12 = 15 * ct * st
    assert abs(u[0] + u[1] + u[3] - C11) < 1e-12 and abs(u[1] + u[2] + u[3] - C22) < 1e-12
    assert abs(u[1] - u[3] - C12) < 1e-12
    # on the kernel's covariance the clamps show up only as the added
    # (n c^2 / 12) v v^T of the directions that were clamped
    cov = np.zeros((2, 2))
    for ck, v in zip(c, V):
        cov += n * ck * ck / 12.0 * np.outer(v, v)
    ref = np.array([[C11, C12], [C12, C22]])
    for uk, ck, v in zip(u, c, V):
        if uk <= 0:
            ref += (n * ck * ck / 12.0 - uk) * np.outer(v, v)
    assert np.allclose(cov, ref, rtol=0, atol=1e-9)


def test_ellipse_rule_infeasible_branch_uses_the_smaller_diagonal():
    """A slip to max(C11, C22), or to the midpoint of an empty family, moves
    the steps: the hand case above gives these four steps only with the min."""
    c = scales.c_from_ellipse_scalar(2.0, 4.0, 0.6, 0.8, 1, 1e9)
    assert c[0] == 1.0 and c[3] == 1.0
    assert abs(c[1] * c[1] - 81.6) < 1e-9 and abs(c[2] * c[2] - 50.4) < 1e-9


def test_a4_steps_use_paper_diagonal_convention():
    """c = (a1, a2/sqrt2, a3, a4/sqrt2): Table "Mesh Vertices" uses a'_j = a_j/sqrt2."""
    c = scales.c_from_a4(np.array([2.0, 2.0 * math.sqrt(2), 3.0, math.sqrt(2)]))
    assert np.allclose(c, [2.0, 2.0, 3.0, 1.0], rtol=0, atol=1e-15)
    C = scales.quantise([0.5 / 256, 1.5 / 256, 2.5 / 256], 8)
    assert list(C) == [0, 2, 2]   # ties to even


@pytest.mark.slow
def test_order3_reproduces_linear_and_constant():
    """Order 3: linear reproduction (and so partition of unity) in the interior."""
    Q = 1
    C = [2, 3, 4, 5]
    H, W = 20, 17
    yy, xx = np.mgrid[0:H, 0:W]
    f = 2 * xx + yy + 1
    pix = _interior(H, W, C, 3, Q)[:6]
    Sp, sp = paper.filter_pixels(f, _const_C(H, W, C), 3, Q, 0, pix)
    assert list(sp) == [float(f[y, x]) for x, y in pix]
