"""Per-pixel scale readings (test infrastructure only; see package header).

The paper's scale vector a = (a1, a2, a3, a4) (Sec. 7) measures each
directional box in Euclidean length along r_{theta_k}.  On the lattice the k-th
box is the segment c_k v_k with v = (1,0), (1,1), (0,1), (-1,1), so
c1 = a1, c3 = a3 and c_k = a_k / sqrt2 for the diagonals -- the paper's own
a'_j = a_j / sqrt2 of Table "Mesh Vertices".

Quantisation (a reading: the paper takes real scales): C_k = rint(c_k 2^Q) with
ties to even; both the oracle and the CUDA path consume these integers, so the
problem is defined exactly.  Every step is IEEE binary64 with no fused
multiply-add, so both sides reach the same integers.

Ellipse to scales (a reading: Sec. 6 assumes a pre-assigned scale map and
Sec. 8 defers its computation).  The kernel with steps c_k, each n times, has
covariance sum_k (n c_k^2 / 12) v_k v_k^T.  Matching it to the ellipse
covariance C = R diag(sigma^2 e, sigma^2 / e) R^T with u_k = n c_k^2 / 12 gives

    u1 + u2 + u4 = C11,   u2 + u3 + u4 = C22,   u2 - u4 = C12,

a one-parameter family u2,4 = t +- C12/2, u1 = C11 - 2t, u3 = C22 - 2t,
t in [|C12|/2, min(C11, C22)/2].  The midpoint t is taken; for C = sigma^2 I it
gives every paper scale a_k = sigma sqrt(6/n), which for n = 1 is Theorem
(convergence) of Sec. 4 with N = 4 (a_k = sigma sqrt(24/N)).  When the family is
empty (|C12| > min(C11, C22)) t = min(C11, C22)/2 and negative u are set to 0.
Then c_k = clamp(sqrt(12 u_k / n), 1, cmax).
"""
import numpy as np

INV_SQRT2 = 0.7071067811865476


def c_from_a4(a):
    """Paper scales (..., 4) -> lattice steps c (float64)."""
    a = np.asarray(a, dtype=np.float64)
    c = a.copy()
    c[..., 1] = a[..., 1] * INV_SQRT2
    c[..., 3] = a[..., 3] * INV_SQRT2
    return c


def c_from_ellipse_scalar(sigma, elong, ct, st, n, cmax):
    """The moment rule for one pixel; plain Python floats (binary64, no FMA)."""
    s2 = sigma * sigma
    ev1 = s2 * elong
    ev2 = s2 / elong
    cc = ct * ct
    ss = st * st
    cs = ct * st
    c11 = ev1 * cc + ev2 * ss
    c22 = ev1 * ss + ev2 * cc
    c12 = (ev1 - ev2) * cs
    a12 = abs(c12)
    mn = c11 if c11 < c22 else c22
    if a12 <= mn:
        t = 0.25 * (a12 + mn)
    else:
        t = 0.5 * mn
    h = 0.5 * c12
    u = [c11 - 2.0 * t, t + h, c22 - 2.0 * t, t - h]
    out = []
    for uk in u:
        if uk < 0.0:
            uk = 0.0
        ck = float(np.sqrt((12.0 * uk) / n))
        if ck < 1.0:
            ck = 1.0
        if ck > cmax:
            ck = cmax
        out.append(ck)
    return out


def c_from_ellipse(field, n, cmax):
    """field (..., 4) = (sigma, elongation, cos theta, sin theta) -> c (..., 4)."""
    f = np.asarray(field, dtype=np.float64)
    flat = f.reshape(-1, 4)
    out = np.array([c_from_ellipse_scalar(*map(float, r), n, float(cmax)) for r in flat])
    return out.reshape(f.shape[:-1] + (4,))


def quantise(c, q_bits):
    """C_k = rint(c_k 2^Q), ties to even (int64)."""
    c = np.asarray(c, dtype=np.float64)
    return np.rint(c * float(1 << q_bits)).astype(np.int64)


def scales_to_C(kind, field, n, q_bits, cmax):
    """kind in {'c4', 'a4', 'ellipse'}: the three scale inputs the filter takes."""
    field = np.asarray(field)
    if kind == 'c4':
        c = np.asarray(field, dtype=np.float64)
    elif kind == 'a4':
        c = c_from_a4(np.asarray(field, dtype=np.float64))
    elif kind == 'ellipse':
        c = c_from_ellipse(field.astype(np.float64), n, cmax)
    else:
        raise ValueError(kind)
    return quantise(c, q_bits)
