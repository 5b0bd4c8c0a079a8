"""The filter from its definition (test infrastructure only; see package header).

Sec. 6: s[m] = <f, beta^N_{a(m)}(. - m)> for the continuous model
f(x) = sum_k c[k] phi(x - k); Sec. 7 (1) takes phi = delta, so c = f and

    s[m] = sum_j f[j] beta^4_{a(m)}(j - m) = sum_j f[j] B_{c(m)}(m - j)

(the box spline is centred, hence symmetric).  B_c is the box spline with
direction vectors c_k v_k, each n times (Sec. 4 Eq. (def), N = 4), evaluated
exactly by de Boor's recurrence.  A plain double loop; tiny images only.
"""
from fractions import Fraction as Fr

import numpy as np

from .boxspline import kernel_B


def filter_direct(f_int, C, n, q_bits, f_bits=0):
    """Exact s for every pixel (list of Fractions, row-major) and its binary64
    rounding.  C: integer steps (H, W, 4) in units of 2^-Q."""
    f_int = np.asarray(f_int)
    C = np.asarray(C)
    H, W = f_int.shape
    kernels = {}
    exact = np.empty((H, W), dtype=object)
    for m2 in range(H):
        for m1 in range(W):
            key = tuple(int(v) for v in C[m2, m1])
            kb = kernels.get(key)
            if kb is None:
                kb = kernel_B([Fr(v, 1 << q_bits) for v in key], n)
                kernels[key] = kb
            c = [Fr(v, 1 << q_bits) for v in key]
            ex = Fr(n, 2) * (c[0] + c[1] + c[3])
            ey = Fr(n, 2) * (c[1] + c[2] + c[3])
            acc = Fr(0)
            for j2 in range(max(0, int(m2 - ey) - 1), min(H, int(m2 + ey) + 2)):
                for j1 in range(max(0, int(m1 - ex) - 1), min(W, int(m1 + ex) + 2)):
                    fv = int(f_int[j2, j1])
                    if fv:
                        acc += fv * kb.centred_value(m1 - j1, m2 - j2)
            exact[m2, m1] = acc / (1 << f_bits)
    s = np.vectorize(float, otypes=[np.float64])(exact)
    return exact, s
