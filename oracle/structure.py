"""Scale-map estimation for the adaptive filter, binary64.  TEST INFRASTRUCTURE
ONLY (see the package header).

The paper leaves the computation of the scale map to other work (Sec. 8); this
is the reading taken here, an edge-following ellipse per pixel from the
image's structure tensor:

  1. gradient by central differences, the image zero outside its support:
         gx[y,x] = (f[y,x+1] - f[y,x-1]) / 2,   gy[y,x] = (f[y+1,x] - f[y-1,x]) / 2;
  2. tensor J = G_rho * (g g^T): the products gx^2, gx gy, gy^2 smoothed with a
     sampled Gaussian of standard deviation rho (weights exp(-k^2 / (2 rho^2)),
     |k| <= ceil(3 rho), normalised to sum 1), zero outside the image,
     separably (rows, then columns);
  3. eigenvalues l1 >= l2 >= 0 of J, coherence
         coh = ((l1 - l2) / (l1 + l2 + eps))^2   in [0, 1];
  4. ellipse: size sigma0, elongation e = 1 + (e_max - 1) coh, major axis along
     the eigenvector of l2 (along the edge), given as (cos t, sin t) with
     sin t >= 0 (t in [0, pi)); where l1 == l2 the axis is (1, 0).

The result feeds the ellipse scale kind of the filter (sigma, e, cos t, sin t).
"""
import math

import numpy as np


def gaussian_taps(rho):
    """Sampled, normalised Gaussian of std rho on |k| <= ceil(3 rho)."""
    r = int(math.ceil(3.0 * rho))
    k = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * rho * rho))
    return w / w.sum(), r


def gradient(f):
    f = np.asarray(f, dtype=np.float64)
    p = np.pad(f, 1)
    gx = (p[1:-1, 2:] - p[1:-1, :-2]) / 2.0
    gy = (p[2:, 1:-1] - p[:-2, 1:-1]) / 2.0
    return gx, gy


def smooth(a, rho):
    """Separable zero-padded Gaussian: rows (along x) first, then columns."""
    w, r = gaussian_taps(rho)
    H, W = a.shape
    p = np.pad(a, ((0, 0), (r, r)))
    b = sum(w[i] * p[:, i:i + W] for i in range(2 * r + 1))
    p = np.pad(b, ((r, r), (0, 0)))
    return sum(w[i] * p[i:i + H, :] for i in range(2 * r + 1))


def ellipse_field(f, rho=2.0, sigma0=4.0, e_max=4.0, eps=1e-12):
    """(H, W, 4) binary64: sigma, elongation, cos t, sin t."""
    gx, gy = gradient(f)
    j11 = smooth(gx * gx, rho)
    j12 = smooth(gx * gy, rho)
    j22 = smooth(gy * gy, rho)
    tr = j11 + j22
    d = np.sqrt((j11 - j22) ** 2 + 4.0 * j12 * j12)
    l1 = 0.5 * (tr + d)
    l2 = 0.5 * (tr - d)
    coh = ((l1 - l2) / (l1 + l2 + eps)) ** 2
    # eigenvector of l2: (j12, l2 - j11) or (l2 - j22, j12), whichever is longer
    ax, ay = j12, l2 - j11
    bx, by = l2 - j22, j12
    use_b = (bx * bx + by * by) > (ax * ax + ay * ay)
    vx = np.where(use_b, bx, ax)
    vy = np.where(use_b, by, ay)
    n = np.sqrt(vx * vx + vy * vy)
    flat = n == 0.0
    vx = np.where(flat, 1.0, vx / np.where(flat, 1.0, n))
    vy = np.where(flat, 0.0, vy / np.where(flat, 1.0, n))
    # orientation in [0, pi): sin t >= 0 (and (1, 0) for t = 0)
    flip = (vy < 0.0) | ((vy == 0.0) & (vx < 0.0))
    vx = np.where(flip, -vx, vx)
    vy = np.where(flip, -vy, vy)
    e = 1.0 + (e_max - 1.0) * coh
    sig = np.full(vx.shape, float(sigma0))
    return np.stack([sig, e, vx, vy], axis=-1)
