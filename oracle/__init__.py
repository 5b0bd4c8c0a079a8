"""Exact CPU oracle for the adaptive elliptical box-spline filter.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with ``paper_0908_3861_gb300`` (the CUDA path) and neither
imports the other.

What it computes, and where the paper defines it (Chaudhury, Munoz-Barrutia,
Unser, "Fast adaptive elliptical filtering using box splines"):

* ``boxspline``  -- exact values of box splines.  The four-direction box spline
  of Sec. 4, Eq. (def) with N=4 and the lattice directions of Sec. 7; the
  Zwart-Powell (ZP) element of Sec. 7 and its n-fold self-convolution (the
  interpolation kernel of Eq. (final_eqn)).  Evaluated with de Boor's
  recurrence in exact rational arithmetic.
* ``paper``      -- the paper's algorithm step by step in exact integer
  arithmetic: the four running-sum recursions of Sec. 7 (1) (Eq. (RS)), the
  16-vertex affine FD mesh of Eq. (final_eqn) / Table "Mesh Vertices" with its
  shift vector tau, ZP interpolation, and the normalisation alpha.
* ``direct``     -- the quantity the algorithm computes, written from its
  definition: s[m] = <f, beta_a(m)(. - m)> of Sec. 6 with phi = delta
  (Sec. 7 (1)), i.e. a plain sum of the image against the box-spline kernel.
* ``line1d``     -- the 1-D scale-adaptive B-spline filter of Sec. 3
  (Proposition "prop"): B-splines and their dilates (Sec. 2), the projection
  s[m] = <f, beta_a^{n2}(. - m)> from its definition by exact piecewise
  integration, and the Proposition's two steps (running sums, then the FD
  mask with B-spline interpolation) in exact integers; for model degrees
  n1 >= 2 the interpolation prefilter c = f * (b^{n1})^-1, its inverse taken
  from the definition (an exact banded solve of b * h = delta).
* ``structure``  -- scale-map estimation (the paper defers it, Sec. 8): a
  reading, the structure tensor of the image turned into an edge-following
  ellipse per pixel (binary64).
* ``scales``     -- the per-pixel scale readings: paper scales a_k (Sec. 7)
  to lattice steps c_k, and the ellipse-to-scales moment rule (a reading: the
  paper leaves the scale map to other work, Sec. 8; Theorem (convergence) of
  Sec. 4 fixes the isotropic case).

Readings of the paper that the oracle fixes:
  * order n >= 1 means every one of the four directional B-splines is the
    n-fold self-convolution of the box (n=1 is Sec. 7 exactly); the mesh then
    has (n+1)^4 vertices with binomial weights, tau scales by n, the
    interpolation kernel is ZP^{*n};
  * unit-weight running sums (the sqrt(2) factors of Sec. 7 (1) folded into the
    normaliser: alpha * g_b = (c1 c2 c3 c4)^{-1} g, exactly);
  * zero padding outside the image (Sec. 2 leaves the boundary open).

Exactness: integer images (or images on a 2^-F grid) and scales on a 2^-Q
grid make every quantity a rational number.  The oracle keeps them exact
(Python integers / ``fractions.Fraction``) and rounds once, at the end.
"""
