"""Generalised plans on the GPU against oracle.general: directional order
N = 2 (Sec. 4 Eq. (def), theta = 0, pi/2) and the B-spline model phi of
Sec. 6 (with its separable interpolation prefilter for degrees >= 2).

Numerators bit-exact (mod 2^(64 L)) at every pixel of images that span several
CTAs with ragged edges; s within 1e-13 relative of the correctly rounded
oracle.  For a prefiltered model the oracle's c_q comes from its own exact
rational prefilter; the model is also checked against the definition on the
unrounded coefficients (within the half-step rounding bound)."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import synthetic
from oracle import general, scales as oscales
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _steps(rng, shape, lo, hi, directions):
    sc = synthetic.scales_a4(rng, shape, lo, hi, 6.0).astype(np.float32)
    if directions == 2:
        sc[..., 1] = 1.0
        sc[..., 3] = 1.0
    return sc


def _run(img, sc, n, q, F, cmax, directions, E, vb, want_num=True, debug_bounds=False):
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter
    H, W = img.shape
    filt = AdaptiveFilter(W, H, n, gu.torch_dtype(img.dtype), scale_kind="c4", q_bits=q, frac_bits=F,
                          max_scale=cmax, out="f64", value_bound=vb, device="cuda:0", directions=directions,
                          model_boxes=E, debug_bounds=debug_bounds)
    filt.integrate(gu.to_device(img, "cuda:0"))
    s_t = gu.to_device(sc, "cuda:0")
    s = filt.filter(s_t).cpu().numpy()
    num = filt.numerators(s_t).cpu().numpy().astype(np.uint64) if want_num else None
    torch.cuda.synchronize()
    st = filt.device_status()
    L = filt.limbs
    if debug_bounds:
        assert filt.bounds_violation() == -1
    filt.close()
    return s, num, st, L


CASES = [
    # directions, n, E (model boxes), shape, Q, step range, input kind
    (2, 2, 0, (37, 70), 3, (1.0, 6.0), "u8"),
    (2, 3, 0, (21, 45), 2, (1.0, 4.0), "f32"),
    (4, 1, 2, (26, 40), 3, (1.0, 5.0), "u8"),
    (2, 1, 2, (30, 41), 3, (1.0, 6.0), "f32"),
    (2, 2, 0, (29, 37), 3, (1.0, 6.0), "f32big"),   # two limbs
]


@pytest.mark.parametrize("directions,n,E,shape,q,rng_c,kind", CASES)
def test_general_plan_bit_exact(directions, n, E, shape, q, rng_c, kind):
    rng = np.random.default_rng(70 + 7 * n + E)
    if kind == "u8":
        img, F, vb = rng.integers(0, 256, shape).astype(np.uint8), 0, 255.0
    elif kind == "f32big":
        # samples up to 2^43 (24-bit integers times 2^20, exact in binary32): the
        # numerators need a second limb
        img, F, vb = (rng.integers(-2**23, 2**23, shape) * 2.0**20).astype(np.float32), 16, 2.0**43
    else:
        img, F, vb = synthetic.image_f32_grid(rng, shape, 6.0, 3, 8), 8, 255.0
    sc = _steps(rng, shape, rng_c[0], rng_c[1], directions)
    cmax = rng_c[1]
    s, num, st, L = _run(img, sc, n, q, F, cmax, directions, E, vb)
    assert st == 0
    if kind == "f32big":
        assert L == 2
    C = oscales.scales_to_C("c4", sc, n, q, cmax)
    H, W = shape
    fi = (img.astype(np.float64) * (1 << F)).astype(np.int64)
    r = (n, n if directions == 4 else 0, n, n if directions == 4 else 0)
    pix = [(x, y) for y in range(H) for x in range(W)]
    S_ref, s_ref = general.filter_image(fi, (0, 0), C, r, E - 1 if E else None, q, F)
    got = gu.wide_to_int(num, L)
    mod = 1 << (64 * L)
    bad = [p for p, a, b in zip(pix, S_ref, got) if a % mod != b]
    assert not bad, "numerators differ at %d pixels, first %s" % (len(bad), bad[:3])
    ref = np.array([float(v) for v in s_ref]).reshape(H, W)
    gu.assert_close_f64(s, ref, rel=1e-13, absol=1e-300)


@pytest.mark.parametrize("directions,n,E,shape", [(4, 1, 4, (23, 39)), (2, 2, 4, (23, 39)), (4, 1, 6, (9, 35))])
def test_model_with_prefilter(directions, n, E, shape):
    """B-spline models of degree E - 1 = 3 (cubic) and 5: abf_integrate
    prefilters f along rows and columns into c_q = rint(c 2^F) on an extended
    frame, then runs the exact method on it.  Numerators equal the oracle's on
    its own exact c_q (bit for bit, wherever the two c_q agree: everywhere
    here), and (degree 3) s is within half a grid step of the definition on the
    unrounded model.  The stencils have 60, 36 and 96 neighbours (two per lane
    of a warp, and the pair-dealt kernel beyond 64)."""
    rng = np.random.default_rng(91 + n + E)
    q = 2
    img = rng.integers(0, 256, shape).astype(np.uint8)
    sc = _steps(rng, shape, 1.0, 4.0, directions)
    s, num, st, L = _run(img, sc, n, q, 0, 4.0, directions, E, 255.0)
    assert st == 0
    C = oscales.scales_to_C("c4", sc, n, q, 4.0)
    H, W = shape
    n1 = E - 1
    cq, origin = general.prefilter2d(img.astype(np.int64), n1, bits=120)
    r = (n, n if directions == 4 else 0, n, n if directions == 4 else 0)
    pix = [(x, y) for y in range(H) for x in range(W)]
    S_ref, s_ref = general.filter_image(cq, origin, C, r, n1, q, 0)
    got = gu.wide_to_int(num, L)
    mod = 1 << (64 * L)
    bad = [p for p, a, b in zip(pix, S_ref, got) if a % mod != b]
    assert not bad, "numerators differ at %d pixels, first %s" % (len(bad), bad[:3])
    ref = np.array([float(v) for v in s_ref]).reshape(H, W)
    gu.assert_close_f64(s, ref, rel=1e-13, absol=1e-300)
    if E > 4:
        return  # the definition's exact sums at degree 5 take minutes in the oracle
    # the rounded model against the definition on the exact coefficients, a few pixels
    cx, ox = general.prefilter2d(img.astype(np.int64) << 20, n1, bits=120)   # c 2^20: 20 more bits of c
    few = [(0, 0), (W // 2, H // 2)]
    sd = general.filter_direct(cx, ox, C, r, n1, q, 20, few)
    for (x, y), v in zip(few, sd):
        assert abs(Fr(s[y, x]) - v) <= Fr(1, 2) + Fr(1, 1 << 18)


@pytest.mark.parametrize("directions,n,E,shape", [(2, 2, 0, (37, 70)), (2, 3, 0, (21, 45)), (4, 1, 2, (26, 40)),
                                                  (4, 1, 4, (23, 39)), (4, 1, 6, (9, 35))])
def test_general_debug_bounds_checks_find_no_violation(directions, n, E, shape):
    """Generalised plans with every read checked against the lattice box (the
    group kernels, the N = 2 unrolled taps, the pair-dealt kernel): steps at
    the plan's maximum somewhere, no violation, and the unchecked plan's
    numerators."""
    rng = np.random.default_rng(120 + n + E)
    img = rng.integers(0, 256, shape).astype(np.uint8)
    sc = _steps(rng, shape, 1.0, 4.0, directions)
    sc[0, 0, :] = 4.0      # the widest reach at two corners
    sc[-1, -1, :] = 4.0
    if directions == 2:
        sc[..., 1] = sc[..., 3] = 1.0
    a = _run(img, sc, n, 2, 0, 4.0, directions, E, 255.0)
    b = _run(img, sc, n, 2, 0, 4.0, directions, E, 255.0, debug_bounds=True)
    assert a[2] == 0 and b[2] == 0
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], b[0])

