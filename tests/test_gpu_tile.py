"""GPU floating-point forms (per-tile restart windows in pair arithmetic)
against the exact oracle, at the tolerances the forms state: binary64 pairs
within 1e-12 of the value range, binary32 pairs within 1e-5 (order 1).

Every pixel checks an a-priori bound on its own error and is NaN, with
ABF_DEV_PRECISION set, where the bound exceeds the tolerance; so the tests
require (a) every pixel that is not NaN to be within the tolerance of the
oracle and (b) no NaN at all where the bound is small (binary64 pairs on every
case here).  Errors are range-relative: max |s - s_oracle| / (max f - min f).
"""
import numpy as np
import pytest

import synthetic
from oracle import paper
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

PRECISION = 16   # ABF_DEV_PRECISION


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run_tile(w, form, out="f64"):
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter
    img, sc = w["image"], w["scales"]
    H, W = img.shape
    filt = AdaptiveFilter(W, H, w["n"], gu.torch_dtype(img.dtype), scale_kind=w["scale_kind"], q_bits=w["q_bits"],
                          frac_bits=w["frac_bits"], max_scale=w["cmax"], out=out, form=form,
                          value_bound=w["value_bound"], device="cuda:0")
    s = filt(gu.to_device(img, "cuda:0"), gu.to_device(sc.astype(np.float32), "cuda:0"))
    torch.cuda.synchronize()
    st = filt.device_status()
    filt.close()
    return s.cpu().numpy().astype(np.float64), st


def _err_range(s, ref, img):
    rng = float(img.max()) - float(img.min())
    return float(np.abs(s - ref).max()) / max(rng, 1e-300)


# (order, shape spanning several tiles with ragged edges, Q, largest paper scale)
CASES = [(1, (40, 300), 4, 6.0), (2, (70, 290), 3, 4.0), (3, (24, 60), 2, 3.0)]


@pytest.mark.parametrize("n,shape,q,hi", CASES)
def test_plain_f64_within_1e12_every_pixel(n, shape, q, hi):
    rng = np.random.default_rng(40 + n)
    img = rng.integers(0, 256, shape).astype(np.float64)
    sc = synthetic.scales_a4(rng, shape, 1.0, hi, 12.0)
    w = dict(image=img, frac_bits=0, scale_kind="a4", scales=sc, n=n, q_bits=q, cmax=hi, value_bound=255.0)
    C = gu.oracle_C(w)
    _, s_ref = paper.filter_image(img.astype(np.int64), C, n, q, 0)
    s, st = _run_tile(w, "plain_f64")
    assert st == 0 and np.isfinite(s).all()
    err = _err_range(s, s_ref, img)
    print("plain_f64 n=%d err_range=%.3g" % (n, err))
    assert err <= 1e-12


def test_plain_f64_within_1e12_on_the_ellipse_recipe():
    """The order-2 ellipse workload's recipe (f32 on the 2^-16 grid, sigma up
    to 24, elongation up to 6, steps up to 150) at 384 x 320: 120 random
    pixels, the four corners and every 16th pixel of the middle row (the
    oracle evaluates each on its own window)."""
    w = synthetic.workload("c2", shape=(384, 320))
    img = w["image"]
    H, W = img.shape
    C = gu.oracle_C(w)
    s, st = _run_tile(w, "plain_f64")
    assert st == 0 and np.isfinite(s).all()
    rng = np.random.default_rng(5)
    pts = [(int(x), int(y)) for x, y in zip(rng.integers(0, W, 120), rng.integers(0, H, 120))]
    pts += [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1)] + [(x, H // 2) for x in range(0, W, 16)]
    fi = gu.f_int(w)
    _, sv = paper.filter_pixels(fi, C, w["n"], w["q_bits"], w["frac_bits"], pts)
    got = np.array([s[y, x] for x, y in pts])
    err = float(np.abs(got - np.asarray(sv, dtype=np.float64)).max()) / (float(img.max()) - float(img.min()))
    print("plain_f64 ellipse recipe err_range=%.3g over %d pixels" % (err, len(pts)))
    assert err <= 1e-12


def test_tile_f32_within_1e5_where_its_bound_holds():
    rng = np.random.default_rng(50)
    shape = (40, 300)
    img = rng.integers(0, 256, shape).astype(np.float64)
    sc = synthetic.scales_a4(rng, shape, 1.0, 6.0, 12.0)
    w = dict(image=img, frac_bits=0, scale_kind="a4", scales=sc, n=1, q_bits=4, cmax=6.0, value_bound=255.0)
    C = gu.oracle_C(w)
    _, s_ref = paper.filter_image(img.astype(np.int64), C, 1, 4, 0)
    s, st = _run_tile(w, "tile_f32", out="f64")
    ok = np.isfinite(s)
    assert (st & ~PRECISION) == 0
    assert (st & PRECISION != 0) == (not ok.all())
    err = float(np.abs(s[ok] - s_ref[ok]).max()) / 255.0
    print("tile_f32 n=1 err_range=%.3g, %d of %d pixels within the bound" % (err, ok.sum(), ok.size))
    assert err <= 1e-5
    assert ok.mean() >= 0.99


def test_precision_flag_marks_pixels_the_bound_cannot_cover():
    """Unit steps everywhere except one pixel with steps of 60: its 8 x 8 tile
    gets a window of about 190 x 190, so the unit-step pixels there have a
    binary32-pair bound far above 1e-5 and are NaN with ABF_DEV_PRECISION;
    binary64 pairs cover them (bound ~1e-17) and stay within 1e-12 everywhere."""
    rng = np.random.default_rng(51)
    shape = (24, 40)
    img = rng.integers(0, 256, shape).astype(np.float64)
    sc = np.ones(shape + (4,), dtype=np.float32)
    sc[3, 3, :] = 60.0
    w = dict(image=img, frac_bits=0, scale_kind="c4", scales=sc, n=1, q_bits=4, cmax=64.0, value_bound=255.0)
    C = gu.oracle_C(w)
    _, s_ref = paper.filter_image(img.astype(np.int64), C, 1, 4, 0)
    s32, st32 = _run_tile(w, "tile_f32")
    bad = ~np.isfinite(s32)
    assert st32 == PRECISION and bad[:8, :8].sum() > 0 and not bad[8:, 8:].any()
    assert float(np.abs(s32[~bad] - s_ref[~bad]).max()) / 255.0 <= 1e-5
    s64, st64 = _run_tile(w, "plain_f64")
    assert st64 == 0 and np.isfinite(s64).all()
    assert _err_range(s64, s_ref, img) <= 1e-12
