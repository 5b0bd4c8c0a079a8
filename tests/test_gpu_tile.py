"""GPU floating-point forms (per-tile restart windows, binary64 and binary32)
against the exact oracle.

These forms are not exact: rounding in the running sums and weights is
amplified by the cancellation of the FD mesh, by about the window extent over
the step to the power 4n.  The tests state the error each form reaches
(range-relative, max over all pixels) and check it against a bound derived
from that amplification; they also check that the forms agree with the oracle
at all, pixel by pixel, on images of several tiles with ragged edges.
"""
import numpy as np
import pytest

import synthetic
from oracle import paper
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


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
                          frac_bits=w["frac_bits"], max_scale=w["cmax"], out=out, form=form, device="cuda:0")
    s = filt(gu.to_device(img, "cuda:0"), gu.to_device(sc.astype(np.float32), "cuda:0"))
    torch.cuda.synchronize()
    st = filt.device_status()
    filt.close()
    return s.cpu().numpy().astype(np.float64), st


def _err_range(s, ref, img):
    rng = float(img.max()) - float(img.min())
    return float(np.abs(s - ref).max()) / max(rng, 1e-300)


# Bounds: the window side l is at most about T + 6n c_max with T <= c_min, and
# the amplification is about 2^(4n) (l / c_min)^(4n) / (4n)! times the unit
# roundoff; with c_min = a/sqrt2 >= 0.7 here that is ~1e-13 (n = 1, integers
# stay exact), ~1e-4 (n = 2) and ~1e-3 (n = 3) for binary64.
CASES = [(1, (40, 300), 4, 6.0, 1e-12), (2, (70, 290), 3, 4.0, 1e-4), (3, (24, 60), 2, 3.0, 1e-3)]


@pytest.mark.parametrize("n,shape,q,hi,tol", CASES)
def test_plain_f64_matches_oracle(n, shape, q, hi, tol):
    rng = np.random.default_rng(40 + n)
    img = rng.integers(0, 256, shape).astype(np.float64)
    sc = synthetic.scales_a4(rng, shape, 1.0, hi, 12.0)
    w = dict(image=img, frac_bits=0, scale_kind="a4", scales=sc, n=n, q_bits=q, cmax=hi, value_bound=255.0)
    C = gu.oracle_C(w)
    _, s_ref = paper.filter_image(img.astype(np.int64), C, n, q, 0)
    s, st = _run_tile(w, "plain_f64")
    assert st == 0
    err = _err_range(s, s_ref, img)
    print("plain_f64 n=%d err_range=%.3g" % (n, err))
    assert err <= tol


def test_tile_f32_reports_its_error():
    rng = np.random.default_rng(50)
    shape = (40, 300)
    img = rng.integers(0, 256, shape).astype(np.float64)
    sc = synthetic.scales_a4(rng, shape, 1.0, 6.0, 12.0)
    w = dict(image=img, frac_bits=0, scale_kind="a4", scales=sc, n=1, q_bits=4, cmax=6.0, value_bound=255.0)
    C = gu.oracle_C(w)
    _, s_ref = paper.filter_image(img.astype(np.int64), C, 1, 4, 0)
    s, st = _run_tile(w, "tile_f32", out="f32")
    assert st == 0
    err = _err_range(s, s_ref, img)
    print("tile_f32 n=1 err_range=%.3g" % err)
    assert err <= 1e-2
