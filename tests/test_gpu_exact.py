"""GPU parity of the exact form (wrap-around integer running sums, integer
ZP^{*n} weights) against the exact CPU oracle, through the C ABI.

Bit-exact: the per-pixel integer steps C_k, the numerators S (modulo
2^(64 L)), and the integrated image wherever the 3pi/4 recursion's backward ray
leaves the lattice box through its bottom row.  Floating point: the binary64
output s = S / Den within 1e-13 relative (a handful of roundings in the final
division; the oracle rounds the exact rational once).
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


def _small_workload(n, shape, q, dtype, seed, lo=1.0, hi=6.0, neg=False):
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        img = rng.integers(0, 256, shape).astype(np.uint8)
        fb, vb = 0, 255.0
    elif dtype == "u16":
        img = rng.integers(0, 65536, shape).astype(np.uint16)
        fb, vb = 0, 65535.0
    elif dtype == "f32":
        img = synthetic.image_f32_grid(rng, shape, 6.0, 4, 16)
        fb, vb = 16, 255.0
    else:
        img = rng.integers(-300 if neg else 0, 300, shape).astype(np.float64)
        fb, vb = 0, 300.0
    sc = synthetic.scales_a4(rng, shape, lo, hi, 8.0)
    return dict(image=img, frac_bits=fb, scale_kind="a4", scales=sc, n=n, q_bits=q, cmax=hi, value_bound=vb)


def _check_all_pixels(w, res):
    C_ref = gu.oracle_C(w)
    assert (res["C"] == C_ref).all(), "integer steps differ"
    S_ref, s_ref = paper.filter_image(gu.f_int(w), C_ref, w["n"], w["q_bits"], w["frac_bits"])
    L = res["limbs"]
    got = gu.wide_to_int(res["num"], L)
    mod = 1 << (64 * L)
    ref = [int(v) % mod for v in S_ref.ravel()]
    bad = [i for i, (a, b) in enumerate(zip(got, ref)) if a != b]
    assert not bad, "numerators differ at %d pixels, first %s" % (len(bad), divmod(bad[0], w["image"].shape[1]))
    gu.assert_close_f64(res["s"], s_ref, rel=1e-13, absol=1e-300)
    return S_ref, s_ref


def _check_g(w, res):
    """Integrated image vs the oracle's recursions, where the GPU's is exact."""
    H, W = w["image"].shape
    left, right, _, above = res["halo"]
    L = res["limbs"]
    g_or = paper.integrate(gu.f_int(w), w["n"], -left, W + right, 0, H + above, exact=True)
    g = res["g"]
    mod = 1 << (64 * L)
    for yi in range(H + above):
        for xi in range(W + left + right):
            x = xi - left
            if x + yi < W + right:   # backward 3pi/4 ray reaches row 0 inside the box
                v = sum(int(g[yi, xi, i]) << (64 * i) for i in range(L))
                assert v == int(g_or[yi, xi]) % mod, (xi, yi)


CASES = [
    (1, (37, 70), 4, "u8", 1),
    (1, (45, 33), 8, "f64", 2),
    (2, (37, 70), 4, "f32", 3),
    (2, (19, 129), 3, "u16", 4),
    (3, (14, 23), 2, "u8", 5),
    (3, (18, 70), 2, "f32", 6),
]


@pytest.mark.parametrize("n,shape,q,dtype,seed", CASES)
def test_exact_small_images_all_pixels(n, shape, q, dtype, seed):
    w = _small_workload(n, shape, q, dtype, seed, neg=(dtype == "f64"))
    res = gu.run_exact(w, want=("s", "num", "C", "g"))
    assert res["status"] == 0
    _check_all_pixels(w, res)
    _check_g(w, res)


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (17, 1), (2, 3)])
def test_degenerate_sizes(n, shape):
    w = _small_workload(n, shape, 3, "u8", 10 + n)
    res = gu.run_exact(w)
    assert res["status"] == 0
    _check_all_pixels(w, res)


@pytest.mark.parametrize("n,shape", [(2, (1, 40)), (2, (3, 40)), (2, (2, 70)), (3, (1, 40)), (3, (4, 40)),
                                     (3, (2, 33))])
def test_shallow_box_general_and_fast_paths(n, shape):
    """Scales below one leave a lattice box of fewer than 3n rows (H + above
    < 3n, e.g. shape (1, 40)): the mesh then runs its general path; (3, 40) at
    n = 2 and (4, 40) at n = 3 sit exactly at the fast path's limit of 3n
    rows."""
    w = _small_workload(n, shape, 4, "u8", 30 + 10 * n + shape[0], lo=0.3, hi=0.9)
    w["min_scale"] = 0.1
    res = gu.run_exact(w)
    assert res["status"] == 0
    _check_all_pixels(w, res)


def test_zero_and_constant_images():
    for val in (0, 200):
        w = _small_workload(1, (20, 30), 3, "u8", 7)
        w["image"] = np.full((20, 30), val, dtype=np.uint8)
        w["scales"] = np.broadcast_to(np.array([2.0, 2.0 * np.sqrt(2), 3.0, np.sqrt(2)], np.float32),
                                      (20, 30, 4)).copy()
        res = gu.run_exact(w)
        _check_all_pixels(w, res)
        if val == 0:
            assert (res["s"] == 0).all()
        else:   # integer c1, c3: unit lattice sum in the interior
            assert (res["s"][6:-6, 6:-6] == val).all()


def test_repeatable_bitwise():
    """Two runs give identical numerators (no order dependence in the scans)."""
    w = _small_workload(2, (64, 150), 5, "f32", 21)
    a = gu.run_exact(w, want=("num",))["num"]
    b = gu.run_exact(w, want=("num",))["num"]
    assert (a == b).all()


def test_invalid_scales_are_flagged():
    from paper_0908_3861_gb300 import _abf
    w = _small_workload(1, (16, 40), 3, "u8", 8)
    sc = w["scales"].copy()
    sc[3, 5, 0] = np.nan
    sc[7, 9, 2] = 0.0
    sc[10, 30, 1] = 100.0      # above max_scale
    w["scales"] = sc
    res = gu.run_exact(w, want=("s",))
    assert res["status"] & _abf.ABF_DEV_BAD_SCALE
    s = res["s"]
    assert np.isnan(s[3, 5]) and np.isnan(s[7, 9]) and np.isnan(s[10, 30])
    ok = ~np.isnan(s)
    assert ok.sum() == s.size - 3


def test_bad_input_is_flagged():
    from paper_0908_3861_gb300 import _abf
    w = _small_workload(1, (16, 40), 3, "f32", 9)
    img = w["image"].copy()
    img[2, 3] = 1.0 + 2.0 ** -20        # not on the 2^-16 grid
    w["image"] = img
    res = gu.run_exact(w, want=("s",))
    assert res["status"] & _abf.ABF_DEV_BAD_INPUT


def test_plan_refuses_numerator_beyond_four_limbs():
    import torch
    from paper_0908_3861_gb300 import _abf, AdaptiveFilter
    with pytest.raises(_abf.AbfError) as e:
        AdaptiveFilter(64, 64, 3, torch.float64, scale_kind="a4", q_bits=8, frac_bits=40, max_scale=1000.0,
                       value_bound=1e30)
    assert e.value.status == 5   # ABF_ERR_RANGE


def _sample_pixels(H, W, k, seed):
    rng = np.random.default_rng(seed)
    pts = {(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, 0), (0, H // 2), (W - 1, H // 2),
           (W // 2, H - 1)}
    while len(pts) < k:
        pts.add((int(rng.integers(0, W)), int(rng.integers(0, H))))
    return sorted(pts)


def _measured_product(w):
    import torch
    from paper_0908_3861_gb300 import _abf
    H, W = w["image"].shape
    d = _abf.abf_desc()
    d.width, d.height, d.order_n = W, H, w["n"]
    d.scale_kind = _abf.SCALE_KINDS[w["scale_kind"]]
    d.q_bits, d.max_scale = w["q_bits"], w["cmax"]
    sc = gu.to_device(w["scales"].astype(np.float32), "cuda:0")
    mx, prod = _abf.abf_measure_scales(d, sc, W * 16)
    assert mx <= w["cmax"]
    return prod


def test_full_size_256_order1_all_pixels():
    """256x256 integer image, n = 1, paper scales in [1, 8], Q = 8 (every pixel)."""
    w = synthetic.workload("c1")
    res = gu.run_exact(w)
    assert res["status"] == 0 and res["limbs"] == 1
    _check_all_pixels(w, res)


@pytest.mark.slow
def test_full_size_2048_order2_ellipse_sampled():
    """2048x2048 float32 on the 2^-16 grid, n = 2, ellipse scales, Q = 8:
    2^16 random pixels plus every pixel of the four border rows and columns,
    numerators bit-exact and s within 1e-13 (the oracle per pixel, on every
    host core)."""
    w = synthetic.workload("c2")
    prod = _measured_product(w)
    res = gu.run_exact(w, max_scale_product=prod)
    assert res["status"] == 0
    assert np.isfinite(res["s"]).all()
    H, W = w["image"].shape
    rng = np.random.default_rng(1)
    pts = set((int(x), int(y)) for x, y in zip(rng.integers(0, W, 1 << 16), rng.integers(0, H, 1 << 16)))
    pts |= {(x, 0) for x in range(W)} | {(x, H - 1) for x in range(W)}
    pts |= {(0, y) for y in range(H)} | {(W - 1, y) for y in range(H)}
    pix = sorted(pts)
    C_ref = gu.oracle_C(w)
    assert (res["C"] == C_ref).all(), "integer steps differ"
    S_ref, s_ref = gu.oracle_pixels_parallel("c2", None, pix)
    L = res["limbs"]
    mod = 1 << (64 * L)
    num = res["num"]
    bad = 0
    for (x, y), S, sv in zip(pix, S_ref, s_ref):
        got = sum(int(num[y, x, i]) << (64 * i) for i in range(L))
        if got != S % mod or not abs(res["s"][y, x] - sv) <= 1e-13 * abs(sv) + 1e-300:
            bad += 1
    assert bad == 0, "%d of %d pixels differ" % (bad, len(pix))
    assert len(pix) >= (1 << 16)


@pytest.mark.slow
def test_full_size_8192_order3_sampled():
    """8192x8192 uint16, n = 3, paper scales in [1, 48], Q = 8: numerators at
    sampled pixels (corners, borders, interior), and the whole integrated image
    modulo 2^64."""
    w = synthetic.workload("c3")
    prod = _measured_product(w)
    res = gu.run_exact(w, max_scale_product=prod, want=("s", "num", "C"))
    assert res["status"] == 0
    H, W = w["image"].shape
    # numerators at the corners, edge midpoints, 8 points along every border and
    # random interior pixels (the oracle per pixel, on every host core)
    pix = set(_sample_pixels(H, W, 200, 2))
    for t in range(8):
        pix |= {((t * W) // 8, 0), ((t * W) // 8, H - 1), (0, (t * H) // 8), (W - 1, (t * H) // 8)}
    pix = sorted(pix)
    assert (res["C"] == gu.oracle_C(w)).all(), "integer steps differ"
    S_ref, s_ref = gu.oracle_pixels_parallel("c3", None, pix, chunk=8)
    L = res["limbs"]
    mod = 1 << (64 * L)
    for (x, y), S, sv in zip(pix, S_ref, s_ref):
        got = sum(int(res["num"][y, x, i]) << (64 * i) for i in range(L))
        assert got == S % mod, (x, y)
        assert abs(res["s"][y, x] - sv) <= 1e-13 * abs(sv) + 1e-300, (x, y, res["s"][y, x], sv)
    # the whole integrated image modulo 2^64 (the low limb), wherever the
    # 3pi/4 rays leave the box through its bottom row
    filt = res["filt"]
    left, right, _, above = res["halo"]
    rows = H + above
    g = filt.integrated().cpu().numpy()[..., 0].astype(np.uint64)
    g_or = paper.integrate(gu.f_int(w), w["n"], -left, W + right, 0, rows, exact=False)
    xs = np.arange(W + left + right)[None, :] - left
    for y0 in range(0, rows, 512):
        ys = np.arange(y0, min(rows, y0 + 512))[:, None]
        region = xs + ys < W + right
        assert (g[y0:y0 + 512, :W + left + right][region] == g_or[y0:y0 + 512][region]).all(), y0


def test_two_plans_share_one_workspace():
    """A workspace left behind by one plan's scans is safe for another plan."""
    wa = _small_workload(2, (40, 90), 4, "u8", 31)
    wb = _small_workload(2, (52, 70), 4, "u8", 32)
    ra = gu.run_exact(wa, want=("num",))
    rb = gu.run_exact(wb, want=("num",))
    fa, fb = ra["filt"], rb["filt"]
    big = fa.ws if fa.ws.numel() >= fb.ws.numel() else fb.ws
    fa.ws = big
    fb.ws = big
    import torch
    for _ in range(2):
        for w, f, ref in ((wa, fa, ra["num"]), (wb, fb, rb["num"])):
            f.integrate(gu.to_device(w["image"], "cuda:0"))
            got = f.numerators(gu.to_device(w["scales"].astype(np.float32), "cuda:0"))
            torch.cuda.synchronize()
            assert (got.cpu().numpy().astype(np.uint64) == ref).all()


def test_lookback_wait_times_out_then_the_context_recovers():
    """Failure path of the scans: a line pass whose first band never runs
    leaves the next band waiting on a flag nothing sets.  The wait is bounded:
    the pass completes with ABF_DEV_TIMEOUT in the status word, and the same
    process then filters correctly."""
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter, _abf
    w = _small_workload(1, (100, 60), 4, "u8", 77)   # two bands of 64 rows: band 1 waits on band 0
    H, W = w["image"].shape
    filt = AdaptiveFilter(W, H, 1, torch.uint8, scale_kind="a4", q_bits=4, frac_bits=0, max_scale=w["cmax"],
                          out="f64", value_bound=255.0, device="cuda:0")
    assert 64 < H + filt.info["halo_lrbt"][3] <= 128
    _abf.abf_debug_starved_lookback(filt.plan, filt.g, filt.ws)
    torch.cuda.synchronize()
    assert filt.device_status() & _abf.ABF_DEV_TIMEOUT
    filt.close()
    res = gu.run_exact(w)
    assert res["status"] == 0
    _check_all_pixels(w, res)


@pytest.mark.parametrize("n,shape,q,dtype,seed,lo", [c + (1.0,) for c in CASES] +
                         [(1, (37, 70), 4, "u8", 11, 6.0), (2, (37, 70), 4, "f32", 12, 6.0),
                          (3, (18, 70), 2, "f32", 13, 6.0)])
def test_debug_bounds_checks_find_no_violation(n, shape, q, dtype, seed, lo):
    """With ABF_FLAG_DEBUG_BOUNDS every tap of every pixel is checked against
    the lattice box before it is read: the box the plan sizes from the taps'
    reach holds at every pixel (also with every step at the plan's maximum,
    lo = 6), and the checked plan gives the unchecked plan's numerators."""
    w = _small_workload(n, shape, q, dtype, seed, lo=lo, hi=6.0)
    a = gu.run_exact(w, want=("s", "num"))
    b = gu.run_exact(w, want=("s", "num"), debug_bounds=True)
    assert a["status"] == 0 and b["status"] == 0
    assert b["filt"].bounds_violation() == -1
    assert np.array_equal(a["num"], b["num"])
    assert np.array_equal(a["s"], b["s"])


def test_debug_bounds_full_size_2048_order2_ellipse():
    """The bench workload (2048^2, order 2, ellipse fields, the plan sized for
    the parameter range) with every tap checked: no pixel reads outside the
    lattice box, and the output equals the unchecked plan's bit for bit."""
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter, ellipse_product_bound
    w = synthetic.workload("c2")
    img, sc = w["image"], w["scales"]
    H, W = img.shape
    dev = "cuda:0"
    prod = ellipse_product_bound(w["sigma_max"], w["e_max"], 2, w["q_bits"], w["cmax"], device=dev)
    outs = []
    for dbg in (False, True):
        f = AdaptiveFilter(W, H, 2, torch.float32, scale_kind="ellipse", q_bits=w["q_bits"],
                           frac_bits=w["frac_bits"], max_scale=w["cmax"], out="f64",
                           value_bound=w["value_bound"], max_scale_product=prod, device=dev, debug_bounds=dbg)
        f.integrate(gu.to_device(img, dev))
        outs.append(f.filter(gu.to_device(sc.astype(np.float32), dev)).cpu().numpy())
        torch.cuda.synchronize()
        assert f.device_status() == 0
        if dbg:
            assert f.bounds_violation() == -1
        f.close()
    assert np.array_equal(outs[0], outs[1])



@pytest.mark.parametrize("n,shape,dtype", [(1, (300, 257), "u8"), (2, (257, 300), "f32"), (3, (130, 140), "u16")])
def test_repeated_runs_are_bit_identical(n, shape, dtype):
    """Race check without a sanitizer: ten integrate + filter runs of the same
    plan on the same input (several bands per line pass, so the look-back
    chains race each time) give bit-identical integrated images and
    numerators; the first run's numerators also equal the oracle's at
    sampled pixels."""
    import torch
    w = _small_workload(n, shape, 4 if n < 3 else 2, dtype, 90 + n)
    res = gu.run_exact(w, want=("num", "g"))
    filt = res["filt"]
    f_t = gu.to_device(w["image"], "cuda:0")
    s_t = gu.to_device(w["scales"].astype(np.float32), "cuda:0")
    for _ in range(9):
        filt.integrate(f_t)
        g = filt.integrated().cpu().numpy().astype(np.uint64)
        num = filt.numerators(s_t).cpu().numpy().astype(np.uint64)
        torch.cuda.synchronize()
        assert np.array_equal(g, res["g"])
        assert np.array_equal(num, res["num"])
    assert filt.device_status() == 0
    rng = np.random.default_rng(7)
    H, W = shape
    pix = [(int(rng.integers(0, W)), int(rng.integers(0, H))) for _ in range(24)]
    C_ref = gu.oracle_C(w)
    S_ref, _ = paper.filter_pixels(gu.f_int(w), C_ref, n, w["q_bits"], w["frac_bits"], pix)
    L = res["limbs"]
    mod = 1 << (64 * L)
    got = gu.wide_to_int(res["num"], L)
    for (x, y), S in zip(pix, S_ref):
        assert got[y * W + x] == int(S) % mod, (x, y)


@pytest.mark.parametrize("n,q", [(1, 4), (2, 4), (3, 2)])
def test_transpose_and_mirror_symmetries(n, q):
    """The dihedral symmetries of v1..v4 on the device path: transposing the
    image swaps a1 and a3, mirroring k1 swaps a2 and a4 (v2 = (1,1) mirrors to
    (-1,1) = v4).  The numerators are exact, so they must agree bit for bit:
    this also checks that the 3pi/4 pass' truncation at the box's right edge
    (which the mirror moves to the 45 degree pass) does not reach them."""
    w = _small_workload(n, (37, 53), q, "u8", 40 + n, lo=1.0, hi=5.0)
    base = gu.run_exact(w, want=("num",))
    img, sc = w["image"], w["scales"]
    wt = dict(w, image=np.ascontiguousarray(img.T), scales=np.ascontiguousarray(sc.transpose(1, 0, 2)[..., [2, 1, 0, 3]]))
    wm = dict(w, image=np.ascontiguousarray(img[:, ::-1]), scales=np.ascontiguousarray(sc[:, ::-1][..., [0, 3, 2, 1]]))
    rt = gu.run_exact(wt, want=("num",))
    rm = gu.run_exact(wm, want=("num",))
    assert base["status"] == rt["status"] == rm["status"] == 0
    assert base["limbs"] == rt["limbs"] == rm["limbs"]
    assert np.array_equal(rt["num"], base["num"].transpose(1, 0, 2))
    assert np.array_equal(rm["num"], base["num"][:, ::-1])


@pytest.mark.parametrize("n,dtype", [(1, "u8"), (2, "f32"), (3, "u16")])
def test_integrated_image_odd_size_several_bands(n, dtype):
    """An odd size (257 x 129) whose lattice box spans several 64-row bands of
    the line passes with a ragged last band, ragged groups of 32 lines and a
    ragged last row chunk: the integrated image equals the oracle's exact
    recursions at every cell where the GPU's is exact."""
    w = _small_workload(n, (257, 129), 3 if n < 3 else 2, dtype, 60 + n)
    res = gu.run_exact(w, want=("g",))
    assert res["status"] == 0
    _check_g(w, res)
