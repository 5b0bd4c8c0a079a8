"""GPU parity of the 1-D scale-adaptive B-spline filter (Sec. 3, Proposition
"prop") against the exact oracle, through the C ABI.

Bit-exact: the integrated signals g (modulo 2^(64 L)) and the numerators S.
Floating point: s = S / Den within 1e-13 relative (binary64 division).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import synthetic
from oracle import line1d as o
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _signals(dtype, count, length, rng, frac_bits):
    if dtype == "u8":
        return rng.integers(0, 256, (count, length)).astype(np.uint8), 0, 255.0
    if dtype == "u16":
        return rng.integers(0, 65536, (count, length)).astype(np.uint16), 0, 65535.0
    if dtype == "f64":
        return rng.integers(-400, 400, (count, length)).astype(np.float64), 0, 400.0
    f = synthetic.signals_1d(rng, count, length, smooth=8.0, steps=3, frac_bits=frac_bits)
    return f, frac_bits, 255.0


def _run(f, a, n1, n2, q, F, vb, amax, want_g=False):
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter1D
    count, length = f.shape
    flt = AdaptiveFilter1D(length, count, n1, n2, gu.torch_dtype(f.dtype), q_bits=q, frac_bits=F, max_scale=amax,
                           value_bound=vb, out="f64", device="cuda:0")
    ft = gu.to_device(f, "cuda:0")
    at = torch.from_numpy(a.astype(np.float32)).to("cuda:0")
    flt.integrate(ft)
    s = flt.filter(at).cpu().numpy()
    num = flt.numerators(at).cpu().numpy().astype(np.uint64)
    g = flt.integrated().cpu().numpy().astype(np.uint64) if want_g else None
    st = flt.device_status()
    res = dict(s=s, num=num, g=g, status=st, limbs=flt.limbs, right=flt.info["right"], left=flt.info["left"])
    flt.close()
    return res


def _fint(f, F):
    return (f.astype(np.float64) * float(1 << F)).astype(np.int64)


CASES = [
    (0, 0, 3, "u8", 3, 37),
    (0, 2, 2, "f64", 2, 50),
    (1, 1, 4, "u16", 4, 70),
    (1, 3, 3, "f32", 3, 65),
    (1, 2, 5, "u8", 1, 1),
    (1, 3, 2, "u8", 5, 300),
    (0, 3, 8, "f32", 2, 530),
]


@pytest.mark.parametrize("n1,n2,q,dtype,count,length", CASES)
def test_line1d_all_samples_bit_exact(n1, n2, q, dtype, count, length):
    rng = np.random.default_rng(500 + 10 * n1 + n2 + length)
    f, F, vb = _signals(dtype, count, length, rng, 8)
    amax = 9.0
    a = rng.uniform(0.4, amax, (count, length)).astype(np.float32)
    res = _run(f, a, n1, n2, q, F, vb, amax, want_g=True)
    assert res["status"] == 0
    L = res["limbs"]
    mod = 1 << (64 * L)
    fi = _fint(f, F)
    for r in range(count):
        A = o.quantise(a[r], q)
        S, s = o.filter_paper(list(fi[r]), A, n1, n2, q, F)
        got = gu.wide_to_int(res["num"][r], L)
        assert got == [v % mod for v in S], "row %d numerators" % r
        ref = np.array([float(v) for v in s])
        gu.assert_close_f64(res["s"][r], ref, rel=1e-13, absol=1e-300)
        left = res["left"]
        g_or = o.running_sums(list(fi[r]), n2 + 1, length + res["right"])
        g_gpu = gu.wide_to_int(res["g"][r, : left + length + res["right"]], L)
        assert g_gpu[:left] == [0] * left, "row %d zeros before the signal" % r
        assert g_gpu[left:] == [v % mod for v in g_or], "row %d integrated signal" % r


def test_line1d_invalid_scales_are_flagged():
    rng = np.random.default_rng(9)
    f = rng.integers(0, 256, (2, 40)).astype(np.uint8)
    a = rng.uniform(1.0, 4.0, (2, 40)).astype(np.float32)
    a[0, 3], a[0, 7], a[1, 20], a[1, 30] = np.nan, -1.0, 0.0, 100.0
    res = _run(f, a, 1, 1, 4, 0, 255.0, 4.0)
    assert res["status"] & 1
    bad = {(0, 3), (0, 7), (1, 20), (1, 30)}
    for r in range(2):
        A = o.quantise(np.where(np.isfinite(a[r]) & (a[r] > 0) & (a[r] <= 4.0), a[r], 1.0), 4)
        _, s = o.filter_paper(list(f[r].astype(np.int64)), A, 1, 1, 4)
        for m in range(40):
            if (r, m) in bad:
                assert np.isnan(res["s"][r, m])
            else:
                assert res["s"][r, m] == pytest.approx(float(s[m]), rel=1e-13, abs=1e-300)


def test_line1d_bench_recipe_sampled():
    """The 1-D workload recipe (float32 on the 2^-16 grid, n1 = 1, n2 = 3,
    a in [1, 64]) at 8 x 65536, checked on sampled samples of every row."""
    rng = np.random.default_rng(synthetic.SEED_BASE + 5)
    count, length = 8, 65536
    f = synthetic.signals_1d(rng, count, length)
    a = synthetic.scales_1d(rng, count, length, 1.0, 64.0, 2048.0)
    res = _run(f, a, 1, 3, 8, 16, 255.0, 64.0)
    assert res["status"] == 0
    L = res["limbs"]
    mod = 1 << (64 * L)
    fi = _fint(f, 16)
    pick = np.random.default_rng(1)
    for r in range(count):
        ms = sorted(set([0, 1, length - 1, length - 2] + list(pick.integers(0, length, 60))))
        A = o.quantise(a[r], 8)
        S, s = o.filter_paper_at(list(fi[r]), A, 1, 3, 8, 16, ms)
        got = gu.wide_to_int(res["num"][r][ms], L)
        assert got == [v % mod for v in S]
        for m, v in zip(ms, s):
            assert res["s"][r, m] == pytest.approx(float(v), rel=1e-13)


def test_line1d_model_degree_six_is_refused():
    from paper_0908_3861_gb300 import AdaptiveFilter1D, AbfError
    import torch
    with pytest.raises(AbfError):
        AdaptiveFilter1D(100, 2, 6, 1, torch.uint8, device="cuda:0")


# ------------------------------------------------ prefiltered models (n1 >= 2)
# The GPU rounds c = f * (b^{n1})^-1 to the 2^-F grid from a fixed-point
# recursion whose error is far below the grid (about 2^-46 |f 2^F| steps), the
# oracle from c kept to 2^-200.  Where c 2^F lies within TIE of a rounding tie
# either neighbour is a valid c_q; elsewhere c_q is unique and everything
# downstream (g, S) is compared bit for bit.  s is always compared with the
# definition on the exact c: |s - s(c)| <= 2^-(F+1) (unit-sum non-negative
# kernel) + the prefilter error + the binary64 division.

TIE = 2.0 ** -16


def _ties(cs, bits=200):
    """Positions whose c 2^F is within TIE of a half-integer."""
    half = 1 << (bits - 1)
    one = 1 << bits
    tol = int(TIE * one)
    return {i for i, v in enumerate(cs) if abs((v % one) - half) <= tol}


def _diffs(g, times, mod):
    """Backward differences of g, `times` times (the inverse of the running sums)."""
    x = list(g)
    for _ in range(times):
        x = [(x[i] - (x[i - 1] if i else 0)) % mod for i in range(len(x))]
    return [v - mod if v >= mod // 2 else v for v in x]


PF_CASES = [
    (2, 0, 3, "u8", 3, 37),
    (3, 1, 4, "f32", 2, 9000),
    (3, 0, 2, "f64", 2, 300),
    (4, 1, 3, "u16", 2, 300),
    (5, 0, 3, "u8", 2, 4097),
    (2, 2, 5, "f32", 1, 1),
]


@pytest.mark.parametrize("n1,n2,q,dtype,count,length", PF_CASES)
def test_line1d_prefiltered_model(n1, n2, q, dtype, count, length):
    rng = np.random.default_rng(900 + 10 * n1 + n2 + length)
    f, F, vb = _signals(dtype, count, length, rng, 8)
    if dtype != "f32":
        F = 6  # integer samples lie on every 2^-F grid; c_q gets 6 fraction bits
    amax = 9.0
    a = rng.uniform(0.4, amax, (count, length)).astype(np.float32)
    res = _run(f, a, n1, n2, q, F, vb, amax, want_g=True)
    assert res["status"] == 0
    L, left, right = res["limbs"], res["left"], res["right"]
    mod = 1 << (64 * L)
    fi = _fint(f, F)
    pick = np.random.default_rng(2)
    for r in range(count):
        x = [int(v) for v in fi[r]]
        kf, cs = o.prefilter(x, n1)
        kq, cq = o.prefilter_quantised(x, n1)
        # the GPU's tail bound: every c_q before -left is zero
        assert all(v == 0 for v in cq[: -left - kq]), "c_q beyond the left margin"
        ties = {kf + i for i in _ties(cs)}
        # c_q as the GPU used it: the differences of its running sums
        g_gpu = gu.wide_to_int(res["g"][r, : left + length + right], L)
        c_gpu = _diffs(g_gpu, n2 + 1, mod)
        for i, v in enumerate(c_gpu):
            k = i - left
            want = cq[k - kq]
            if k in ties:
                lo = (cs[k - kf] >> 200)
                assert v in (lo, lo + 1), k
            else:
                assert v == want, (r, k, v, want)
        A = o.quantise(a[r], q)
        if not [k for k in ties if -left <= k < length + right]:
            S, s = o.filter_paper(cq, A, n1, n2, q, F, k_first=kq)
            got = gu.wide_to_int(res["num"][r], L)
            assert got == [v % mod for v in S], "row %d numerators" % r
            gu.assert_close_f64(res["s"][r], np.array([float(v) for v in s]), rel=1e-13, absol=1e-300)
        ms = sorted(set([0, length - 1] + [int(v) for v in pick.integers(0, length, 24)]))
        sd = o.filter_direct([Fr(v, 1 << (200 + F)) for v in cs], A, n2, q, n1, k_first=kf, ms=ms)
        bound = 2.0 ** -(F + 1) * (1 + 2 * TIE) + 1e-12 * vb
        for m, v in zip(ms, sd):
            assert abs(res["s"][r, m] - float(v)) <= bound, (r, m)


def test_line1d_prefiltered_cubic_model_recipe_sampled():
    """The 1-D workload recipe (float32 on the 2^-16 grid, a in [1, 64]) with a
    cubic signal model (n1 = 3, n2 = 1) at 4 x 65536, sampled per row."""
    rng = np.random.default_rng(synthetic.SEED_BASE + 6)
    count, length = 4, 65536
    f = synthetic.signals_1d(rng, count, length)
    a = synthetic.scales_1d(rng, count, length, 1.0, 64.0, 2048.0)
    res = _run(f, a, 3, 1, 8, 16, 255.0, 64.0)
    assert res["status"] == 0
    L = res["limbs"]
    mod = 1 << (64 * L)
    fi = _fint(f, 16)
    pick = np.random.default_rng(4)
    for r in range(count):
        x = [int(v) for v in fi[r]]
        kf, cs = o.prefilter(x, 3)
        kq, cq = o.prefilter_quantised(x, 3)
        ms = sorted(set([0, 1, length - 1, length - 2] + [int(v) for v in pick.integers(0, length, 40)]))
        A = o.quantise(a[r], 8)
        if not _ties(cs):
            S, s = o.filter_paper_at(cq, A, 3, 1, 8, 16, ms, k_first=kq)
            got = gu.wide_to_int(res["num"][r][ms], L)
            assert got == [v % mod for v in S]
            for m, v in zip(ms, s):
                assert res["s"][r, m] == pytest.approx(float(v), rel=1e-13)
        sd = o.filter_direct([Fr(v, 1 << 216) for v in cs], A, 1, 8, 3, k_first=kf, ms=ms[:12])
        for m, v in zip(ms[:12], sd):
            assert abs(res["s"][r, m] - float(v)) <= 2.0 ** -17 * (1 + 2 * TIE) + 1e-12 * 255.0
