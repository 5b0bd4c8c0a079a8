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
    res = dict(s=s, num=num, g=g, status=st, limbs=flt.limbs, right=flt.info["right"])
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
        g_or = o.running_sums(list(fi[r]), n2 + 1, length + res["right"])
        g_gpu = gu.wide_to_int(res["g"][r, : length + res["right"]], L)
        assert g_gpu == [v % mod for v in g_or], "row %d integrated signal" % r


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


def test_line1d_prefilter_degree_two_is_refused():
    from paper_0908_3861_gb300 import AdaptiveFilter1D, AbfError
    import torch
    with pytest.raises(AbfError):
        AdaptiveFilter1D(100, 2, 3, 1, torch.uint8, device="cuda:0")
