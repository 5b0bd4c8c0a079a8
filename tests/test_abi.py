"""The C-ABI library builds, loads and exports every entry point include/abf.h
declares; its host-side ZP^{*n} weight table equals the oracle's exact
weights (no GPU needed for either)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "abf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(abf(?:1d)?_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0908_3861_gb300 import _abf
    return _abf.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_fault_injection_arguments(lib):
    """abf_debug_inject_fault takes the three kinds and a count >= 0 (host
    only: arming and disarming touch no device)."""
    from paper_0908_3861_gb300 import _abf
    assert lib.abf_debug_inject_fault(0, 1) == _abf.ABF_ERR_INVALID
    assert lib.abf_debug_inject_fault(4, 1) == _abf.ABF_ERR_INVALID
    assert lib.abf_debug_inject_fault(_abf.ABF_FAULT_ALLOC, -1) == _abf.ABF_ERR_INVALID
    for k in (_abf.ABF_FAULT_ALLOC, _abf.ABF_FAULT_QUEUE_STALL, _abf.ABF_FAULT_BAD_DESC):
        assert lib.abf_debug_inject_fault(k, 3) == _abf.ABF_OK
        assert lib.abf_debug_inject_fault(k, 0) == _abf.ABF_OK


def test_status_strings(lib):
    from paper_0908_3861_gb300 import _abf
    assert _abf.abf_status_str(0) == "ok"
    assert _abf.abf_version() >= 1


def _stencil(n):
    """Neighbours d of a tap that can carry a non-zero ZP^{*n} weight: the box
    of r - d (r in [0,1)^2 for even n, [-1/2,1/2)^2 for odd n) must meet the
    open octagon |x|,|y| < 3n/2, |x +- y| < 2n."""
    dmin = -(3 * n) // 2 + 1 if n % 2 == 0 else -(3 * n - 1) // 2
    lo = 0.0 if n % 2 == 0 else -0.5
    out = []
    for iy in range(3 * n):
        for ix in range(3 * n):
            dx, dy = dmin + ix, dmin + iy
            x0, x1, y0, y1 = lo - dx, lo - dx + 1, lo - dy, lo - dy + 1
            if (x0 < 1.5 * n and -1.5 * n < x1 and y0 < 1.5 * n and -1.5 * n < y1
                    and x0 + y0 < 2 * n and -2 * n < x1 + y1 and x0 - y1 < 2 * n and -2 * n < x1 - y0):
                out.append((ix, iy))
    return out


@pytest.mark.parametrize("n,q", [(1, 3), (1, 8), (2, 3), (2, 8), (3, 2)])
def test_host_weight_table_equals_oracle(lib, n, q):
    """Library: refinement cascade of the box spline in exact integers.
    Oracle: de Boor's recurrence on polynomial pieces.  Same weights, same D;
    the neighbours the library drops carry zero weight in the oracle."""
    from paper_0908_3861_gb300 import _abf
    from oracle.boxspline import ZPIntegerWeights
    raw, wb, D = _abf.abf_weight_table_host(n, q)
    P = q if n % 2 == 0 else q + 1
    zw = ZPIntegerWeights(n, P)
    assert D == zw.D
    st = _stencil(n)
    assert len(st) == {1: 9, 2: 32, 3: 69}[n]
    if wb == 16:
        w = np.frombuffer(raw, dtype=np.uint64).reshape(-1, 2)
        vals = [int(a) + (int(b) << 64) for a, b in w]
    else:
        vals = [int(v) for v in np.frombuffer(raw, dtype=np.uint32 if wb == 4 else np.uint64)]
    rows = (1 << P) ** 2
    R = len(st)
    assert len(vals) == rows * R
    rng = np.random.default_rng(n * 100 + q)
    idx = range(rows) if rows <= 256 else rng.integers(0, rows, 60)
    for r in idx:
        r = int(r)
        full = zw.row(r % (1 << P), r >> P)
        assert vals[r * R:(r + 1) * R] == [full[iy][ix] for ix, iy in st]
        kept = set(st)
        assert all(full[iy][ix] == 0 for iy in range(3 * n) for ix in range(3 * n) if (ix, iy) not in kept)


def test_plan_rejects_bad_descriptors(lib):
    from paper_0908_3861_gb300 import _abf
    d = _abf.abf_desc()
    d.width, d.height, d.order_n = 16, 16, 4          # order out of range
    d.in_dtype, d.out_dtype, d.form, d.scale_kind = 0, 3, 0, 0
    d.q_bits, d.max_scale = 4, 4.0
    with pytest.raises(_abf.AbfError) as e:
        _abf.abf_plan_create(d)
    assert e.value.status == 1
    d.order_n = 1
    d.width = 0
    with pytest.raises(_abf.AbfError):
        _abf.abf_plan_create(d)


@pytest.mark.parametrize("n1,n2,q", [(0, 0, 3), (1, 1, 2), (0, 2, 4), (1, 3, 3), (1, 2, 8), (3, 1, 8), (5, 0, 3)])
def test_line1d_host_table_matches_oracle(n1, n2, q):
    """The 1-D B-spline table (built by the degree recurrence) against the
    oracle's truncated-power B-spline, entry by entry."""
    from oracle import line1d as o
    from paper_0908_3861_gb300 import _abf
    rows, dmin, D = _abf.abf1d_weight_table_host(n1, n2, q)
    N, P = n1 + n2 + 1, q + 1
    assert D == o.denominator(N, P)
    assert len(rows) == 1 << P
    for R, row in enumerate(rows):
        ref = [o.dbspline_int(N, P, R - ((dmin + c) << P)) for c in range(len(row))]
        assert row == ref, R
        assert sum(row) == D


@pytest.mark.parametrize("n1", [2, 3, 4, 5])
def test_line1d_prefilter_constants_match_the_oracle_inverse(n1):
    """The poles and weights the 1-D plan derives for the interpolation
    prefilter (partial fractions of the B-spline filter's symbol, binary64)
    against the oracle's inverse from its definition (exact banded solve)."""
    from oracle import line1d as o
    from paper_0908_3861_gb300 import _abf
    z, A, hnorm = _abf.abf1d_prefilter_host(n1)
    assert len(z) == n1 // 2 and all(-1.0 < p < 0.0 for p in z)
    h = o.inverse_filter(n1)
    h0 = float(h[0])
    for k in range(0, 25):
        got = sum(a * p ** k for a, p in zip(A, z))
        assert abs(got - float(h[k])) <= 4e-16 * abs(h0) * (k + 1), k
    l1 = sum(abs(float(h[k])) for k in range(-60, 61))
    assert l1 <= hnorm * (1 + 1e-12)
    with pytest.raises(_abf.AbfError):
        _abf.abf1d_prefilter_host(6)


def _c_kind(param):
    p = " ".join(param.replace("const", " ").split())
    if "*" in p or p.split()[0] in ("abf_plan", "abf1d_plan", "abf_server", "cudaStream_t"):
        return "ptr"
    t = p.split()[0]
    return {"double": "f64", "float": "f32", "size_t": "u64", "uint64_t": "u64", "int64_t": "i64",
            "int32_t": "i32", "uint32_t": "i32", "abf_dtype": "i32", "abf_status": "i32", "int": "i32"}[t]


def _ctypes_kind(t):
    import ctypes
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and not isinstance(t._type_, str):
        return "ptr"
    return {ctypes.c_double: "f64", ctypes.c_float: "f32", ctypes.c_size_t: "u64", ctypes.c_uint64: "u64",
            ctypes.c_int64: "i64", ctypes.c_int32: "i32", ctypes.c_uint32: "i32", ctypes.c_int: "i32"}[t]


def test_binding_signatures_match_the_header():
    """Every entry point's parameter list in include/abf.h against the ctypes
    argtypes the binding installs: same count, same kinds (pointer, integer
    width, floating type), so the two cannot drift apart silently."""
    from paper_0908_3861_gb300 import _abf
    src = open(os.path.join(ROOT, "include", "abf.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    decls = dict(re.findall(r"\b(abf(?:1d)?_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src))
    sigs = _abf.signatures()
    assert set(sigs) == set(decls)
    for name, params in decls.items():
        plist = [q.strip() for q in params.split(",") if q.strip() and q.strip() != "void"]
        args, _ = sigs[name]
        assert len(args) == len(plist), name
        assert [_c_kind(q) for q in plist] == [_ctypes_kind(a) for a in args], name


def test_plan_refuses_forms_that_cannot_meet_their_tolerance(lib):
    """Host-side checks of abf_plan_create that come before any device call:
    binary32 pairs are refused beyond order 1 (their error bound exceeds 1e-5
    of the value range there), and float inputs need a value bound (it sizes
    the exact form's limbs and the floating-point forms' tolerance)."""
    import ctypes
    import torch
    from paper_0908_3861_gb300 import _abf, make_desc
    plan = ctypes.c_void_p()
    for n in (2, 3):
        d = make_desc(64, 64, n, torch.float32, form="tile_f32", q_bits=4, frac_bits=16, max_scale=8.0,
                      value_bound=255.0)
        assert lib.abf_plan_create(ctypes.byref(d), ctypes.byref(plan)) == _abf.ABF_ERR_UNSUPPORTED
    for form in ("exact", "plain_f64", "tile_f32"):
        d = make_desc(64, 64, 1, torch.float32, form=form, q_bits=4, frac_bits=16, max_scale=8.0, value_bound=0.0)
        assert lib.abf_plan_create(ctypes.byref(d), ctypes.byref(plan)) == _abf.ABF_ERR_INVALID


@pytest.mark.parametrize("directions,n,E,q", [(2, 2, 0, 2), (2, 3, 0, 1), (4, 1, 1, 2), (4, 1, 2, 2), (2, 1, 2, 2),
                                              (4, 1, 4, 1)])
def test_general_table_equals_oracle(lib, directions, n, E, q):
    """Generalised interpolation tables (N = 2, B-spline models): the library's
    refinement cascade against the oracle's de Boor pieces (oracle.general),
    every row and every neighbour; D the same; neighbours outside the listed
    stencil carry no weight (rows sum to D)."""
    from paper_0908_3861_gb300 import _abf
    from oracle import general
    rows, stencil, D, wb = _abf.abf_general_table_host(directions, n, E, q)
    r = (n, n if directions == 4 else 0, n, n if directions == 4 else 0)
    mw = general.MeshWeights(general.interp_counts(r, E - 1 if E else None), q + 1)
    assert D == mw.D
    P = q + 1
    one = 1 << P
    for ry in range(one):
        for rx in range(one):
            row = rows[ry * one + rx]
            assert sum(row) == D
            for (dx, dy), w in zip(stencil, row):
                assert w == mw.value(rx - (dx << P), ry - (dy << P)), (rx, ry, dx, dy)
