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
    return sorted(set(re.findall(r"\b(abf_[a-z0-9_]+)\s*\(", src)))


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


def test_status_strings(lib):
    from paper_0908_3861_gb300 import _abf
    assert _abf.abf_status_str(0) == "ok"
    assert _abf.abf_version() >= 1


@pytest.mark.parametrize("n,q", [(1, 3), (1, 8), (2, 3), (2, 8), (3, 2)])
def test_host_weight_table_equals_oracle(lib, n, q):
    """Library: refinement cascade of the box spline in exact integers.
    Oracle: de Boor's recurrence on polynomial pieces.  Same table, same D."""
    from paper_0908_3861_gb300 import _abf
    from oracle.boxspline import ZPIntegerWeights
    raw, wb, D = _abf.abf_weight_table_host(n, q)
    P = q if n % 2 == 0 else q + 1
    zw = ZPIntegerWeights(n, P)
    assert D == zw.D
    n3 = 3 * n
    if wb == 16:
        w = np.frombuffer(raw, dtype=np.uint64).reshape(-1, 2)
        vals = [int(a) + (int(b) << 64) for a, b in w]
    else:
        vals = [int(v) for v in np.frombuffer(raw, dtype=np.uint32 if wb == 4 else np.uint64)]
    rows = (1 << P) ** 2
    assert len(vals) == rows * n3 * n3
    rng = np.random.default_rng(n * 100 + q)
    idx = range(rows) if rows <= 256 else rng.integers(0, rows, 60)
    for r in idx:
        r = int(r)
        ref = [v for line in zw.row(r % (1 << P), r >> P) for v in line]
        assert vals[r * n3 * n3:(r + 1) * n3 * n3] == ref


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
