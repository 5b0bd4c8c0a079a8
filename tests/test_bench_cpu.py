"""Host-side pieces of bench.py, on CPU: the algorithmic unit of the mesh
roofline against the oracle's weights, the clock-record summary, the error
metric and the all-cores oracle sampler."""
import numpy as np
import pytest

import bench
from oracle import boxspline


@pytest.mark.parametrize("n", [1, 2, 3])
def test_mesh_macs_per_tap_is_the_mean_nonzero_weight_count(n):
    # (n+1)^4 taps x 7 n^2: the support octagon |x|, |y| < 3n/2, |x +- y| < 2n of
    # ZP^{*n} has area 7 n^2, so a tap at a uniformly distributed offset has
    # that many non-zero lattice weights on average.  Counted on the oracle's
    # integer weight rows over the whole 2^-P grid (P = 4): away from the knot
    # lines every offset has exactly 7 n^2 of them; grid points on the lines lose
    # the weights that vanish there, so the mean sits just below.
    P = 4
    wts = boxspline.ZPIntegerWeights(n, P)
    counts = [sum(1 for row in wts.row(rx, ry) for v in row if v != 0)
              for ry in range(1 << P) for rx in range(1 << P)]
    mean = float(np.mean(counts))
    assert 7 * n * n - 1.0 < mean <= 7 * n * n
    assert max(counts) == 7 * n * n
    assert bench._algorithmic_macs(n) == (n + 1) ** 4 * 7 * n * n


def test_clock_summary_takes_median_max_and_reasons():
    cs = bench.ClockSampler()
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 950.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = cs.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert bench.ClockSampler().summary()["reasons"] == ["unsampled"]


def test_err_range_is_relative_to_the_image_range():
    img = np.array([[0.0, 10.0], [5.0, 20.0]])
    out = np.array([[1.0, 10.0], [5.5, 20.0]])
    pts = [(0, 0), (0, 1)]          # (x, y)
    vals = [0.0, 5.0]
    assert bench.err_range(out, pts, vals, img) == pytest.approx(1.0 / 20.0)
    assert bench.err_range(out, [], [], img) is None


def test_all_cores_sampler_runs_the_oracle_in_spawned_processes():
    done, el, procs = bench.cpu_baseline_all_cores("c1", (48, 48), 0.5, procs=2)
    assert procs == 2 and done >= 2 and el >= 0.5
