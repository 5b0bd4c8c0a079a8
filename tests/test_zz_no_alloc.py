"""abf_integrate_noalloc: the integration step for callers that cannot
allocate device memory themselves (a serving loop whose memory was all
reserved up front, or code that must not trigger the device synchronisation a
cudaMalloc / cudaFree can cause).  It keeps its look-back scratch in a fixed
32 MiB array inside the library instead of a caller workspace.

Checked here through the C ABI against abf_integrate, the entry point that
takes a workspace: the integrated image must be bit-identical (it is integer
data), on two calls in a row, and so must the filtered output computed from
it.  Plans that need more than the fixed scratch are refused.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0908_3861_gb300 import _abf
    return _abf


def test_noalloc_integrate_equals_workspace_integrate_twice(lib):
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter
    rng = np.random.default_rng(77)
    H, W = 300, 420
    img = synthetic.image_f32_grid(rng, (H, W), 12.0, 6, 16)
    sc = synthetic.ellipse_field(rng, (H, W), sig=(1.0, 6.0), elong=(1.0, 3.0))
    dev = torch.device("cuda:0")
    filt = AdaptiveFilter(W, H, 2, torch.float32, scale_kind="ellipse", q_bits=8, frac_bits=16, max_scale=40.0,
                          out="f64", value_bound=255.0, device=dev)
    f_t = torch.from_numpy(img).to(dev)
    s_t = torch.from_numpy(sc).to(dev)
    left, right, _, above = filt.info["halo_lrbt"]
    gw = W + left + right

    filt.integrate(f_t)
    g_ref = filt.integrated()[:, :gw].clone()
    s_ref = filt.filter(s_t).clone()
    torch.cuda.synchronize()
    g_ws = filt.g

    for call in range(2):
        g_new = torch.full_like(g_ws, 0xA5)      # stale bytes the call must overwrite
        lib.abf_integrate_noalloc(filt.plan, f_t, W * 4, g_new)
        filt.g = g_new
        torch.cuda.synchronize()
        assert torch.equal(filt.integrated()[:, :gw], g_ref), "integrated image differs on call %d" % call
        s_new = filt.filter(s_t)
        torch.cuda.synchronize()
        assert torch.equal(s_new, s_ref), "filtered output differs on call %d" % call
    assert filt.device_status() == 0
    filt.g = g_ws
    filt.close()


def test_noalloc_integrate_refuses_plans_beyond_the_fixed_scratch(lib):
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter
    filt = AdaptiveFilter(8192, 8192, 1, torch.uint8, scale_kind="a4", q_bits=8, max_scale=8.0, out="f32",
                          device="cuda:0")
    assert filt.info["workspace_bytes"] > 32 << 20
    f_t = torch.zeros((8192, 8192), dtype=torch.uint8, device="cuda:0")
    with pytest.raises(lib.AbfError) as e:
        lib.abf_integrate_noalloc(filt.plan, f_t, 8192, filt.g)
    assert e.value.status == 4   # ABF_ERR_UNSUPPORTED
    filt.close()
