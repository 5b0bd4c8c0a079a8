"""Serving loop (abf_server_*): jobs from host memory, admitted by device
memory footprint into a bounded number of concurrent slots.  Each result must
equal the same job filtered alone (bit for bit), device memory must stay
within the budget, a resident integrated image must be reused, and a bounded
wait must time out (and the job still finish) when admission is paused."""
import numpy as np
import pytest

import synthetic
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _job(seed, h, w, n):
    r = np.random.default_rng(seed)
    img = synthetic.image_f32_grid(r, (h, w), 6.0, 4, 16)
    sc = synthetic.ellipse_field(r, (h, w), sig=(1.0, 5.0), elong=(1.0, 3.0))
    return img, sc, n


def _alone(img, sc, n):
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter
    H, W = img.shape
    f = AdaptiveFilter(W, H, n, torch.float32, scale_kind="ellipse", q_bits=6, frac_bits=16, max_scale=20.0,
                       out="f32", value_bound=255.0, device="cuda:0")
    out = f(gu.to_device(img, "cuda:0"), gu.to_device(sc, "cuda:0")).cpu()
    f.close()
    return out


def _desc(img, n):
    import torch
    from paper_0908_3861_gb300 import make_desc
    H, W = img.shape
    return make_desc(W, H, n, torch.float32, scale_kind="ellipse", q_bits=6, frac_bits=16, max_scale=20.0,
                     out="f32", value_bound=255.0)


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.mark.parametrize("group", [False, True])
def test_mixed_jobs_equal_single_runs_within_budget(group):
    import torch
    from paper_0908_3861_gb300 import Server
    jobs = [_job(100 + i, int(h), int(w), n) for i, (h, w, n) in
            enumerate([(40, 70, 1), (90, 33, 2), (64, 64, 2), (17, 120, 1), (50, 50, 2), (75, 40, 1), (33, 90, 2)])]
    budget = 256 << 20
    srv = Server(budget, max_inflight=3, device="cuda:0", group_mesh=group)
    tickets, outs = [], []
    for img, sc, n in jobs:
        o = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
        tickets.append(srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o))
        outs.append(o)
    for t in tickets:
        st = srv.wait(t, timeout_s=120)
        assert st["status"] == 0 and st["device_status"] == 0
        assert st["t_submit_us"] <= st["t_admit_us"] <= st["t_done_us"]
    for (img, sc, n), o in zip(jobs, outs):
        assert torch.equal(o, _alone(img, sc, n))
    assert srv.stats()["peak"] <= budget
    srv.close()


def test_small_budget_serialises_but_stays_correct():
    import torch
    from paper_0908_3861_gb300 import Server
    jobs = [_job(200 + i, 60, 80, 2) for i in range(4)]
    # room for one job at a time (one 60x80 order-2 job holds about 0.6 MB)
    srv = Server(1 << 20, max_inflight=4, device="cuda:0")
    outs, tickets = [], []
    for img, sc, n in jobs:
        o = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
        tickets.append(srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o))
        outs.append(o)
    for t in tickets:
        assert srv.wait(t, timeout_s=120)["status"] == 0
    assert srv.stats()["peak"] <= 1 << 20
    for (img, sc, n), o in zip(jobs, outs):
        assert torch.equal(o, _alone(img, sc, n))
    srv.close()


def test_resident_integrated_image_is_reused():
    import torch
    from paper_0908_3861_gb300 import Server
    img, sc, n = _job(300, 70, 90, 2)
    _, sc2, _ = _job(301, 70, 90, 2)
    srv = Server(256 << 20, max_inflight=2, device="cuda:0")
    o1 = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
    o2 = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
    t1 = srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o1, image_id=42)
    assert srv.wait(t1, timeout_s=60)["resident_hit"] == 0
    t2 = srv.submit(_desc(img, n), None, _pinned(sc2), o2, image_id=42)
    st = srv.wait(t2, timeout_s=60)
    assert st["resident_hit"] == 1
    assert torch.equal(o1, _alone(img, sc, n))
    assert torch.equal(o2, _alone(img, sc2, n))
    assert srv.stats()["resident"] == 1
    srv.close()


def test_bounded_wait_times_out_then_completes():
    import torch
    from paper_0908_3861_gb300 import Server, AbfError
    img, sc, n = _job(400, 40, 40, 1)
    srv = Server(64 << 20, max_inflight=1, device="cuda:0")
    srv.pause(True)
    o = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
    t = srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o)
    with pytest.raises(AbfError) as e:
        srv.wait(t, timeout_s=0.1)
    assert e.value.status == 6   # ABF_ERR_TIMEOUT
    assert srv.stats()["queued"] == 1
    srv.pause(False)
    assert srv.wait(t, timeout_s=60)["status"] == 0
    assert torch.equal(o, _alone(img, sc, n))
    srv.close()


def test_job_larger_than_budget_is_refused():
    import torch
    from paper_0908_3861_gb300 import Server, AbfError
    img, sc, n = _job(500, 200, 200, 2)
    srv = Server(1 << 20, max_inflight=1, device="cuda:0")
    o = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
    with pytest.raises(AbfError) as e:
        srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o)
    assert e.value.status == 7   # ABF_ERR_BUSY
    srv.close()


def test_device_status_is_per_job_not_per_descriptor():
    """A job with an invalid scale raises its own status bit; the next job
    with the same descriptor (so the same plan) starts from a clear word."""
    import torch
    from paper_0908_3861_gb300 import Server
    img, sc, n = _job(600, 48, 64, 2)
    bad = sc.copy()
    bad[5, 7, 0] = np.nan   # sigma not finite: ABF_DEV_BAD_SCALE for that pixel
    srv = Server(64 << 20, max_inflight=1, device="cuda:0")
    o1 = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
    o2 = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
    t1 = srv.submit(_desc(img, n), _pinned(img), _pinned(bad), o1)
    t2 = srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o2)
    s1 = srv.wait(t1, timeout_s=60)
    s2 = srv.wait(t2, timeout_s=60)
    assert s1["status"] == 0 and s1["device_status"] == 1
    assert torch.isnan(o1[5, 7]) and int(torch.isnan(o1).sum()) == 1
    assert s2["status"] == 0 and s2["device_status"] == 0
    assert torch.equal(o2, _alone(img, sc, n))
    srv.close()


def _footprint(img, n, hit):
    """Device bytes the server charges for a job (f32 image, f32 output)."""
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter
    H, W = img.shape
    f = AdaptiveFilter(W, H, n, torch.float32, scale_kind="ellipse", q_bits=6, frac_bits=16, max_scale=20.0,
                       out="f32", value_bound=255.0, device="cuda:0")
    g, ws = f.info["integrated_bytes"], f.info["workspace_bytes"]
    f.close()
    return H * W * (16 + 4) + (0 if hit else H * W * 4 + g + ws), g


def test_resident_image_named_at_submit_survives_a_later_eviction():
    """A request without an image (h_f = NULL) holds its resident image from
    submit on.  Here a job queued before it needs the room that image takes:
    that job must wait for the resident job instead of evicting its image."""
    import torch
    from paper_0908_3861_gb300 import Server
    img_a, sc_a, n = _job(700, 64, 64, 2)
    _, sc_b, _ = _job(701, 64, 64, 2)
    img_c, sc_c, _ = _job(702, 64, 64, 2)
    need_c, g_a = _footprint(img_c, n, hit=False)
    need_b, _ = _footprint(img_a, n, hit=True)
    budget = need_c           # C alone fits; C beside the resident image does not
    assert g_a + need_b <= budget < g_a + need_c
    srv = Server(budget, max_inflight=2, device="cuda:0")
    oa = torch.zeros(img_a.shape, dtype=torch.float32).pin_memory()
    assert srv.wait(srv.submit(_desc(img_a, n), _pinned(img_a), _pinned(sc_a), oa, image_id=9),
                    timeout_s=60)["status"] == 0
    assert srv.stats()["resident"] == 1
    srv.pause(True)
    oc = torch.zeros(img_c.shape, dtype=torch.float32).pin_memory()
    ob = torch.zeros(img_a.shape, dtype=torch.float32).pin_memory()
    tc = srv.submit(_desc(img_c, n), _pinned(img_c), _pinned(sc_c), oc)
    tb = srv.submit(_desc(img_a, n), None, _pinned(sc_b), ob, image_id=9)
    srv.pause(False)
    sb = srv.wait(tb, timeout_s=60)
    sc_ = srv.wait(tc, timeout_s=60)
    assert sb["status"] == 0 and sb["resident_hit"] == 1
    assert sc_["status"] == 0
    assert torch.equal(ob, _alone(img_a, sc_b, n))
    assert torch.equal(oc, _alone(img_c, sc_c, n))
    assert srv.stats()["peak"] <= budget
    srv.close()


def test_concurrent_jobs_overlap_on_the_device():
    """With two slots, two long jobs submitted together are on the device at
    the same time: their device-clock intervals (CUDA events on their own
    streams) intersect, and each result equals the job run alone."""
    import torch
    from paper_0908_3861_gb300 import Server
    jobs = [_job(800 + i, 512, 512, 2) for i in range(2)]
    srv = Server(1 << 30, max_inflight=2, device="cuda:0")
    outs, tickets = [], []
    for img, sc, n in jobs:
        o = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
        tickets.append(srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o))
        outs.append(o)
    st = [srv.wait(t, timeout_s=120) for t in tickets]
    for s in st:
        assert s["status"] == 0 and s["t_gpu_end_us"] > s["t_gpu_start_us"] > 0
    a, b = st
    assert a["t_gpu_start_us"] < b["t_gpu_end_us"] and b["t_gpu_start_us"] < a["t_gpu_end_us"]
    for (img, sc, n), o in zip(jobs, outs):
        assert torch.equal(o, _alone(img, sc, n))
    srv.close()


def test_grouped_launch_keeps_results_and_status_per_job():
    """Jobs admitted in one round (submitted while paused) share one batched
    launch of the adaptive step: every result equals the job run alone, and
    the one job with an invalid scale is the only one whose status shows it."""
    import torch
    from paper_0908_3861_gb300 import Server
    specs = [(40, 70, 1), (90, 33, 2), (64, 64, 2), (17, 120, 1), (50, 50, 2)]
    jobs = [_job(900 + i, h, w, n) for i, (h, w, n) in enumerate(specs)]
    img2, sc2, n2 = jobs[2]
    bad = sc2.copy()
    bad[3, 4, 0] = np.nan
    jobs[2] = (img2, bad, n2)
    srv = Server(256 << 20, max_inflight=len(jobs), device="cuda:0", group_mesh=True)
    srv.pause(True)
    outs, tickets = [], []
    for img, sc, n in jobs:
        o = torch.zeros(img.shape, dtype=torch.float32).pin_memory()
        tickets.append(srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o))
        outs.append(o)
    srv.pause(False)
    st = [srv.wait(t, timeout_s=120) for t in tickets]
    assert all(s["status"] == 0 for s in st)
    assert [s["device_status"] for s in st] == [0, 0, 1, 0, 0]
    for k, ((img, sc, n), o) in enumerate(zip(jobs, outs)):
        if k == 2:
            ref = _alone(img, sc2, n)
            ok = ~torch.isnan(o)
            assert int((~ok).sum()) == 1 and torch.equal(o[ok], ref[ok])
        else:
            assert torch.equal(o, _alone(img, sc, n))
    srv.close()
