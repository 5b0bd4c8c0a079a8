"""Failure detection with host-side fault injection (abf_debug_inject_fault,
ABF_FAULT): a failed device allocation, a withheld job queue and an invalid
descriptor surface as error codes, nothing is left half-built, and the
library (and the GPU) stay usable: the next plan or job gives the same result
as a run without faults.  No GPU fault is caused: every injected failure
happens on the host before any kernel sees it."""
import os
import subprocess
import sys

import pytest

from tests.test_gpu_serve import _alone, _desc, _job, _pinned

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(autouse=True)
def _disarm():
    """Faults are process-wide: every test leaves all kinds disarmed."""
    yield
    from paper_0908_3861_gb300 import _abf as C
    for k in (C.ABF_FAULT_ALLOC, C.ABF_FAULT_QUEUE_STALL, C.ABF_FAULT_BAD_DESC):
        C.abf_debug_inject_fault(k, 0)


def test_plan_allocation_failure_then_recovery():
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter, AbfError, _abf as C
    img, sc, n = _job(500, 33, 47, 2)
    want = _alone(img, sc, n)
    C.abf_debug_inject_fault(C.ABF_FAULT_ALLOC, 1)
    with pytest.raises(AbfError) as e:
        AdaptiveFilter(47, 33, n, torch.float32, scale_kind="ellipse", q_bits=6, frac_bits=16, max_scale=20.0,
                       out="f32", value_bound=255.0, device="cuda:0")
    assert e.value.status == C.ABF_ERR_OOM
    assert torch.equal(_alone(img, sc, n), want)   # the fault was used up; the next plan works


def test_invalid_descriptor_then_recovery():
    import torch
    from paper_0908_3861_gb300 import AdaptiveFilter, AbfError, _abf as C
    img, sc, n = _job(501, 29, 40, 1)
    want = _alone(img, sc, n)
    C.abf_debug_inject_fault(C.ABF_FAULT_BAD_DESC, 2)
    for _ in range(2):
        with pytest.raises(AbfError) as e:
            AdaptiveFilter(40, 29, n, torch.float32, scale_kind="ellipse", q_bits=6, frac_bits=16, max_scale=20.0,
                           out="f32", value_bound=255.0, device="cuda:0")
        assert e.value.status == C.ABF_ERR_INVALID
    assert torch.equal(_alone(img, sc, n), want)


def test_server_job_allocation_failure_then_next_job():
    import torch
    from paper_0908_3861_gb300 import Server, AbfError, _abf as C
    img, sc, n = _job(502, 40, 52, 2)
    want = _alone(img, sc, n)
    srv = Server(256 << 20, max_inflight=2, device="cuda:0")
    try:
        outs = [torch.zeros(img.shape, dtype=torch.float32).pin_memory() for _ in range(3)]
        # the first job builds the server's plan for this descriptor, so the
        # armed fault hits the second job's own buffers
        t0 = srv.submit(_desc(img, n), _pinned(img), _pinned(sc), outs[0])
        assert srv.wait(t0, timeout_s=60)["status"] == 0
        C.abf_debug_inject_fault(C.ABF_FAULT_ALLOC, 1)
        t1 = srv.submit(_desc(img, n), _pinned(img), _pinned(sc), outs[1])
        with pytest.raises(AbfError) as e:   # abf_wait returns the job's own status
            srv.wait(t1, timeout_s=60)
        assert e.value.status == C.ABF_ERR_OOM
        assert srv.stats()["used"] == 0   # the failed job released what it had
        t2 = srv.submit(_desc(img, n), _pinned(img), _pinned(sc), outs[2])
        st = srv.wait(t2, timeout_s=60)
        assert st["status"] == 0 and st["device_status"] == 0
        assert torch.equal(outs[0], want) and torch.equal(outs[2], want)
    finally:
        srv.close()


def test_withheld_queue_times_out_then_drains():
    import torch
    from paper_0908_3861_gb300 import Server, AbfError, _abf as C
    img, sc, n = _job(503, 36, 44, 1)
    want = _alone(img, sc, n)
    srv = Server(256 << 20, max_inflight=2, device="cuda:0")
    try:
        C.abf_debug_inject_fault(C.ABF_FAULT_QUEUE_STALL, 1)
        outs = [torch.zeros(img.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        ts = [srv.submit(_desc(img, n), _pinned(img), _pinned(sc), o) for o in outs]
        with pytest.raises(AbfError) as e:
            srv.wait(ts[0], timeout_s=0.2)
        assert e.value.status == C.ABF_ERR_TIMEOUT
        assert srv.stats()["queued"] == 2
        C.abf_debug_inject_fault(C.ABF_FAULT_QUEUE_STALL, 0)
        for t, o in zip(ts, outs):
            assert srv.wait(t, timeout_s=60)["status"] == 0
            assert torch.equal(o, want)
    finally:
        srv.close()


def test_fault_environment_variable():
    """ABF_FAULT arms faults for a whole process: bad_desc:2 makes the first
    two plan creations fail, the third succeeds."""
    code = (
        "import torch\n"
        "from paper_0908_3861_gb300 import AdaptiveFilter, AbfError\n"
        "res = []\n"
        "for _ in range(3):\n"
        "    try:\n"
        "        AdaptiveFilter(20, 10, 1, torch.uint8, q_bits=4, max_scale=4.0, device='cuda:0').close()\n"
        "        res.append(0)\n"
        "    except AbfError as e:\n"
        "        res.append(e.status)\n"
        "print(res)\n")
    env = dict(os.environ, ABF_FAULT="bad_desc:2")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip().splitlines()[-1] == "[1, 1, 0]"
