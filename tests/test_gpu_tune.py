"""The autotuner's choices outlive the process when ABF_TUNE_CACHE names a
file: a plan created later with the same key (GPU, order, limbs, size, Q,
scale kind) starts from the kept rows per CTA; a file that does not parse is
ignored.  Each step runs in its own process (the cache is read once)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_MAKE = (
    "import numpy as np, torch, synthetic\n"
    "from paper_0908_3861_gb300 import AdaptiveFilter\n"
    "rng = np.random.default_rng(5)\n"
    "img = rng.integers(0, 256, (96, 160)).astype(np.uint8)\n"
    "sc = synthetic.scales_a4(rng, (96, 160), 1.0, 6.0, 8.0).astype(np.float32)\n"
    "f = AdaptiveFilter(160, 96, 2, torch.uint8, scale_kind='a4', q_bits=4, max_scale=6.0, device='cuda:0')\n"
    "f.integrate(torch.from_numpy(img).cuda())\n"
    "st = torch.from_numpy(sc).cuda()\n")


def _run(code, cache):
    env = dict(os.environ, ABF_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    return out.stdout.strip().splitlines()[-1]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_tuning_is_kept_in_the_cache_file(tmp_path):
    cache = tmp_path / "tune.json"
    rows = int(_run(_MAKE + "rows, _ = f.autotune(st)\nprint(rows)\n", cache))
    assert rows in (4, 8, 16)
    kept = json.loads(cache.read_text())
    keys = [k for k in kept if k.startswith("plan:")]
    assert len(keys) == 1 and kept[keys[0]] == rows
    # another value under the same key: a new process must start from it
    other = 4 if rows != 4 else 16
    kept[keys[0]] = other
    cache.write_text(json.dumps(kept))
    assert int(_run(_MAKE + "print(f.launch_rows())\n", cache)) == other


def test_unreadable_cache_file_is_ignored(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("not a tuning cache")
    assert int(_run(_MAKE + "print(f.launch_rows())\n", cache)) == 8
