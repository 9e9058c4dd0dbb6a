"""The debug build (compiled with -DFHP_DEBUG): device-side index checks
that report into the error word instead of trapping, and canary blocks after
every device buffer -- the race and bounds detection available where
compute-sanitizer is not.  Tiny lattices, where every edge path (word, warp,
tile and periodic wrap) is taken, run through every kernel in a subprocess
that loads the debug library (FHP_DEBUG=1); each result equals the oracle,
no check fails and no canary changes.  A self-test shows that a failing check
is recorded."""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_runs_every_kernel_clean(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2428_gb300 import build as cuda_build
    cuda_build.build(debug=True)
    env = dict(os.environ, FHP_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_probe.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert r.returncode == 0 and lines, r.stdout[-2000:] + r.stderr[-2000:]
    out = json.loads(lines[-1])
    assert out["ok"], out
    assert out["selftest"] == {"bounds_bit": True, "site": 99}
    assert out["cases"] >= 200


def test_release_build_has_no_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2428_gb300 import fhp
    lib = fhp.load()
    if os.environ.get("FHP_DEBUG") == "1":
        pytest.skip("this process loaded the debug build")
    assert lib.fhp_debug_build() == 0
    word = fhp.ctypes.c_uint32(0)
    assert lib.fhp_debug_selftest(fhp.ctypes.byref(word)) == fhp.FHP_EINVAL
