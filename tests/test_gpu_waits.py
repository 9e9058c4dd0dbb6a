"""Failure detection without a GPU fault: the bounded device-side waits of
the ring and multi-step kernels give up on conditions that never hold, report
it, and leave the device usable."""
from __future__ import annotations

import time

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2428_gb300 import build as cuda_build
    cuda_build.build()
    import paper_1208_2428_gb300 as p
    p.load()
    return p


def test_waits_give_up_and_the_device_stays_usable(pkg, oracle_mod):
    from paper_1208_2428_gb300.fhp import selftest_wait_limits
    t0 = time.perf_counter()
    status = selftest_wait_limits()
    elapsed = time.perf_counter() - t0
    assert status == 3                      # both the barrier wait and the counter wait gave up
    assert 3.5 < elapsed < 30.0             # after their 2 s limits, not at once and not never
    s0 = workloads.bernoulli_lattice(256, 64, 0.3, 3)
    with pkg.Lattice(256, 64, seed=3, step_kernel=3) as lat:
        lat.set_state(s0)
        lat.step(5)
        lat.synchronize()                   # no error left behind
        got = lat.get_state()
    want, _ = oracle_mod.run(s0, 3, 0, 5, 0.0)
    assert np.array_equal(got, want)
