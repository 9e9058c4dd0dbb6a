"""Autotuner of the single-lattice step: it leaves the lattice's state and
step counter as they were, records a configuration per lattice description,
and lattices that then run the recorded configuration stay bit-exact with the
oracle."""
from __future__ import annotations

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


SHAPES = [
    # W, H, p, obstacle
    (2048, 512, 1e-3, "cylinder"),
    (256, 256, 0.0, "none"),
    (1024, 96, 0.0, "points"),
    (4096, 1024, 5e-4, "walls"),
]


@pytest.mark.parametrize("W,H,p,obstacle", SHAPES)
def test_autotune_keeps_state_and_stays_exact(pkg, oracle_mod, W, H, p, obstacle):
    job = workloads.Lattice("tune", W, H, 0.3, 4242, p, 0, obstacle=obstacle, point_frac=0.02)
    s0 = job.initial_state()
    with pkg.Lattice(W, H, seed=job.seed, forcing_p=p) as a:
        a.set_state(s0)
        a.set_time(7)
        kern, k = a.autotune(16)
        assert kern in (1, 2, 3, 4) and k in (1, 2, 4, 8)
        assert a.t == 7
        assert np.array_equal(a.get_state(), s0)
        assert a.temporal_block == k
        assert a.step_kernel == kern
    with pkg.Lattice(W, H, seed=job.seed, forcing_p=p) as b:    # same description: uses the recorded choice
        b.set_state(s0)
        b.set_time(7)
        assert b.temporal_block == k
        b.step(29)
        got = b.get_state()
    want, _ = oracle_mod.run(s0, job.seed, 7, 29, p)
    assert np.array_equal(got, want)


def test_explicit_settings_override_the_recorded_choice(pkg):
    with pkg.Lattice(2048, 512, seed=1) as a:
        a.set_state(workloads.bernoulli_lattice(2048, 512, 0.2, 1))
        a.autotune(8)
        a.set_step_kernel(1)
        assert a.step_kernel == 1 and a.temporal_block == 1
        a.set_step_kernel(0)
        a.set_temporal_block(2)
        assert a.temporal_block == 2


def test_autotune_rejects_bad_trial_counts(pkg):
    with pkg.Lattice(256, 64, seed=1) as a:
        for bad in (0, 4, 12, 8192):
            with pytest.raises(pkg.FhpError):
                a.autotune(bad)
