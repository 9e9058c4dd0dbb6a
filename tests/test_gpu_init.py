"""Generated initial states on the device (a lattice and a batch member)
against the oracle's counter-based fill, bit-exact, and a run from them."""
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


CASES = [
    # W, H, seed, density, obstacle
    (32, 2, 1, 0.5, "none"),
    (96, 6, 2**40 + 17, 0.3, "points"),       # ragged quad, high seed word
    (160, 10, 3, 0.123456, "walls"),
    (4128, 4, 4, 1.0, "cylinder"),             # every fluid node full
    (256, 256, 5, 0.0, "cylinder"),            # empty
    (640, 130, 6, 0.25 + 0.5 / 65536, "points"),   # rounding tie of the threshold
]


@pytest.mark.parametrize("W,H,seed,density,obstacle", CASES)
def test_lattice_init_matches_oracle(pkg, oracle_mod, W, H, seed, density, obstacle):
    job = workloads.Lattice("init", W, H, density, seed, 0.0, 0, obstacle=obstacle, point_frac=0.05)
    solid = job.solid()
    want = oracle_mod.init_random(W, H, seed, density, solid)
    with pkg.Lattice(W, H, seed=seed) as lat:
        lat.set_state(np.full((H, W), 0x55, np.uint8))   # stale particles must be replaced
        if solid is not None:
            lat.load_obstacles(solid)
        lat.init_random(density)
        got = lat.get_state()
    assert np.array_equal(got, want), int((got != want).sum())


def test_batch_init_and_run_match_oracle(pkg, oracle_mod):
    rng = np.random.Generator(np.random.PCG64(11))
    jobs = []
    for i in range(10):
        W = int(rng.choice(np.arange(64, 641, 32)))
        H = int(rng.choice(np.arange(64, 401, 2)))
        obstacle = ["none", "cylinder", "points", "walls"][i % 4]
        jobs.append(workloads.Lattice(f"b{i}", W, H, float(rng.uniform(0.1, 0.4)), 70_000 + i,
                                      5e-4 if i % 3 == 0 else 0.0, int(rng.integers(1, 30)),
                                      obstacle=obstacle, point_frac=0.02))
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        b.set_graph_steps(4)
        slots = []
        for j in jobs:
            k = b.add(j.W, j.H, j.seed, j.p)
            if j.solid() is not None:
                b.load_obstacles(k, j.solid())
            b.init_random(k, j.density)
            b.set_steps_left(k, j.steps)
            slots.append(k)
        for j, k in zip(jobs, slots):
            s0 = oracle_mod.init_random(j.W, j.H, j.seed, j.density, j.solid())
            assert np.array_equal(b.get_state(k), s0), j.name
        b.step(30)
        for j, k in zip(jobs, slots):
            s0 = oracle_mod.init_random(j.W, j.H, j.seed, j.density, j.solid())
            want, _ = oracle_mod.run(s0, j.seed, 0, j.steps, j.p)
            assert b.time(k) == j.steps
            assert np.array_equal(b.get_state(k), want), j.name


def test_init_rejects_bad_density(pkg):
    with pkg.Lattice(64, 4, seed=1) as lat:
        for bad in (-0.1, 1.5, float("nan")):
            with pytest.raises(pkg.FhpError):
                lat.init_random(bad)
