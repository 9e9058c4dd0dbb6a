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


def shape_mask(W, H, shapes):
    """The nodes the shapes cover, written out on the host (index coordinates)."""
    yy, xx = np.mgrid[0:H, 0:W]
    m = np.zeros((H, W), dtype=bool)
    for kind, a, b, c in shapes:
        if kind == 2:
            m |= (yy >= a) & (yy < b)
        else:
            m |= (xx - a) ** 2 + (yy - b) ** 2 <= c * c
    return m


SHAPE_CASES = [
    (512, 256, workloads.cylinder_shapes(512, 256)),
    (160, 66, [(1, -5, 10, 12), (1, 170, 60, 9), (2, -3, 2, 0), (2, 60, 99, 0)]),   # shapes past the edges
    (4128, 32, [(1, 4127, 16, 40), (1, 0, 0, 0)]),                                  # a one-node disc
    (96, 8, []),                                                                    # no shape: no solid node
]


@pytest.mark.parametrize("W,H,shapes", SHAPE_CASES)
def test_obstacle_shapes_equal_the_mask(pkg, oracle_mod, W, H, shapes):
    mask = shape_mask(W, H, shapes)
    if shapes == workloads.cylinder_shapes(W, H):
        assert np.array_equal(mask, workloads.cylinder_mask(W, H))
    s0 = workloads.bernoulli_lattice(W, H, 0.3, 5)
    with pkg.Lattice(W, H, seed=5, forcing_p=0.01) as lat:
        lat.set_state(s0)
        lat.load_obstacle_shapes(shapes)
        got = lat.get_state()
        lat.step(7)
        after = lat.get_state()
    want = s0.copy()
    want[mask] = 0x80
    assert np.array_equal(got, want)
    ref, _ = oracle_mod.run(want, 5, 0, 7, 0.01)
    assert np.array_equal(after, ref)
    # the batch version, with the state drawn after the obstacles
    with pkg.Batch(pkg.Batch.lattice_bytes(W, H) + (8 << 20)) as b:
        k = b.add(W, H, 9, 0.0)
        b.load_obstacle_shapes(k, shapes)
        b.init_random(k, 0.4)
        b.step(5)
        s_init = oracle_mod.init_random(W, H, 9, 0.4, mask.astype(np.uint8))
        ref_b, _ = oracle_mod.run(s_init, 9, 0, 5, 0.0)
        assert np.array_equal(b.get_state(k), ref_b)


def test_obstacle_shapes_reject_bad_lists(pkg):
    with pkg.Lattice(64, 8) as lat:
        with pytest.raises(pkg.FhpError):
            lat.load_obstacle_shapes([(3, 0, 0, 0)])
        with pytest.raises(pkg.FhpError):
            lat.load_obstacle_shapes([(1, 0, 0, -1)])
        with pytest.raises(pkg.FhpError):
            lat.load_obstacle_shapes([(2, 0, 1, 0)] * 9)
