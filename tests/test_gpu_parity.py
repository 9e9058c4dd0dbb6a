"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Lattice states and integer coarse-grained counts must be bit-exact; derived
float fields within 1e-6 relative (they are computed in double on both sides
and rounded to float, so they usually agree exactly)."""
from __future__ import annotations

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

FLOAT_RTOL = 1e-6


@pytest.fixture(scope="module")
def fhp_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2428_gb300 import build as cuda_build
    cuda_build.build()
    import paper_1208_2428_gb300 as pkg
    pkg.load()
    return pkg


def gpu_run(pkg, s0, seed, t0, n, p, chunks=None, kernel=0, k_block=1, bk=0):
    H, W = s0.shape
    with pkg.Lattice(W, H, seed=seed, forcing_p=p, step_kernel=kernel) as lat:
        lat.set_temporal_block(k_block)
        lat.set_temporal_block_kernel(bk)
        lat.set_state(s0)
        if bk and k_block > 1:
            assert lat.temporal_block_kernel == bk, "the requested temporal-block kernel must run"
        lat.set_time(t0)
        for c in (chunks or [n]):
            lat.step(c)
        assert lat.t == t0 + n
        return lat.get_state()


def assert_same(got, want, what=""):
    if not np.array_equal(got, want):
        diff = np.argwhere(got != want)
        y, x = diff[0]
        raise AssertionError(f"{what}: {len(diff)} nodes differ; first at (x={x}, y={y}): "
                             f"gpu {got[y, x]:08b} oracle {want[y, x]:08b}")


def test_roundtrip_bytes(fhp_mod):
    rng = np.random.Generator(np.random.PCG64(5))
    for W, H in [(32, 2), (96, 6), (160, 4), (4128, 4), (256, 256)]:
        s = rng.integers(0, 256, size=(H, W), dtype=np.uint8)  # includes particles on solid nodes
        with fhp_mod.Lattice(W, H, seed=1) as lat:
            lat.set_state(s)
            assert_same(lat.get_state(), s, f"roundtrip {W}x{H}")
            lat.step(0)
            assert_same(lat.get_state(), s, "step(0)")


SHAPES = [
    (32, 2), (32, 4), (64, 2), (96, 6), (128, 8), (160, 4), (192, 10), (224, 6), (256, 12),
    (384, 4), (480, 6), (992, 8),          # narrow rows: several rows of one parity per warp
    (4096, 4), (4128, 4), (4160, 6), (4192, 2), (8192 + 96, 4), (12288, 2),  # wide rows, ragged tails
]


# direct register loads; bulk-copy ring; multi-step ring (one launch); shared-memory resident lattice
# (falls back to the automatic choice where the strips do not fit)
KERNELS = [1, 2, 3, 4]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("W,H", SHAPES)
@pytest.mark.parametrize("variant", ["periodic", "walls_forcing", "points_forcing"])
def test_parity_shapes(fhp_mod, oracle_mod, W, H, variant, kernel):
    seed = 1000 + W + 7 * H
    rng = np.random.Generator(np.random.PCG64(seed))
    if variant == "periodic":
        solid, p = None, 0.0
    elif variant == "walls_forcing":
        solid, p = workloads.channel_walls(W, H), 0.05
    else:
        solid, p = workloads.random_points(W, H, 0.05, rng), 0.2
    s0 = workloads.bernoulli_lattice(W, H, 0.35, seed, solid)
    steps = 9
    want, _ = oracle_mod.run(s0, seed, 3, steps, p)
    got = gpu_run(fhp_mod, s0, seed, 3, steps, p, kernel=kernel)
    assert_same(got, want, f"{W}x{H} {variant} kernel {kernel}")


@pytest.mark.parametrize("kernel", KERNELS)
def test_parity_empty_and_full(fhp_mod, oracle_mod, kernel):
    for W, H in [(64, 4), (4160, 2)]:
        for fill in (0x00, 0x7F, 0x3F, 0x40):
            s0 = np.full((H, W), fill, dtype=np.uint8)
            want, _ = oracle_mod.run(s0, 3, 0, 5, 0.5)
            got = gpu_run(fhp_mod, s0, 3, 0, 5, 0.5, kernel=kernel)
            assert_same(got, want, f"fill {fill:#x}")
        s0 = np.full((H, W), 0xFF, dtype=np.uint8)   # all solid, full of particles
        want, _ = oracle_mod.run(s0, 3, 0, 4, 0.5)
        assert_same(gpu_run(fhp_mod, s0, 3, 0, 4, 0.5, kernel=kernel), want, "all solid")


@pytest.mark.parametrize("kernel", [2, 3, 4])
@pytest.mark.parametrize("W,H", [(256, 2048), (4096, 1024), (2048, 512), (96, 4096), (4128, 6000)])
def test_parity_ring_many_tiles(fhp_mod, oracle_mod, W, H, kernel):
    """Shapes where the ring kernels walk many tiles per CTA (pipeline wrap-around,
    dependency waits across step boundaries for the multi-step kernel)."""
    seed = W + H
    s0 = workloads.bernoulli_lattice(W, H, 0.3, seed, workloads.cylinder_mask(W, H))
    want, _ = oracle_mod.run(s0, seed, 0, 7, 0.01)
    got = gpu_run(fhp_mod, s0, seed, 0, 7, 0.01, kernel=kernel)
    assert_same(got, want, f"kernel {kernel} {W}x{H}")


# (temporal block k, its kernel): row wavefronts (1) for k = 2, 3, 4; 2-D tiles (2) for k = 2, 4, 8
BLOCKS = [(2, 1), (3, 1), (4, 1), (2, 2), (4, 2), (8, 2)]


@pytest.mark.parametrize("k,bk", BLOCKS)
@pytest.mark.parametrize("W,H", [(512, 18), (640, 46), (4224, 100), (2048, 512), (4096, 1030)])
@pytest.mark.parametrize("variant", ["periodic", "walls_forcing", "points_forcing"])
def test_parity_temporal_block(fhp_mod, oracle_mod, W, H, k, bk, variant):
    """k steps per pass on chip (row wavefronts through per-level row rings,
    or 2-D tiles with a k-row / 128-node halo; periodic wrap in x and y):
    bit-exact for passes plus a remainder of single steps."""
    seed = 77 + W + H + k
    rng = np.random.Generator(np.random.PCG64(seed))
    if variant == "periodic":
        solid, p = None, 0.0
    elif variant == "walls_forcing":
        solid, p = workloads.channel_walls(W, H), 0.05
    else:
        solid, p = workloads.random_points(W, H, 0.05, rng), 0.2
    s0 = workloads.bernoulli_lattice(W, H, 0.35, seed, solid)
    steps = 2 * k + 3
    want, _ = oracle_mod.run(s0, seed, 5, steps, p)
    got = gpu_run(fhp_mod, s0, seed, 5, steps, p, k_block=k, bk=bk)
    assert_same(got, want, f"{W}x{H} {variant} k={k} kernel {bk}")


# Row-wavefront shapes: 1 to 4 columns of 32 quads (one to four warps per
# level row), ragged last quads, lattices lower than a band's halo (rows wrap
# more than once), and the widest rows each k supports.
WAVE_SHAPES = [(32, 2), (32, 6), (96, 4), (128, 10), (1024, 16), (4096, 12), (4128, 8), (8192 + 96, 6),
               (12288, 4), (16384, 8), (256, 2048)]


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("W,H", WAVE_SHAPES)
@pytest.mark.parametrize("variant", ["periodic", "walls_forcing", "points_forcing"])
def test_parity_wavefront_shapes(fhp_mod, oracle_mod, W, H, k, variant):
    seed = 31 + 3 * W + H + k
    rng = np.random.Generator(np.random.PCG64(seed))
    if variant == "periodic":
        solid, p = None, 0.0
    elif variant == "walls_forcing":
        solid, p = workloads.channel_walls(W, H), 0.05
    else:
        solid, p = workloads.random_points(W, H, 0.05, rng), 0.3
    s0 = workloads.bernoulli_lattice(W, H, 0.35, seed, solid)
    steps = 2 * k + 1
    want, _ = oracle_mod.run(s0, seed, 7, steps, p)
    with fhp_mod.Lattice(W, H, seed=seed, forcing_p=p) as lat:
        lat.set_temporal_block(k)
        lat.set_temporal_block_kernel(1)
        lat.set_state(s0)
        assert lat.temporal_block == k and lat.temporal_block_kernel == 1
        lat.set_time(7)
        lat.step(steps)
        assert_same(lat.get_state(), want, f"{W}x{H} {variant} wavefront k={k}")


@pytest.mark.parametrize("k", [4, 8])
def test_temporal_block_forcing_near_tile_edges(fhp_mod, oracle_mod, k):
    """Forcing decides the 32 nodes of a word together, so an inexact node at
    the edge of a staged block spoils its whole word: the horizontal halo must
    be k words.  Dense forcing on the smallest supported height and several
    seeds exercises exactly that."""
    W, H = 512, 2 * k + 2
    for seed in range(600, 608):
        rng = np.random.Generator(np.random.PCG64(seed))
        s0 = workloads.bernoulli_lattice(W, H, 0.35, seed, workloads.random_points(W, H, 0.05, rng))
        for p in (0.2, 0.5):
            want, _ = oracle_mod.run(s0, seed, 5, k, p)
            got = gpu_run(fhp_mod, s0, seed, 5, k, p, k_block=k, bk=2)
            assert_same(got, want, f"seed {seed} p {p} k {k}")


def test_temporal_block_full_size_all_k(fhp_mod, oracle_mod):
    """16384 x 4096 cylinder: 24 steps give the same state for k = 1 and every
    blocked kernel and k, and equal the oracle."""
    job = workloads.cylinder_16384x4096()
    s0 = job.initial_state()
    want, _ = oracle_mod.run(s0, job.seed, 0, 24, job.p)
    assert_same(gpu_run(fhp_mod, s0, job.seed, 0, 24, job.p), want, "k=1")
    for k, bk in BLOCKS:
        assert_same(gpu_run(fhp_mod, s0, job.seed, 0, 24, job.p, k_block=k, bk=bk), want, f"k={k} kernel {bk}")


def test_cylinder_1000_steps_same_for_every_k(fhp_mod):
    """16384 x 4096 cylinder, the benchmark's 1,000 steps: the final state is
    the same for k = 1, 2, 4, 8 and for the single-step ring (the oracle pins
    the first 24 steps above; here the kernels must agree over the full run)."""
    job = workloads.cylinder_16384x4096()
    s0 = job.initial_state()
    ref = gpu_run(fhp_mod, s0, job.seed, 0, job.steps, job.p)
    for k, bk in BLOCKS:
        assert_same(gpu_run(fhp_mod, s0, job.seed, 0, job.steps, job.p, k_block=k, bk=bk), ref,
                    f"1000 steps, k={k} kernel {bk}")
    assert_same(gpu_run(fhp_mod, s0, job.seed, 0, job.steps, job.p, kernel=2), ref, "1000 steps, ring")


def test_parity_large_step_counter(fhp_mod, oracle_mod):
    """Counters above 2^32 use the high half of t in the random streams."""
    W, H = 256, 16
    s0 = workloads.bernoulli_lattice(W, H, 0.3, 9, workloads.channel_walls(W, H))
    t0 = (7 << 32) - 3
    want, _ = oracle_mod.run(s0, 0xFEDCBA9876543210, t0, 6, 0.1)
    got = gpu_run(fhp_mod, s0, 0xFEDCBA9876543210, t0, 6, 0.1)
    assert_same(got, want, "t across 2^32")


def test_periodic_256_full(fhp_mod, oracle_mod):
    """256 x 256 periodic, density 0.3, seed 1, 100 steps: final state and
    per-direction totals bit-exact."""
    job = workloads.periodic_256()
    s0 = job.initial_state()
    want, _ = oracle_mod.run(s0, job.seed, 0, job.steps, job.p)
    got = gpu_run(fhp_mod, s0, job.seed, 0, job.steps, job.p, chunks=[1, 36, 63])
    assert_same(got, want, "periodic_256")
    for k in range(7):
        assert int(np.count_nonzero(got >> k & 1)) == int(np.count_nonzero(want >> k & 1))


def test_channel_coarse_grain(fhp_mod, oracle_mod):
    """4096 x 1024 channel (walls, p = 1e-3) over its full 10,000 steps: the
    32 x 32 coarse-grained fields at every output time (t = 1,000, 2,000,
    ..., 10,000) and the state at the first and last of them equal the
    oracle's (counts bit-exact, derived floats within 1e-6 relative)."""
    job = workloads.channel_4096x1024()
    s0 = job.initial_state()
    every, outputs = 1000, 10
    assert job.steps == every * outputs
    want = s0
    with fhp_mod.Lattice(job.W, job.H, seed=job.seed, forcing_p=job.p) as lat:
        lat.set_state(s0)
        for i in range(outputs):
            want, ev = oracle_mod.run(want, job.seed, i * every, every, job.p)
            assert ev > 0
            lat.step(every)
            counts, rho, ux, uy = lat.coarse_grain(32)
            c_ref, rho_ref, ux_ref, uy_ref = oracle_mod.coarse_grain(want, 32)
            assert np.array_equal(counts, c_ref), f"counts at t = {(i + 1) * every}"
            for g, r in ((rho, rho_ref), (ux, ux_ref), (uy, uy_ref)):
                np.testing.assert_allclose(g, r.astype(np.float32), rtol=FLOAT_RTOL, atol=1e-30)
            if i in (0, outputs - 1):
                assert_same(lat.get_state(), want, f"channel at t = {(i + 1) * every}")
                d_counts, d_rho, d_ux, d_uy = lat.coarse_grain_tensor(32)
                assert np.array_equal(d_counts.cpu().numpy(), c_ref)
                np.testing.assert_array_equal(d_rho.cpu().numpy(), rho)
        assert lat.t == job.steps
    # physics sanity (qualitative): forcing drives a mean flow toward +x
    assert float(ux[1:-1].mean()) > 0


def test_cylinder_full_size(fhp_mod, oracle_mod):
    """16384 x 4096 cylinder workload at full size in the benchmark's launch
    configuration (automatic kernel choice, as bench.py runs it): whole state
    bit-exact after 12 steps; the direct kernel agrees too."""
    job = workloads.cylinder_16384x4096()
    s0 = job.initial_state()
    n = 12
    want, ev = oracle_mod.run(s0, job.seed, 0, n, job.p)
    with fhp_mod.Lattice(job.W, job.H, seed=job.seed, forcing_p=job.p) as lat:
        lat.set_state(s0)
        assert lat.step_kernel == 3      # the multi-step ring kernel is what the benchmark times
        lat.step(n)
        assert_same(lat.get_state(), want, "cylinder 16384x4096")
    for k in (1, 2):
        assert_same(gpu_run(fhp_mod, s0, job.seed, 0, n, job.p, kernel=k), want, f"cylinder, kernel {k}")


def test_paper_size_lattice(fhp_mod, oracle_mod):
    """The paper's GPU lattice size (29,970 x 27,990; W rounded up to 29,984,
    a ragged row of 937 words): 2 steps bit-exact."""
    job = workloads.cylinder_paper_size()
    s0 = job.initial_state()
    want, _ = oracle_mod.run(s0, job.seed, 0, 2, job.p)
    got = gpu_run(fhp_mod, s0, job.seed, 0, 2, job.p)
    assert_same(got, want, "29984 x 27990")


def test_resume_from_checkpoint(fhp_mod):
    W, H = 4160, 6
    s0 = workloads.bernoulli_lattice(W, H, 0.3, 21, workloads.channel_walls(W, H))
    full = gpu_run(fhp_mod, s0, 21, 0, 30, 0.05)
    with fhp_mod.Lattice(W, H, seed=21, forcing_p=0.05) as a:
        a.set_state(s0)
        a.step(13)
        ckpt, t = a.get_state(), a.t
    with fhp_mod.Lattice(W, H, seed=21, forcing_p=0.05) as b:
        b.set_state(ckpt)
        b.set_time(t)
        b.step(17)
        assert_same(b.get_state(), full, "resume")


def test_load_obstacles_clears_particles(fhp_mod, oracle_mod):
    W, H = 256, 32
    s0 = workloads.bernoulli_lattice(W, H, 0.4, 4)
    mask = workloads.cylinder_mask(W, H)
    with fhp_mod.Lattice(W, H, seed=4, forcing_p=0.01) as lat:
        lat.set_state(s0)
        lat.load_obstacles(mask)
        after = lat.get_state()
        expect = np.where(mask, 0x80, s0).astype(np.uint8)
        assert_same(after, expect, "load_obstacles")
        lat.step(7)
        got = lat.get_state()
    want, _ = oracle_mod.run(expect, 4, 0, 7, 0.01)
    assert_same(got, want, "after obstacles")


def test_device_state_io(fhp_mod, oracle_mod):
    import torch
    W, H = 4128, 4
    s0 = workloads.bernoulli_lattice(W, H, 0.3, 8, workloads.channel_walls(W, H))
    with fhp_mod.Lattice(W, H, seed=8, forcing_p=0.02) as lat:
        lat.set_state_tensor(torch.from_numpy(s0).cuda())
        lat.step(5)
        got = lat.get_state_tensor().cpu().numpy()
    want, _ = oracle_mod.run(s0, 8, 0, 5, 0.02)
    assert_same(got, want, "device io")


def test_errors(fhp_mod):
    with pytest.raises(fhp_mod.FhpError):
        fhp_mod.Lattice(48, 4)
    with pytest.raises(fhp_mod.FhpError):
        fhp_mod.Lattice(64, 5)
    with fhp_mod.Lattice(64, 64) as lat:
        with pytest.raises(fhp_mod.FhpError):
            lat.coarse_grain(48)
        with pytest.raises(fhp_mod.FhpError):
            lat.step(-1)
        with pytest.raises(fhp_mod.FhpError):
            lat.set_forcing(2.0)
        with pytest.raises(fhp_mod.FhpError):
            lat.set_time(1 << 48)


def test_device_philox_matches_oracle(fhp_mod, oracle_mod):
    import torch
    rng = np.random.Generator(np.random.PCG64(77))
    n = 200_000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    out = fhp_mod.philox4x32_10_device(torch.from_numpy(ctr.view(np.int32)).cuda(),
                                       torch.from_numpy(key.view(np.int32)).cuda())
    got = out.cpu().numpy().view(np.uint32)
    for i in list(range(0, n, 997)) + [n - 1]:
        assert np.array_equal(got[i], oracle_mod.philox4x32_10(ctr[i], key[i])), i


@pytest.mark.parametrize("kernel,k", [(1, 1), (2, 1), (3, 1), (0, 2), (0, 4), (4, 1)])
def test_fhp1_rules_parity(fhp_mod, oracle_mod, kernel, k):
    """FHP-I (no rest-particle collisions) on every kernel, with walls,
    points and forcing, against the oracle's FHP-I run."""
    W, H, seed, p = 1024, 130, 4321, 0.01
    job = workloads.Lattice("fhp1", W, H, 0.3, seed, p, 0, obstacle="points", point_frac=0.02)
    s0 = job.initial_state()
    want, _ = oracle_mod.run(s0, seed, 2, 17, p, rules=1)
    with fhp_mod.Lattice(W, H, seed=seed, forcing_p=p, step_kernel=kernel) as lat:
        lat.set_rules(1)
        assert lat.rules == 1
        lat.set_temporal_block(k)
        lat.set_state(s0)
        lat.set_time(2)
        lat.step(17)
        got = lat.get_state()
    assert_same(got, want, f"FHP-I kernel {kernel} k {k}")
    # rest particles are spectators under FHP-I
    assert int(np.count_nonzero(got & 0x40)) == int(np.count_nonzero(s0 & 0x40))
    # and FHP-II gives a different result on the same input
    other, _ = oracle_mod.run(s0, seed, 2, 17, p, rules=2)
    assert not np.array_equal(other, want)


def test_fhp1_batch_member(fhp_mod, oracle_mod):
    W, H = 512, 64
    jobs = [workloads.Lattice(f"r{r}", W, H, 0.3, 70 + r, 0.0, 0) for r in (1, 2)]
    with fhp_mod.Batch(2 * fhp_mod.Batch.lattice_bytes(W, H) + (16 << 20)) as b:
        slots = []
        for r, j in zip((1, 2), jobs):
            k = b.add(W, H, j.seed, 0.0)
            b.set_rules(k, r)
            b.set_state(k, j.initial_state())
            slots.append(k)
        b.step(9)
        for r, j, k in zip((1, 2), jobs, slots):
            want, _ = oracle_mod.run(j.initial_state(), j.seed, 0, 9, 0.0, rules=r)
            assert np.array_equal(b.get_state(k), want), r
    with fhp_mod.Lattice(W, H) as lat:
        with pytest.raises(fhp_mod.FhpError):
            lat.set_rules(4)


@pytest.mark.parametrize("W,H,p,obstacle,kernel,k", [
    (1024, 130, 0.01, "points", 0, 1), (4096, 256, 0.0, "cylinder", 3, 1), (96, 8, 0.05, "walls", 4, 2),
    (160, 66, 0.0, "none", 2, 4), (4128, 4, 0.2, "points", 0, 1), (1024, 130, 0.01, "points", 1, 1),
    (4096, 256, 0.01, "cylinder", 2, 1), (4128, 64, 0.2, "points", 2, 1), (4128, 64, 0.2, "points", 3, 1),
    (2080, 96, 0.05, "walls", 3, 8)])
def test_fhp3_rules_parity(fhp_mod, oracle_mod, W, H, p, obstacle, kernel, k):
    """FHP-III (collision-saturated) runs on the direct, ring and multi-step
    kernels (the resident kernel and temporal blocks fall back to those);
    bit-exact with the oracle's FHP-III run on walls, points, a cylinder,
    forcing and ragged rows."""
    seed = 999 + W + H
    job = workloads.Lattice("fhp3", W, H, 0.35, seed, p, 0, obstacle=obstacle, point_frac=0.02)
    s0 = job.initial_state()
    want, _ = oracle_mod.run(s0, seed, 3, 21, p, rules=3)
    with fhp_mod.Lattice(W, H, seed=seed, forcing_p=p, step_kernel=kernel) as lat:
        lat.set_rules(3)
        lat.set_temporal_block(k)
        lat.set_state(s0)
        assert lat.rules == 3 and lat.step_kernel in (1, 2, 3) and lat.temporal_block == 1
        if kernel in (1, 2, 3):
            assert lat.step_kernel == kernel
        lat.set_time(3)
        lat.step(21)
        got = lat.get_state()
        assert_same(got, want, f"FHP-III {W}x{H} kernel {lat.step_kernel}")
        # back to FHP-II for the next steps
        lat.set_rules(2)
        lat.step(5)
        more, _ = oracle_mod.run(want, seed, 24, 5, p, rules=2)
        assert_same(lat.get_state(), more, "FHP-II after FHP-III")
    other, _ = oracle_mod.run(s0, seed, 3, 21, p, rules=2)
    assert not np.array_equal(other, want)


def test_fhp3_autotune_and_batch(fhp_mod, oracle_mod):
    """An FHP-III lattice tunes among the kernels that carry it without
    touching the choice recorded for FHP-II lattices of its shape; batches
    refuse FHP-III."""
    W, H = 2048, 512
    s0 = workloads.bernoulli_lattice(W, H, 0.3, 12)
    with fhp_mod.Lattice(W, H, seed=12) as a:
        a.set_state(s0)
        kern2, k2 = a.autotune(16)
        a.set_rules(3)
        kern3, k3 = a.autotune(16)
        assert kern3 in (1, 2, 3) and k3 == 1
        assert a.step_kernel == kern3
        a.step(7)
        want, _ = oracle_mod.run(s0, 12, 0, 7, 0.0, rules=3)
        assert_same(a.get_state(), want, "FHP-III after autotune")
    with fhp_mod.Lattice(W, H, seed=12) as b:
        assert (b.step_kernel, b.temporal_block) == (kern2, k2)
    with fhp_mod.Batch(fhp_mod.Batch.lattice_bytes(W, H) + (16 << 20)) as bt:
        slot = bt.add(W, H, 1, 0.0)
        with pytest.raises(fhp_mod.FhpError):
            bt.set_rules(slot, 3)


@pytest.mark.parametrize("W,H,steps", [(4096, 1024, 1), (4096, 1024, 2), (4096, 1024, 37), (2048, 512, 40),
                                       (256, 2048, 9), (96, 4096, 8), (512, 150, 11), (640, 2, 5), (32, 2, 6)])
def test_resident_kernel(fhp_mod, oracle_mod, W, H, steps):
    """The shared-memory resident kernel (one strip per SM, edge rows exchanged
    between steps): odd and even step counts (the result buffer alternates),
    strips of one row, more SMs than rows, walls, a cylinder, forcing."""
    seed = 77 + W + H
    s0 = workloads.bernoulli_lattice(W, H, 0.3, seed, workloads.cylinder_mask(W, H) if H >= 16 else None)
    want, _ = oracle_mod.run(s0, seed, 5, steps, 0.02)
    with fhp_mod.Lattice(W, H, seed=seed, forcing_p=0.02, step_kernel=4) as lat:
        lat.set_state(s0)
        lat.set_time(5)
        assert lat.step_kernel == 4
        lat.step(steps)
        assert lat.t == 5 + steps
        assert_same(lat.get_state(), want, f"resident {W}x{H} {steps} steps")
        lat.step(3)                      # a second call continues from the result buffer
        more, _ = oracle_mod.run(want, seed, 5 + steps, 3, 0.02)
        assert_same(lat.get_state(), more, "resident, second call")


@pytest.mark.parametrize("W,H,steps,obstacles,p", [
    (4096, 1024, 1, True, 0.02), (4096, 1024, 2, True, 0.02), (4096, 1024, 3, True, 0.02),
    (4096, 1024, 37, True, 0.02), (2048, 1024, 40, False, 0.0), (256, 2048, 9, True, 0.0),
    (96, 4096, 8, False, 0.02), (512, 608, 7, True, 0.02), (160, 610, 5, True, 0.01), (4128, 640, 12, False, 0.05)])
def test_resident_ghost_rows(fhp_mod, oracle_mod, W, H, steps, obstacles, p):
    """The resident kernel with two ghost rows per strip side (exchanges every
    second step): step counts that end inside a round, strips of exactly four
    rows, ragged rows, with and without obstacles and forcing."""
    seed = 91 + W + H
    s0 = workloads.bernoulli_lattice(W, H, 0.3, seed, workloads.cylinder_mask(W, H) if obstacles else None)
    want, _ = oracle_mod.run(s0, seed, 5, steps, p)
    with fhp_mod.Lattice(W, H, seed=seed, forcing_p=p, step_kernel=4) as lat:
        lat.set_temporal_block(2)
        lat.set_state(s0)
        lat.set_time(5)
        assert lat.step_kernel == 4 and lat.temporal_block == 2
        lat.step(steps)
        assert lat.t == 5 + steps
        assert_same(lat.get_state(), want, f"resident ghost {W}x{H} {steps} steps")
        lat.step(3)
        more, _ = oracle_mod.run(want, seed, 5 + steps, 3, p)
        assert_same(lat.get_state(), more, "resident ghost, second call")


def test_resident_ghost_falls_back_to_one_row(fhp_mod, oracle_mod):
    """Strips shorter than four rows take the one-row exchange."""
    W, H, seed = 512, 150, 4
    s0 = workloads.bernoulli_lattice(W, H, 0.3, seed)
    want, _ = oracle_mod.run(s0, seed, 0, 6, 0.0)
    with fhp_mod.Lattice(W, H, seed=seed, step_kernel=4) as lat:
        lat.set_temporal_block(2)
        assert lat.step_kernel == 4 and lat.temporal_block == 1
        lat.set_state(s0)
        lat.step(6)
        assert_same(lat.get_state(), want, "resident fallback")


def test_fhp1_resident_ghost_rows(fhp_mod, oracle_mod):
    """FHP-I through the two-ghost-row resident kernel (strips of 6-7 rows)."""
    W, H, seed, p = 4096, 1024, 515, 0.01
    s0 = workloads.bernoulli_lattice(W, H, 0.3, seed, workloads.channel_walls(W, H))
    want, _ = oracle_mod.run(s0, seed, 1, 15, p, rules=1)
    with fhp_mod.Lattice(W, H, seed=seed, forcing_p=p, step_kernel=4) as lat:
        lat.set_rules(1)
        lat.set_temporal_block(2)
        assert lat.step_kernel == 4 and lat.temporal_block == 2
        lat.set_state(s0)
        lat.set_time(1)
        lat.step(15)
        assert_same(lat.get_state(), want, "FHP-I resident ghost")


def test_fhp3_row_strips(fhp_mod, oracle_mod):
    """FHP-III on row strips of one lattice (row offsets key the random words;
    ghost rows exchanged through device buffers) equals the whole lattice."""
    from paper_1208_2428_gb300.strips import DeviceStrip, LocalExchange, StripDomain, StripPlan
    W, H, seed, p, steps = 512, 96, 4242, 2e-3, 11
    s0 = workloads.Lattice("s3", W, H, 0.3, seed, p, 0, obstacle="cylinder").initial_state()
    plan = StripPlan(W, H, 3, 4)
    strips = [DeviceStrip(plan, r, seed, p) for r in range(3)]
    try:
        for st in strips:
            st.set_from_global(s0)
            st.lattice.set_rules(3)
        StripDomain(plan, strips, LocalExchange()).step(steps)
        got = np.concatenate([st.owned_state() for st in strips])
    finally:
        for st in strips:
            st.close()
    want, _ = oracle_mod.run(s0, seed, 0, steps, p, rules=3)
    assert_same(got, want, "FHP-III strips")
