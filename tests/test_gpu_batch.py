"""Batches of independent lattices (shared launches, continuous membership):
every member must equal the CPU oracle run of that lattice alone, bit-exact."""
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


def small_ensemble(n, seed, sides=range(128, 641, 64), force_every=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for i in range(n):
        W, H = int(rng.choice(list(sides))), int(rng.choice(list(sides)))
        p = 0.05 if i % force_every == 0 else 0.0
        jobs.append(workloads.Lattice(f"m{i}", W, H, float(rng.uniform(0.1, 0.5)), 9000 + i, p, 0,
                                      obstacle="points", point_frac=0.01))
    return jobs


def oracle_alone(oracle_mod, job, s0, t0, n):
    out, _ = oracle_mod.run(s0, job.seed, t0, n, job.p)
    return out


# 1: one launch per step (CUDA graphs); 2: all steps of a call in one cooperative launch
KERNELS = [1, 2]


@pytest.mark.parametrize("kernel", KERNELS)
def test_batch_matches_oracle(pkg, oracle_mod, kernel):
    jobs = small_ensemble(24, 1)
    states = [j.initial_state() for j in jobs]
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        b.set_step_kernel(kernel)
        assert b.step_kernel == kernel
        b.set_graph_steps(8)
        slots = []
        for j, s0 in zip(jobs, states):
            k = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(k, s0)
            b.set_time(k, 3)
            slots.append(k)
        b.step(37)                       # 4 graph replays of 8 steps + 5 direct launches
        b.synchronize()
        for j, s0, k in zip(jobs, states, slots):
            assert b.time(k) == 40
            want = oracle_alone(oracle_mod, j, s0, 3, 37)
            got = b.get_state(k)
            assert np.array_equal(got, want), (j.name, j.W, j.H, int((got != want).sum()))


@pytest.mark.parametrize("kernel", KERNELS)
def test_batch_continuous_membership_and_budgets(pkg, oracle_mod, kernel):
    """Members join, leave and carry different step budgets; each one's
    result equals its run alone."""
    jobs = small_ensemble(12, 2)
    states = [j.initial_state() for j in jobs]
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        b.set_step_kernel(kernel)
        b.set_graph_steps(4)
        slot = {}
        steps_done = {}
        # first wave
        for i in range(6):
            slot[i] = b.add(jobs[i].W, jobs[i].H, jobs[i].seed, jobs[i].p)
            b.set_state(slot[i], states[i])
            b.set_steps_left(slot[i], [7, 11, 3, 20, 20, 9][i])
        b.step(10)
        for i in range(6):
            steps_done[i] = min(10, [7, 11, 3, 20, 20, 9][i])
        # members 2 and 5 finished and leave; check them now
        for i in (2, 5):
            got = b.get_state(slot[i])
            assert np.array_equal(got, oracle_alone(oracle_mod, jobs[i], states[i], 0, steps_done[i])), i
            b.remove(slot[i])
        # second wave joins (slots are reused)
        for i in range(6, 12):
            slot[i] = b.add(jobs[i].W, jobs[i].H, jobs[i].seed, jobs[i].p)
            b.set_state(slot[i], states[i])
            steps_done[i] = 0
        b.step(13)
        for i in (0, 1, 3, 4):
            budget = [7, 11, 3, 20, 20, 9][i]
            steps_done[i] = min(budget, steps_done[i] + 13)
        for i in range(6, 12):
            steps_done[i] = 13
        for i in list(range(6)) + list(range(6, 12)):
            if i in (2, 5):
                continue
            got = b.get_state(slot[i])
            want = oracle_alone(oracle_mod, jobs[i], states[i], 0, steps_done[i])
            assert np.array_equal(got, want), (i, steps_done[i])
            assert b.time(slot[i]) == steps_done[i]


def test_batch_coarse_grain_and_arena_limits(pkg, oracle_mod):
    job = workloads.Lattice("cg", 256, 192, 0.3, 77, 0.01, 0, obstacle="walls")
    s0 = job.initial_state()
    need = pkg.Batch.lattice_bytes(job.W, job.H)
    with pkg.Batch(4 * need) as b:
        k = b.add(job.W, job.H, job.seed, job.p)
        extra = []
        with pytest.raises(pkg.FhpError) as ei:   # admission control: the arena fills up
            for _ in range(8):
                extra.append(b.add(job.W, job.H, 1, 0.0))
        assert ei.value.code == 2                 # FHP_ENOMEM
        assert 1 <= len(extra) <= 3
        for e in extra:
            b.remove(e)
        b.set_state(k, s0)
        b.step(9)
        counts, rho, ux, uy = b.coarse_grain(k, 64)
        want = oracle_alone(oracle_mod, job, s0, 0, 9)
        c_ref, rho_ref, _, _ = oracle_mod.coarse_grain(want, 64)
        assert np.array_equal(counts, c_ref)
        np.testing.assert_allclose(rho, rho_ref.astype(np.float32), rtol=1e-6)
        b.remove(k)
        k2 = b.add(job.W, job.H, 1, 0.0)          # memory came back
        assert b.count == 1 and k2 == k


def test_multi_step_kernel_edge_cases(pkg, oracle_mod):
    """Lattices of one and two tiles (a tile is its own or its only
    neighbour), one row of quads, single-step calls, members that stop
    inside a call, and a batch with more tiles than resident CTAs."""
    shapes = [(32, 2), (64, 4), (128, 8), (96, 258), (4128, 6), (2048, 64), (160, 130)]
    jobs = []
    for i, (W, H) in enumerate(shapes):
        jobs.append(workloads.Lattice(f"e{i}", W, H, 0.3, 31_000 + i, 0.02 if i % 2 else 0.0, 0,
                                      obstacle="points" if i % 3 else "none", point_frac=0.03))
    states = [j.initial_state() for j in jobs]
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        b.set_step_kernel(2)
        slots = []
        for j, s0 in zip(jobs, states):
            k = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(k, s0)
            slots.append(k)
        b.set_steps_left(slots[1], 3)
        b.set_steps_left(slots[4], 0)
        b.step(1)
        b.step(9)
        b.synchronize()
        for i, (j, s0, k) in enumerate(zip(jobs, states, slots)):
            n = {1: 3, 4: 0}.get(i, 10)
            want, _ = oracle_mod.run(s0, j.seed, 0, n, j.p)
            assert b.time(k) == n
            assert np.array_equal(b.get_state(k), want), (j.name, j.W, j.H)
    # many tiles: 600 lattices of 128 x 512 rows (one quad per row, 256 rows per tile)
    big = [workloads.Lattice(f"t{i}", 128, 512, 0.25, 50_000 + i, 0.0, 0) for i in range(600)]
    with pkg.Batch(sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in big) + (64 << 20)) as b:
        b.set_step_kernel(2)
        slots = []
        for j in big:
            k = b.add(j.W, j.H, j.seed, j.p)
            b.init_random(k, j.density)
            slots.append(k)
        b.step(6)
        for idx in (0, 1, 299, 599):
            j = big[idx]
            s0 = oracle_mod.init_random(j.W, j.H, j.seed, j.density)
            want, _ = oracle_mod.run(s0, j.seed, 0, 6, 0.0)
            assert np.array_equal(b.get_state(slots[idx]), want), j.name


def test_automatic_choice_is_tuned_online_and_exact(pkg, oracle_mod):
    """The automatic choice times both kernels at two tile sizes (256 and 128
    quads per tile) and blocked passes of 2 and 4 steps on a first long call
    (a sixth of its steps each) and records the fastest candidate for the
    batch's size class; members stay bit-exact throughout, across the
    re-tiling and the blocked passes."""
    jobs = small_ensemble(10, 5)
    states = [j.initial_state() for j in jobs]
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        assert b.step_kernel == 0
        slots = []
        for j, s0 in zip(jobs, states):
            k = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(k, s0)
            slots.append(k)
        assert b.tuned_kernel() == 0 and b.tuned_tile_quads() == 0 and b.tile_quads == 256
        b.set_graph_steps(8)
        b.step(14)                 # too short for a trial (four parts of at least 16 steps)
        b.synchronize()
        b.step(1)
        assert b.tuned_kernel() == 0
        b.step(95)
        b.synchronize()
        b.step(1)
        assert b.tuned_kernel() == 0   # 95 steps: too short for six parts of 16
        b.step(96)                 # a trial: 16 steps with each (kernel, tile size) and blocked k = 2, 4
        b.synchronize()
        b.step(3)                  # reads the trial's events
        assert b.tuned_kernel() in (1, 2)
        assert b.tuned_tile_quads() in (128, 256)
        assert b.tuned_temporal_block() in (1, 2, 4)
        assert b.tile_quads == b.tuned_tile_quads()
        b.step(6)
        b.synchronize()
        for j, s0, k in zip(jobs, states, slots):
            want, _ = oracle_mod.run(s0, j.seed, 0, 216, j.p)
            assert b.time(k) == 216
            assert np.array_equal(b.get_state(k), want), j.name


@pytest.mark.parametrize("kernel", [1, 2])
def test_tile_sizes_are_exact(pkg, oracle_mod, kernel):
    """Every tile size (64, 128, 256 quads per tile), changed between calls,
    gives each member its oracle run bit for bit with either batch kernel."""
    jobs = small_ensemble(6, 11)
    states = [j.initial_state() for j in jobs]
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        b.set_step_kernel(kernel)
        slots = []
        for j, s0 in zip(jobs, states):
            k = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(k, s0)
            slots.append(k)
        n = 0
        for quads, steps in ((64, 5), (256, 4), (128, 6), (64, 3)):
            b.set_tile_quads(quads)
            b.step(steps)
            n += steps
            assert b.tile_quads == quads
        b.synchronize()
        for j, s0, k in zip(jobs, states, slots):
            want, _ = oracle_mod.run(s0, j.seed, 0, n, j.p)
            assert np.array_equal(b.get_state(k), want), (j.name, kernel)
        with pytest.raises(pkg.FhpError):
            b.set_tile_quads(96)


def test_ensemble_512_in_the_benchmark_configuration(pkg, oracle_mod):
    """The 512-lattice ensemble (sides 128..2048, 1 % point obstacles) as the
    benchmark runs it (graphs of 64 launches, automatic kernel choice):
    every member equals its oracle run after 50 steps, and a seeded sample
    of 32 members equals theirs after the benchmark's 2,000 steps."""
    jobs = workloads.ensemble_512(512)
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (256 << 20)
    sample = sorted(np.random.Generator(np.random.PCG64(2000)).choice(len(jobs), 32, replace=False).tolist())
    with pkg.Batch(arena) as b:
        b.set_graph_steps(64)
        slots, states = [], []
        for j in jobs:
            s0 = j.initial_state()
            k = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(k, s0)
            slots.append(k)
            states.append(s0)
        b.step(6)
        b.step(44)
        for i, (j, k) in enumerate(zip(jobs, slots)):
            want, _ = oracle_mod.run(states[i], j.seed, 0, 50, j.p)
            assert b.time(k) == 50
            assert np.array_equal(b.get_state(k), want), j.name
        b.step(384)              # warm-up as in the benchmark: the automatic choice measures its candidates
        b.synchronize()
        b.step(2000 - 50 - 384)
        for i in sample:
            j = jobs[i]
            want, _ = oracle_mod.run(states[i], j.seed, 0, 2000, j.p)
            assert b.time(slots[i]) == 2000
            assert np.array_equal(b.get_state(slots[i]), want), (j.name, j.W, j.H)


@pytest.mark.parametrize("k", [2, 4])
def test_batch_temporal_block_matches_oracle(pkg, oracle_mod, k):
    """Blocked passes of k steps inside a batch (tiles of full rows stepped k
    times in shared memory): members too wide for a blocked tile, a ragged
    row, a 2-row lattice, a tall narrow one, FHP-I members, step budgets that
    end between passes, calls that are not multiples of k and a start step
    that is not either -- every member equals its oracle run alone."""
    jobs = small_ensemble(10, 21) + [
        workloads.Lattice("w8192", 8192, 20, 0.3, 31, 0.05, 0, obstacle="points", point_frac=0.01),
        workloads.Lattice("w12288", 12288, 8, 0.3, 35, 0.02, 0),
        workloads.Lattice("narrow", 32, 8, 0.4, 32, 0.02, 0),
        workloads.Lattice("ragged", 160, 50, 0.3, 33, 0.01, 0, obstacle="walls"),
        workloads.Lattice("tall", 96, 1030, 0.25, 34, 0.0, 0, obstacle="points", point_frac=0.02),
        workloads.Lattice("short", 640, 2, 0.3, 36, 0.03, 0),
    ]
    states = [j.initial_state() for j in jobs]
    budgets = [-1] * len(jobs)
    budgets[1], budgets[4], budgets[-3] = 5, 22, 9
    rules = [2] * len(jobs)
    rules[2] = rules[-2] = 1
    blocked = [pkg.Batch.block_rows(j.W, j.H, k) > 0 for j in jobs]
    assert not blocked[11] and blocked[12] and blocked[13] and blocked[14] and blocked[15]
    assert blocked[10] == (k == 2)
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        b.set_temporal_block(k)
        assert b.temporal_block == k
        b.set_step_kernel(1)
        b.set_graph_steps(4)
        slots = []
        for j, s0, bud, ru in zip(jobs, states, budgets, rules):
            s = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(s, s0)
            b.set_time(s, 3)
            if ru != 2:
                b.set_rules(s, ru)
            if bud >= 0:
                b.set_steps_left(s, bud)
            slots.append(s)
        l0 = b.kernel_launches
        b.step(13)
        b.step(10)
        b.synchronize()
        assert b.kernel_launches - l0 < 2 * 23   # blocked passes replace k launches each
        for j, s0, bud, ru, s in zip(jobs, states, budgets, rules, slots):
            n = 23 if bud < 0 else min(bud, 23)
            assert b.time(s) == 3 + n, j.name
            want, _ = oracle_mod.run(s0, j.seed, 3, n, j.p, rules=ru)
            got = b.get_state(s)
            assert np.array_equal(got, want), (j.name, j.W, j.H, k, int((got != want).sum()))
        with pytest.raises(pkg.FhpError):
            b.set_temporal_block(3)


def test_batch_temporal_block_with_multi_step_remainders(pkg, oracle_mod):
    """Temporal block 4 with the multi-step kernel for the remaining steps,
    switched off again between calls: the members still equal their oracle
    runs."""
    jobs = small_ensemble(8, 23)
    states = [j.initial_state() for j in jobs]
    arena = sum(pkg.Batch.lattice_bytes(j.W, j.H) for j in jobs) + (64 << 20)
    with pkg.Batch(arena) as b:
        b.set_step_kernel(2)
        b.set_temporal_block(4)
        slots = []
        for j, s0 in zip(jobs, states):
            s = b.add(j.W, j.H, j.seed, j.p)
            b.set_state(s, s0)
            slots.append(s)
        b.step(19)
        b.set_temporal_block(1)
        b.step(6)
        b.set_temporal_block(2)
        b.step(7)
        b.synchronize()
        for j, s0, s in zip(jobs, states, slots):
            want, _ = oracle_mod.run(s0, j.seed, 0, 32, j.p)
            assert np.array_equal(b.get_state(s), want), j.name


def test_automatic_choice_without_room_for_blocked_tables(pkg, oracle_mod):
    """An arena too full for the blocked passes' tables: a call long enough
    for a trial (six parts of 16 steps) tunes without the blocked candidates
    instead of failing, and the members stay exact."""
    job = workloads.Lattice("tight", 256, 192, 0.3, 78, 0.01, 0, obstacle="walls")
    s0 = job.initial_state()
    need = pkg.Batch.lattice_bytes(job.W, job.H)
    with pkg.Batch(4 * need) as b:
        b.set_graph_steps(8)
        k = b.add(job.W, job.H, job.seed, job.p)
        b.set_state(k, s0)
        b.step(1)                                  # the kernels' tables are in place
        fillers = []
        for w, h, tries in ((256, 192, 8), (128, 64, 8), (32, 2, 8)):
            for _ in range(tries):
                if b.count >= 16:                  # the descriptor table holds 16 members without growing
                    break
                try:
                    fillers.append(b.add(w, h, 5, 0.0))
                except pkg.FhpError as e:
                    assert e.code == 2             # FHP_ENOMEM
                    break
        assert b.free_bytes < 6 << 10, b.free_bytes   # less than one blocked-pass descriptor table
        assert b.tuned_kernel() == 0
        b.step(96)                                 # a trial: four parts of 24 steps, no blocked candidates
        b.synchronize()
        b.step(1)
        assert b.tuned_kernel() in (1, 2)
        assert b.tuned_temporal_block() == 1
        b.remove(fillers[0])                       # room for the read-back staging (W x H bytes)
        want, _ = oracle_mod.run(s0, job.seed, 0, 98, job.p)
        assert np.array_equal(b.get_state(k), want)
