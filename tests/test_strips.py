"""Row-strip decomposition across ranks (the paper's multi-GPU runs,
Table 1), on the CPU: the plan, and the exchange protocol driven with the
oracle as the strip stepper -- in one process and on gloo ranks (world sizes
2 and 3) -- against the undivided oracle run."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import workloads
from paper_1208_2428_gb300.strips import DistExchange, LocalExchange, StripDomain, StripPlan


class OracleStrip:
    """A strip advanced by the CPU oracle (rows keyed on the lattice's rows)."""

    def __init__(self, oracle_mod, plan, r, state, seed, p, t0=0):
        self.oracle, self.plan, self.r = oracle_mod, plan, r
        self.rows = np.ascontiguousarray(state[plan.global_rows(r)])
        self.seed, self.p, self.t = seed, p, t0

    def get_rows(self, y0, n):
        import torch
        return torch.from_numpy(self.rows[y0:y0 + n].copy())

    def empty_rows(self, n):
        import torch
        return torch.empty((n, self.plan.width), dtype=torch.uint8)

    def set_rows(self, y0, rows):
        self.rows[y0:y0 + rows.shape[0]] = rows.numpy()

    def step(self, n):
        self.rows, _ = self.oracle.run_rows(self.rows, self.seed, self.t, n, self.p, self.plan.row_base(self.r),
                                            self.plan.height)
        self.t += n

    def owned(self):
        h = self.plan.halo
        return self.rows[h:h + self.plan.owned(self.r)]


def test_plan_partitions_rows_in_even_pairs():
    for H, parts, halo in [(64, 2, 2), (66, 3, 4), (1024, 7, 8), (8, 1, 2), (12, 3, 2)]:
        plan = StripPlan(64, H, parts, halo)
        rows = np.concatenate([np.arange(plan.y0(r), plan.y1(r)) for r in range(parts)])
        assert np.array_equal(rows, np.arange(H))
        for r in range(parts):
            assert plan.y0(r) % 2 == 0 and plan.row_base(r) % 2 == 0
            assert plan.local_height(r) % 2 == 0 and plan.owned(r) >= halo
            g = plan.global_rows(r)
            assert g[halo] == plan.y0(r) and g[halo + plan.owned(r) - 1] == plan.y1(r) - 1
            # ghost rows are the neighbours' owned rows
            assert set(g[:halo]) <= set(range(plan.y0(plan.below(r)), plan.y1(plan.below(r)))) or parts == 1
    with pytest.raises(ValueError):
        StripPlan(64, 8, 3, 4)          # a strip would own fewer rows than the halo
    with pytest.raises(ValueError):
        StripPlan(64, 16, 2, 3)         # odd halo


@pytest.mark.parametrize("parts,halo,steps", [(1, 2, 7), (2, 2, 9), (3, 4, 13), (5, 2, 10), (4, 6, 17)])
def test_strips_in_one_process_equal_the_whole_lattice(oracle_mod, parts, halo, steps):
    W, H, seed, p = 96, 40, 77, 0.05
    job = workloads.Lattice("strip", W, H, 0.3, seed, p, 0, obstacle="points", point_frac=0.05)
    s0 = job.initial_state()
    plan = StripPlan(W, H, parts, halo)
    strips = [OracleStrip(oracle_mod, plan, r, s0, seed, p, t0=5) for r in range(parts)]
    dom = StripDomain(plan, strips, LocalExchange())
    dom.step(steps)
    got = np.concatenate([s.owned() for s in strips])
    want, _ = oracle_mod.run(s0, seed, 5, steps, p)
    assert np.array_equal(got, want)
    assert dom.exchanges == -(-steps // halo)


def test_stale_ghost_rows_break_the_result(oracle_mod):
    """Without the exchange the strips drift from the whole lattice: the
    protocol, not the stepper, makes the strips exact."""
    W, H, seed = 64, 24, 3
    s0 = workloads.bernoulli_lattice(W, H, 0.35, seed)
    plan = StripPlan(W, H, 3, 2)
    strips = [OracleStrip(oracle_mod, plan, r, s0, seed, 0.0) for r in range(3)]
    for _ in range(4):
        for s in strips:
            s.step(2)                  # no exchange between rounds
    got = np.concatenate([s.owned() for s in strips])
    want, _ = oracle_mod.run(s0, seed, 0, 8, 0.0)
    assert not np.array_equal(got, want)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, halo, steps):
    import torch.distributed as dist

    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        W, H, seed, p = 128, 36, 91, 0.03
        s0 = workloads.Lattice("dist", W, H, 0.25, seed, p, 0, obstacle="walls").initial_state()
        plan = StripPlan(W, H, world, halo)
        strip = OracleStrip(oracle, plan, rank, s0, seed, p)
        dom = StripDomain(plan, [strip], DistExchange())
        dom.step(steps)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), strip.owned())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,halo,steps", [(2, 2, 11), (3, 4, 9)])
def test_gloo_ranks_equal_the_whole_lattice(oracle_mod, tmp_path, world, halo, steps):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), halo, steps), nprocs=world, join=True)
    W, H, seed, p = 128, 36, 91, 0.03
    s0 = workloads.Lattice("dist", W, H, 0.25, seed, p, 0, obstacle="walls").initial_state()
    want, _ = oracle_mod.run(s0, seed, 0, steps, p)
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)])
    assert np.array_equal(got, want)
