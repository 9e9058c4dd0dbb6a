"""Seeded synthetic inputs for the FHP lattice gas (shared by tests, bench, smoke).

This module only builds inputs: obstacle geometry and random initial
occupations.  It holds none of the model's arithmetic (no motion, no
scattering, no forcing, no coarse-graining), so both the CUDA path and the
CPU oracle can be fed from it without sharing method code.

Node byte layout (arXiv:1208.2428, Section 2, Fig. 1): bits 0-5 moving
particles, bit 6 rest particle, bit 7 solid (boundary) node.

Workloads (the five evaluation configurations of this project; the paper's
own runs, Section 4, use a 29,970 x 27,990 lattice with walls at the top and
bottom, periodic x and horizontal forcing):

  * ``periodic_256``   256 x 256, fully periodic, density 0.3, seed 1, 100 steps.
  * ``channel_4096x1024``  walls on rows 0 and H-1, density 0.2, p = 1e-3,
    seed 2, 10,000 steps, 32 x 32 coarse-graining every 1,000 steps.
  * ``cylinder_16384x4096``  walls, a solid disc of radius H/16 centred at
    (W/4, H/2), density 0.25, p = 5e-4, seed 3, 1,000 steps.
  * ``cylinder_paper_size``  the same geometry on the paper's GPU lattice
    (29,970 x 27,990, width rounded up to 29,984 so that W is a multiple of 32).
  * ``ensemble_512``   512 periodic lattices, sides uniform in {128, 192, ..., 2048},
    density U(0.1, 0.5), 1 % random point obstacles, seeds 1000 + i, p = 0.
  * ``serving_jobs``   Poisson arrivals (200/s) of jobs with log-uniform sides
    in [256, 8192] (multiples of 64) and steps in [100, 10000], density
    U(0.1, 0.4); half of them carry the cylinder geometry with p = 5e-4.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SOLID = 0x80


def channel_walls(W: int, H: int) -> np.ndarray:
    """Solid mask (bool H x W) with solid rows 0 and H-1."""
    m = np.zeros((H, W), dtype=bool)
    m[0, :] = True
    m[H - 1, :] = True
    return m


def cylinder_mask(W: int, H: int, walls: bool = True) -> np.ndarray:
    """Walls plus a solid disc of radius H/16 at (W/4, H/2) in index coordinates.

    Node (x, y) is solid iff (x - W/4)^2 + (y - H/2)^2 <= (H/16)^2, with x and
    y the array indices (the half-cell shift of odd rows is ignored)."""
    cx, cy, r = W // 4, H // 2, H // 16
    m = channel_walls(W, H) if walls else np.zeros((H, W), dtype=bool)
    y0, y1 = max(cy - r, 0), min(cy + r + 1, H)
    x0, x1 = max(cx - r, 0), min(cx + r + 1, W)
    yy, xx = np.mgrid[y0:y1, x0:x1]
    m[y0:y1, x0:x1] |= (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
    return m


def cylinder_shapes(W: int, H: int, walls: bool = True) -> list[tuple[int, int, int, int]]:
    """The cylinder_mask geometry as (kind, a, b, c) shapes for device-side
    generation: kind 2 = rows a <= y < b, kind 1 = disc of radius c at (a, b)."""
    shapes = [(2, 0, 1, 0), (2, H - 1, H, 0)] if walls else []
    return shapes + [(1, W // 4, H // 2, H // 16)]


def random_points(W: int, H: int, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Each node solid independently with probability ``frac``."""
    return rng.random((H, W)) < frac


def bernoulli_lattice(W: int, H: int, density: float, seed: int,
                      solid: np.ndarray | None = None, chunk_rows: int = 512) -> np.ndarray:
    """H x W node bytes: each of bits 0..6 set i.i.d. with probability
    round(density * 2^16) / 2^16 on fluid nodes; solid nodes carry only bit 7."""
    if W % 32 or H % 2:
        raise ValueError("W must be a multiple of 32 and H even")
    rng = np.random.Generator(np.random.PCG64(seed))
    thr = int(round(density * 65536))
    weights = (1 << np.arange(7)).astype(np.uint8)
    out = np.empty((H, W), dtype=np.uint8)
    for r0 in range(0, H, chunk_rows):
        r1 = min(H, r0 + chunk_rows)
        u = rng.integers(0, 65536, size=(r1 - r0, W, 7), dtype=np.uint16)
        bits = (u < thr).astype(np.uint8)
        out[r0:r1] = (bits * weights).sum(axis=-1, dtype=np.uint8)
    if solid is not None:
        out[solid] = SOLID
    return out


@dataclass
class Lattice:
    """One synthetic lattice job."""
    name: str
    W: int
    H: int
    density: float
    seed: int
    p: float
    steps: int
    obstacle: str = "none"        # none | walls | cylinder | points
    point_frac: float = 0.0
    cg_block: int = 32
    cg_every: int = 0
    arrival: float = 0.0          # seconds, serving jobs only

    def solid(self) -> np.ndarray | None:
        if self.obstacle == "none":
            return None
        if self.obstacle == "walls":
            return channel_walls(self.W, self.H)
        if self.obstacle == "cylinder":
            return cylinder_mask(self.W, self.H)
        if self.obstacle == "points":
            rng = np.random.Generator(np.random.PCG64(self.seed + 7919))
            return random_points(self.W, self.H, self.point_frac, rng)
        raise ValueError(self.obstacle)

    def initial_state(self) -> np.ndarray:
        return bernoulli_lattice(self.W, self.H, self.density, self.seed, self.solid())

    @property
    def nodes(self) -> int:
        return self.W * self.H


def periodic_256() -> Lattice:
    return Lattice("periodic_256", 256, 256, 0.3, 1, 0.0, 100)


def channel_4096x1024() -> Lattice:
    return Lattice("channel_4096x1024", 4096, 1024, 0.2, 2, 1e-3, 10_000,
                   obstacle="walls", cg_block=32, cg_every=1000)


def cylinder_16384x4096() -> Lattice:
    return Lattice("cylinder_16384x4096", 16384, 4096, 0.25, 3, 5e-4, 1000, obstacle="cylinder")


def cylinder_paper_size() -> Lattice:
    return Lattice("cylinder_29984x27990", 29984, 27990, 0.25, 3, 5e-4, 100, obstacle="cylinder")


def cylinder_scaled(W: int, H: int, seed: int = 3, steps: int = 100) -> Lattice:
    return Lattice(f"cylinder_{W}x{H}", W, H, 0.25, seed, 5e-4, steps, obstacle="cylinder")


def ensemble_512(count: int = 512, master_seed: int = 4, steps: int = 2000) -> list[Lattice]:
    rng = np.random.Generator(np.random.PCG64(master_seed))
    sides = np.arange(128, 2049, 64)
    out = []
    for i in range(count):
        W = int(rng.choice(sides))
        H = int(rng.choice(sides))
        rho = float(rng.uniform(0.1, 0.5))
        out.append(Lattice(f"ensemble_{i}", W, H, rho, 1000 + i, 0.0, steps,
                           obstacle="points", point_frac=0.01))
    return out


def serving_jobs(count: int = 2000, master_seed: int = 5, rate: float = 200.0,
                 side_range=(256, 8192), step_range=(100, 10_000)) -> list[Lattice]:
    rng = np.random.Generator(np.random.PCG64(master_seed))
    t = 0.0
    jobs = []
    lo, hi = np.log(side_range[0]), np.log(side_range[1])
    slo, shi = np.log(step_range[0]), np.log(step_range[1])
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        W = int(max(64, round(float(np.exp(rng.uniform(lo, hi))) / 64) * 64))
        H = int(max(64, round(float(np.exp(rng.uniform(lo, hi))) / 64) * 64))
        steps = int(round(float(np.exp(rng.uniform(slo, shi)))))
        rho = float(rng.uniform(0.1, 0.4))
        cyl = bool(rng.random() < 0.5)
        jobs.append(Lattice(f"job_{i}", W, H, rho, 5_000_000 + i, 5e-4 if cyl else 0.0, steps,
                            obstacle="cylinder" if cyl else "none", arrival=t))
    return jobs
