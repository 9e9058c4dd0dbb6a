"""Row-strip decomposition of one FHP lattice over several devices.

The paper runs one lattice on two GPUs and finds practically linear scaling
(Table 1, mGPU).  Here the W x H lattice is cut into horizontal strips of
whole, even-aligned row pairs, one strip per rank.  A strip is a lattice of
its own (:class:`Lattice`) holding its owned rows plus ``halo`` ghost rows
above and below; its row offset makes every owned row draw the whole
lattice's random words (chirality and forcing are keyed on the global row).
Every ``halo`` steps the ranks exchange their edge rows:

* a rank sends its lowest ``halo`` owned rows to the rank below, where they
  become that rank's upper ghost rows, and its highest ``halo`` owned rows
  to the rank above (its lower ghost rows); the lattice is periodic in y, so
  rank 0's lower neighbour is the last rank;
* then every rank advances up to ``halo`` steps.  A step of the strip reads
  one row above and below, so after j steps the outermost j ghost rows on
  each side are stale and the owned rows are still exact: they equal the
  rows of the undivided lattice.

Only the seven state planes travel (the solid plane is static and each
strip holds its ghost rows' obstacles from the start).  The exchange is one
pair of sends and receives per neighbour and round, of 7 x halo x pitch
words, via ``torch.distributed`` (NCCL for device tensors, gloo for host
tensors) or, for strips that live in one process, direct copies.

The plan and the exchange protocol are independent of what advances a strip:
:class:`DeviceStrip` does it with the library's kernels; the tests also drive
the same protocol with the CPU oracle on gloo ranks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class StripPlan:
    """Rows of strip r: [y0(r), y1(r)), split in whole row pairs as evenly as
    possible; every strip carries ``halo`` (even, >= 2) ghost rows per side
    and must own at least ``halo`` rows."""
    width: int
    height: int
    parts: int
    halo: int = 2

    def __post_init__(self):
        if self.width % 32 or self.width < 32 or self.height % 2 or self.height < 2:
            raise ValueError("width must be a positive multiple of 32 and height even")
        if self.halo < 2 or self.halo % 2:
            raise ValueError("halo must be even and >= 2")
        if self.parts < 1:
            raise ValueError("parts must be >= 1")
        for r in range(self.parts):
            if self.owned(r) < self.halo:
                raise ValueError(f"strip {r} owns {self.owned(r)} rows, fewer than the halo {self.halo}")

    def y0(self, r: int) -> int:
        pairs = self.height // 2
        return 2 * ((r * pairs) // self.parts)

    def y1(self, r: int) -> int:
        return self.y0(r + 1) if r + 1 < self.parts else self.height

    def owned(self, r: int) -> int:
        return self.y1(r) - self.y0(r)

    def local_height(self, r: int) -> int:
        return self.owned(r) + 2 * self.halo

    def row_base(self, r: int) -> int:
        """Lattice row of the strip's array row 0 (may be negative: rows wrap)."""
        return self.y0(r) - self.halo

    def below(self, r: int) -> int:
        return (r - 1) % self.parts

    def above(self, r: int) -> int:
        return (r + 1) % self.parts

    def global_rows(self, r: int) -> np.ndarray:
        """Lattice row of every array row of strip r."""
        return (self.row_base(r) + np.arange(self.local_height(r))) % self.height

    # array rows (local indices) of the strip's edge regions
    def send_down_rows(self, r: int) -> tuple[int, int]:
        return self.halo, self.halo                              # lowest owned rows

    def send_up_rows(self, r: int) -> tuple[int, int]:
        return self.halo + self.owned(r) - self.halo, self.halo  # highest owned rows

    def ghost_below_rows(self, r: int) -> tuple[int, int]:
        return 0, self.halo

    def ghost_above_rows(self, r: int) -> tuple[int, int]:
        return self.halo + self.owned(r), self.halo


class LocalExchange:
    """All strips in one process: ghost rows are copied strip to strip."""

    def exchange(self, plan: StripPlan, strips: list):
        outgoing = []
        for r, s in enumerate(strips):
            outgoing.append((s.get_rows(*plan.send_down_rows(r)), s.get_rows(*plan.send_up_rows(r))))
        for r, s in enumerate(strips):
            from_above = outgoing[plan.above(r)][0]   # the upper neighbour's lowest owned rows
            from_below = outgoing[plan.below(r)][1]   # the lower neighbour's highest owned rows
            s.set_rows(plan.ghost_above_rows(r)[0], from_above)
            s.set_rows(plan.ghost_below_rows(r)[0], from_below)


class DistExchange:
    """One strip per rank of a torch.distributed process group.  NCCL moves
    device tensors directly; on a gloo group the rows of device strips are
    staged through host memory (``via_host``, the default for gloo).  With a
    single rank the strip exchanges with itself (periodic wrap)."""

    def __init__(self, group=None, via_host=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.via_host = (dist.get_backend(group) == "gloo") if via_host is None else bool(via_host)

    def exchange(self, plan: StripPlan, strips: list):
        if len(strips) != 1 or plan.parts != self.size:
            raise ValueError("one strip per rank, plan.parts == world size")
        dist, r, s = self.dist, self.rank, strips[0]
        down = s.get_rows(*plan.send_down_rows(r))
        up = s.get_rows(*plan.send_up_rows(r))
        if self.size == 1:
            s.set_rows(plan.ghost_above_rows(r)[0], down)
            s.set_rows(plan.ghost_below_rows(r)[0], up)
            return
        import torch
        device = down.device if (self.via_host and down.is_cuda) else None
        if device is not None:
            # The rows were gathered on the strip's stream: wait, then stage
            # them in host memory for the host-memory backend.
            torch.cuda.synchronize(device)
            down, up = down.cpu(), up.cpu()
        from_above = torch.empty_like(down)
        from_below = torch.empty_like(down)
        below, above = plan.below(r), plan.above(r)
        ops = [dist.P2POp(dist.isend, down, below, self.group), dist.P2POp(dist.isend, up, above, self.group),
               dist.P2POp(dist.irecv, from_above, above, self.group),
               dist.P2POp(dist.irecv, from_below, below, self.group)]
        if self.size == 2:
            # the same peer is above and below: tag the two directions apart
            ops = [dist.P2POp(dist.isend, down, below, self.group, tag=1),
                   dist.P2POp(dist.isend, up, above, self.group, tag=2),
                   dist.P2POp(dist.irecv, from_above, above, self.group, tag=1),
                   dist.P2POp(dist.irecv, from_below, below, self.group, tag=2)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        if device is not None:
            from_above, from_below = from_above.to(device), from_below.to(device)
            torch.cuda.synchronize(device)
        s.set_rows(plan.ghost_above_rows(r)[0], from_above)
        s.set_rows(plan.ghost_below_rows(r)[0], from_below)


class StripDomain:
    """Advances the strips of one lattice (those this process holds) with
    halo exchanges every ``plan.halo`` steps."""

    def __init__(self, plan: StripPlan, strips: list, exchange):
        self.plan = plan
        self.strips = strips
        self.exchange_impl = exchange
        self.exchanges = 0

    def step(self, n: int):
        left = int(n)
        while left > 0:
            self.exchange_impl.exchange(self.plan, self.strips)
            self.exchanges += 1
            k = min(left, self.plan.halo)
            for s in self.strips:
                s.step(k)
            left -= k


class DeviceStrip:
    """A strip on a CUDA device: a :class:`Lattice` of the strip's rows with
    the row offset of its place in the whole lattice.  Rows travel as int32
    tensors [7, rows, pitch] of bit-plane words."""

    def __init__(self, plan: StripPlan, r: int, seed: int, forcing_p: float = 0.0, device=None, stream=None):
        from .fhp import Lattice
        self.plan, self.r = plan, r
        self.lattice = Lattice(plan.width, plan.local_height(r), seed=seed, forcing_p=forcing_p, device=device,
                               stream=stream)
        self.lattice.set_row_offset(plan.row_base(r))

    def close(self):
        self.lattice.close()

    def set_from_global(self, state: np.ndarray):
        """Load the strip's rows (owned and ghost) from the whole lattice's H x W bytes."""
        self.lattice.set_state(np.ascontiguousarray(state[self.plan.global_rows(self.r)]))

    def owned_state(self) -> np.ndarray:
        s = self.lattice.get_state()
        h = self.plan.halo
        return s[h:h + self.plan.owned(self.r)]

    def set_time(self, t: int):
        self.lattice.set_time(t)

    def get_rows(self, y0: int, n: int):
        return self.lattice.get_rows_tensor(y0, n)

    def empty_rows(self, n: int):
        torch = __import__("torch")
        return torch.empty((7, n, self.lattice.row_pitch_words), dtype=torch.int32, device=self.lattice.device)

    def set_rows(self, y0: int, rows):
        self.lattice.set_rows_tensor(y0, rows)

    def step(self, n: int):
        self.lattice.step(n)
