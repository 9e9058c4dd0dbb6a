"""Serving loop: FHP simulation requests served by continuous batching.

Requests (lattice size, step count, seed, density, forcing probability,
optional obstacle map) arrive over time.  The server keeps every admitted
lattice resident in one device arena (a :class:`Batch`), admits waiting
requests in arrival order whenever the arena has room for them (admission by
HBM budget: a request waits while ``fhp_batch_add`` reports the arena full),
and advances all resident lattices together, one quantum of steps per
scheduling tick, through the batch kernel.  A lattice stops on its own when
its step budget is spent (the batch skips it); at the end of the tick its
result -- the coarse-grained fields of arXiv:1208.2428's model state, and
optionally the final node bytes -- is read back and its memory returned.

Every lattice evolves exactly as it would alone: its generator key, step
counter and obstacles are its own, so a result does not depend on what else
shared the device (the tests check this bit for bit).

All device work goes through the C ABI; this module is scheduling only.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from .fhp import Batch, FhpError, Lattice

FHP_ENOMEM = 2


@dataclass
class Request:
    """One simulation request.

    ``obstacles`` is None, an H x W mask (nonzero = solid), or a callable
    returning one (evaluated at admission, so that queued requests hold no
    mask).  The initial state is the library's generated Bernoulli state of
    ``density`` for ``seed`` (each of the seven bits of a fluid node set
    independently)."""
    width: int
    height: int
    steps: int
    seed: int = 0
    density: float = 0.25
    forcing_p: float = 0.0
    obstacles: np.ndarray | Callable[[], np.ndarray] | None = None
    cg_block: int = 32
    arrival: float = 0.0
    name: str = ""
    keep_state: bool = False
    obstacle_shapes: list | None = None   # (kind, a, b, c) shapes generated on the device instead of a mask

    @property
    def site_updates(self) -> int:
        return self.width * self.height * self.steps


@dataclass
class Completion:
    request: Request
    counts: np.ndarray
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    state: np.ndarray | None
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def queued(self) -> float:
        return self.admitted - self.arrival


@dataclass
class _Resident:
    request: Request
    admitted: float
    left: int


@dataclass
class ServerStats:
    completed: int = 0
    ticks: int = 0
    site_updates: int = 0
    quantum_steps: int = 0
    admissions_deferred: int = 0
    peak_resident: int = 0
    peak_resident_bytes: int = 0
    issued_site_updates: int = 0          # node updates launched (members with steps left)
    issued_solid_site_updates: int = 0    # ... of lattices that carry obstacles
    device_ms: float = 0.0                # batch-kernel time (time_device=True)
    device_launches: int = 0
    latencies: list = field(default_factory=list)

    def summary(self, span: float) -> dict:
        lat = np.asarray(self.latencies, dtype=np.float64)
        out = {
            "completed": self.completed,
            "ticks": self.ticks,
            "span_s": span,
            "gsups": (self.site_updates / span / 1e9) if span > 0 else 0.0,
            "peak_resident": self.peak_resident,
            "peak_resident_gb": self.peak_resident_bytes / 1e9,
            "admissions_deferred": self.admissions_deferred,
        }
        if lat.size:
            out.update({
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3),
                "max_ms": float(lat.max() * 1e3),
            })
        return out


class Server:
    """Continuous-batching server over one device arena of ``hbm_budget`` bytes.

    ``quantum_max``/``quantum_min`` bound the steps advanced per tick: a tick
    runs min(quantum_max, fewest steps any resident lattice still needs), but
    at least quantum_min, so that short requests finish close to their last
    step while long ones share launches.  ``graph_steps`` is the length of the
    captured CUDA graph of batch launches.  ``temporal_block`` (1, 2 or 4)
    is the batch's temporal block.  ``batch`` substitutes another object with
    the :class:`Batch` interface (the scheduling tests use a host-only
    stand-in)."""

    def __init__(self, hbm_budget: int, quantum_max: int = 64, quantum_min: int = 8, graph_steps: int = 16,
                 device=None, stream=None, clock: Callable[[], float] | None = None, batch=None,
                 time_device: bool = False, pipeline: bool = True, temporal_block: int = 1):
        if quantum_min < 1 or quantum_max < quantum_min:
            raise ValueError("need 1 <= quantum_min <= quantum_max")
        self.batch = batch if batch is not None else Batch(hbm_budget, device=device, stream=stream)
        self.batch.set_graph_steps(graph_steps)
        # Temporal block of the batch: quanta (8..64 steps) are too short for a
        # tuning trial that includes blocked passes (six parts of at least 16
        # steps), so it is set here -- 1 (no blocking, the default) or 2 / 4
        # (blocked passes for the lattices narrow enough, the rest of each
        # quantum on the step kernel); the kernel and tile size are still tuned
        # online within a quantum.
        if hasattr(self.batch, "set_temporal_block"):
            self.batch.set_temporal_block(int(temporal_block))
        self.hbm_budget = int(hbm_budget)
        self.quantum_max = int(quantum_max)
        self.quantum_min = int(quantum_min)
        self._clock = clock or time.perf_counter
        self._t0 = self._clock()
        self.waiting: deque[Request] = deque()
        self.resident: dict[int, _Resident] = {}
        self.resident_bytes = 0
        self._blocked = False
        self.time_device = time_device
        # Pipelining: the next quantum is queued before the previous one is
        # waited for, and finished lattices are read back on a side stream
        # while it runs, so the device does not idle between quanta.
        self.pipeline = pipeline
        self._inflight: deque = deque()   # (start event, end event, finishing slots) per issued quantum
        self._retiring: list[int] = []    # finished slots whose read-back could not start yet
        self._virtual = False       # serve(realtime=False): the clock counts ticks
        self._vtick = 0
        self.stats = ServerStats()

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def now(self) -> float:
        if self._virtual:
            return float(self._vtick)
        return self._clock() - self._t0

    def reset_clock(self):
        self._t0 = self._clock()

    # -- requests ---------------------------------------------------------------
    def submit(self, req: Request):
        """Queue a request (it is admitted by a later tick)."""
        need = self.batch.lattice_bytes(req.width, req.height)
        if need == 0:
            raise ValueError(f"{req.name}: invalid lattice {req.width} x {req.height}")
        if need + self.staging_bytes(req) + (64 << 10) > self.hbm_budget:
            raise ValueError(f"{req.name}: a {req.width} x {req.height} lattice never fits the budget")
        if req.steps < 0:
            raise ValueError("steps must be >= 0")
        if req.width % req.cg_block or req.height % req.cg_block:
            raise ValueError("cg_block must divide the lattice sides")
        self.waiting.append(req)

    @property
    def idle(self) -> bool:
        return not self.waiting and not self.resident

    @staticmethod
    def staging_bytes(req: Request) -> int:
        """Transient arena bytes a request's set-up or read-back may take:
        its obstacle mask or final node bytes (H x W) and its coarse-grained
        fields (9 counts and 3 floats per block), with alignment slack."""
        cells = (req.width // req.cg_block) * (req.height // req.cg_block)
        return req.width * req.height + cells * 48 + 4096

    def _admit(self):
        b = self.batch
        while self.waiting:
            if self._blocked:
                return                      # a finished lattice is still waiting to be read back
            req = self.waiting[0]
            # Room for the lattice plus the largest transient staging that any
            # resident lattice or this one may need later, so that a finished
            # lattice can always be read back.
            reserve = max([self.staging_bytes(r.request) for r in self.resident.values()]
                          + [self.staging_bytes(req)])
            if b.free_bytes < b.lattice_bytes(req.width, req.height) + reserve:
                self.stats.admissions_deferred += 1
                return
            try:
                slot = b.add(req.width, req.height, req.seed, req.forcing_p)
            except FhpError as e:
                if e.code != FHP_ENOMEM:
                    raise
                self.stats.admissions_deferred += 1
                return                      # first in line waits for memory (FIFO)
            try:
                if req.obstacle_shapes:
                    b.load_obstacle_shapes(slot, req.obstacle_shapes)
                else:
                    mask = req.obstacles() if callable(req.obstacles) else req.obstacles
                    if mask is not None:
                        b.load_obstacles(slot, mask)
                b.init_random(slot, req.density)
                b.set_steps_left(slot, req.steps)
            except FhpError as e:
                b.remove(slot)
                if e.code != FHP_ENOMEM:
                    raise
                self.stats.admissions_deferred += 1
                return
            self.waiting.popleft()
            self.resident[slot] = _Resident(req, self.now(), req.steps)
            self.resident_bytes += self.batch.lattice_bytes(req.width, req.height)
        return

    def _event(self):
        stream = getattr(self.batch, "stream", None)
        if stream is None:
            return None
        import torch
        ev = torch.cuda.Event(enable_timing=self.time_device)
        ev.record(stream)
        return ev

    def _complete(self, slot: int, results, state) -> Completion:
        r = self.resident.pop(slot)
        req = r.request
        self.batch.remove(slot, wait=False) if self.pipeline else self.batch.remove(slot)
        self.resident_bytes -= self.batch.lattice_bytes(req.width, req.height)
        counts, rho, ux, uy = results
        c = Completion(req, counts, rho, ux, uy, state, req.arrival, r.admitted, self.now())
        self.stats.completed += 1
        self.stats.site_updates += req.site_updates
        self.stats.latencies.append(c.latency)
        return c

    def _retire(self, slots: list[int], after_event=None) -> list[Completion]:
        """Read back finished lattices (their last quantum is complete) and
        return their memory."""
        done = []
        b = self.batch
        self._blocked = False
        handles = {}
        if self.pipeline:
            for slot in slots:                       # all read-backs in flight together
                handles[slot] = b.coarse_grain_begin(slot, self.resident[slot].request.cg_block, after_event)
        for slot in slots:
            req = self.resident[slot].request
            try:
                if self.pipeline:
                    results = b.coarse_grain_finish(handles[slot])
                else:
                    results = b.coarse_grain(slot, req.cg_block)
                state = b.get_state(slot) if req.keep_state else None
            except FhpError as e:
                if e.code != FHP_ENOMEM:
                    raise
                self._blocked = True        # no staging room now: read it back on a later tick
                self._retiring.append(slot)
                continue
            done.append(self._complete(slot, results, state))
        return done

    def _finish_quantum(self) -> list[Completion]:
        """Wait for the oldest quantum in flight and retire the lattices it finished."""
        start, end, fin = self._inflight.popleft()
        if end is not None:
            end.synchronize()
            if self.time_device and start is not None:
                self.stats.device_ms += start.elapsed_time(end)
        else:
            self.batch.synchronize()
        retry, self._retiring = self._retiring, []
        return self._retire(retry + fin, end)

    def tick(self) -> list[Completion]:
        """One scheduling round: queue a quantum of steps for the lattices
        still running, admit waiting requests behind it, then wait for the
        previous quantum (pipelined) or this one, and retire the lattices it
        finished."""
        b = self.batch
        q = 0
        running = [r for r in self.resident.values() if r.left > 0]
        if running:
            fewest = min(r.left for r in running)
            q = max(self.quantum_min, min(self.quantum_max, fewest))
            launches = b.kernel_launches if self.time_device else 0
            start = self._event()
            b.step(q)
            end = self._event()
            if self.time_device:
                self.stats.device_launches += b.kernel_launches - launches
            fin = []
            for slot, r in self.resident.items():
                if r.left == 0:
                    continue
                k = min(q, r.left)
                self.stats.issued_site_updates += k * r.request.width * r.request.height
                self.stats.issued_solid_site_updates += k * r.request.width * r.request.height \
                    if (r.request.obstacles is not None or r.request.obstacle_shapes) else 0
                r.left -= k
                if r.left == 0:
                    fin.append(slot)
            self._inflight.append((start, end, fin))
        else:
            # Lattices admitted with no steps to run are finished as they stand.
            fin = [slot for slot, r in self.resident.items() if r.left == 0
                   and not any(slot in f for _, _, f in self._inflight) and slot not in self._retiring]
            if fin:
                self._inflight.append((None, self._event(), fin))
        self._admit()
        self.stats.peak_resident = max(self.stats.peak_resident, len(self.resident))
        self.stats.peak_resident_bytes = max(self.stats.peak_resident_bytes, self.resident_bytes)
        done = []
        keep = 1 if (self.pipeline and running) else 0
        while len(self._inflight) > keep:
            done.extend(self._finish_quantum())
        if not self._inflight and self._retiring:
            done.extend(self._retire(self._retiring[:], None))
            self._retiring = [s for s in self._retiring if s in self.resident]
        self.stats.ticks += 1
        self.stats.quantum_steps += q
        self._vtick += 1
        return done

    def serve(self, requests: list[Request], realtime: bool = True, max_ticks: int | None = None) -> list[Completion]:
        """Serve a trace: each request is submitted once the clock passes its
        ``arrival`` (seconds after the call).  With ``realtime`` False the
        clock is the tick counter instead (a request arrives at tick
        ceil(arrival)), which makes the schedule deterministic."""
        trace = deque(sorted(requests, key=lambda r: r.arrival))
        out: list[Completion] = []
        self._virtual = not realtime
        self._vtick = 0
        self.reset_clock()
        ticks = 0
        try:
            while trace or not self.idle:
                now = self.now()
                while trace and trace[0].arrival <= now:
                    self.submit(trace.popleft())
                if self.idle:
                    if realtime:
                        time.sleep(max(0.0, min(trace[0].arrival - self.now(), 0.05)))
                    else:
                        self._vtick += 1
                    continue
                out.extend(self.tick())
                ticks += 1
                if max_ticks is not None and ticks >= max_ticks:
                    break
        finally:
            self._virtual = False
        return out


def serve_sequential(requests: list[Request], realtime: bool = True, device=None) -> list[Completion]:
    """The same trace served one lattice at a time in arrival order, each
    with its own launches (the per-lattice comparison for :class:`Server`)."""
    out: list[Completion] = []
    clock = time.perf_counter
    t0 = clock()
    tick = 0
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime:
            wait = req.arrival - (clock() - t0)
            if wait > 0:
                time.sleep(wait)
        start = (clock() - t0) if realtime else float(max(tick, req.arrival))
        with Lattice(req.width, req.height, seed=req.seed, forcing_p=req.forcing_p, device=device) as lat:
            if req.obstacle_shapes:
                lat.load_obstacle_shapes(req.obstacle_shapes)
            else:
                mask = req.obstacles() if callable(req.obstacles) else req.obstacles
                if mask is not None:
                    lat.load_obstacles(mask)
            lat.init_random(req.density)
            lat.step(req.steps)
            counts, rho, ux, uy = lat.coarse_grain(req.cg_block)
            state = lat.get_state() if req.keep_state else None
        tick += 1
        finished = (clock() - t0) if realtime else float(tick)
        out.append(Completion(req, counts, rho, ux, uy, state, req.arrival, start, finished))
    return out


def summarize(completions: list[Completion]) -> dict:
    """p50/p99 latency and aggregate throughput of a served trace."""
    if not completions:
        return {"completed": 0}
    lat = np.array([c.latency for c in completions])
    first = min(c.arrival for c in completions)
    last = max(c.finished for c in completions)
    sups = sum(c.request.site_updates for c in completions)
    return {
        "completed": len(completions),
        "span_s": last - first,
        "gsups": sups / (last - first) / 1e9 if last > first else 0.0,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "max_ms": float(lat.max() * 1e3),
    }
