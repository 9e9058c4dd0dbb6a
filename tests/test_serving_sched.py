"""Scheduling logic of the serving loop on the host, with a stand-in for the
device batch: FIFO admission by memory budget, step quanta, step budgets and
read-back headroom.  (The device path is covered by test_gpu_serving.py.)"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1208_2428_gb300.fhp import FhpError
from paper_1208_2428_gb300.serving import Request, Server, summarize


class FakeBatch:
    """Arena accounting and per-member step budgets, no device."""

    def __init__(self, arena_bytes):
        self.capacity = arena_bytes
        self.used = 0
        self.members = {}
        self.staging_peak = 0
        self.step_calls = []
        self.log = []

    @staticmethod
    def lattice_bytes(w, h):
        if w < 32 or w % 32 or h < 2 or h % 2:
            return 0
        return 2 * w * h

    @property
    def free_bytes(self):
        return self.capacity - self.used

    def set_graph_steps(self, n):
        self.graph = n

    def set_temporal_block(self, k):
        self.temporal_block = k

    def add(self, w, h, seed, p):
        need = self.lattice_bytes(w, h)
        if need > self.free_bytes:
            raise FhpError(2, "arena full")
        slot = next(i for i in range(10_000) if i not in self.members)
        self.members[slot] = {"w": w, "h": h, "seed": seed, "left": -1, "t": 0, "bytes": need}
        self.used += need
        self.log.append(("add", seed))
        return slot

    def _stage(self, n):
        if n > self.free_bytes:
            raise FhpError(2, "no staging room")
        self.staging_peak = max(self.staging_peak, self.used + n)

    def load_obstacles(self, slot, mask):
        m = self.members[slot]
        assert mask.shape == (m["h"], m["w"])
        self._stage(m["w"] * m["h"])

    def init_random(self, slot, density):
        self.members[slot]["density"] = density

    def set_steps_left(self, slot, n):
        self.members[slot]["left"] = n

    def step(self, n):
        self.step_calls.append(n)
        self.log.append(("step", n))
        for m in self.members.values():
            k = n if m["left"] < 0 else min(n, m["left"])
            m["t"] += k
            if m["left"] >= 0:
                m["left"] -= k

    def synchronize(self):
        pass

    def coarse_grain(self, slot, block):
        m = self.members[slot]
        assert m["left"] == 0
        cells = (m["w"] // block) * (m["h"] // block)
        self._stage(cells * 48)
        counts = np.full((m["h"] // block, m["w"] // block, 9), m["t"], np.int32)
        z = np.zeros((m["h"] // block, m["w"] // block), np.float32)
        return counts, z, z, z

    def coarse_grain_begin(self, slot, block, after_event=None):
        self.log.append(("read", self.members[slot]["seed"]))
        return self.coarse_grain(slot, block)

    @staticmethod
    def coarse_grain_finish(handle):
        return handle

    def get_state(self, slot):
        m = self.members[slot]
        self._stage(m["w"] * m["h"])
        return np.full((m["h"], m["w"]), m["seed"] & 0xFF, np.uint8)

    def remove(self, slot, wait=True):
        m = self.members.pop(slot)
        self.used -= m["bytes"]
        self.log.append(("remove", m["seed"]))

    def close(self):
        pass


def make_requests(n, seed=0, sides=(64, 128, 256), max_steps=50):
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(n):
        W, H = int(rng.choice(sides)), int(rng.choice(sides))
        reqs.append(Request(W, H, int(rng.integers(0, max_steps)), seed=i, density=0.2,
                            obstacles=(lambda W=W, H=H: np.zeros((H, W), np.uint8)) if i % 2 else None,
                            arrival=float(rng.integers(0, 20)), name=f"r{i}", keep_state=(i % 3 == 0)))
    return reqs


@pytest.mark.parametrize("pipeline", [True, False])
def test_every_request_runs_exactly_its_steps(pipeline):
    reqs = make_requests(40)
    fake = FakeBatch(64 << 20)
    with Server(64 << 20, quantum_max=16, quantum_min=4, batch=fake, pipeline=pipeline) as srv:
        done = srv.serve(reqs, realtime=False)
    assert sorted(c.request.name for c in done) == sorted(r.name for r in reqs)
    for c in done:
        assert int(c.counts[0, 0, 0]) == c.request.steps            # the lattice's own step count
        assert c.finished >= c.admitted >= c.arrival
        if c.request.keep_state:
            assert c.state is not None and c.state[0, 0] == c.request.seed & 0xFF
    assert all(4 <= q <= 16 for q in fake.step_calls)
    assert not fake.members and fake.used == 0


@pytest.mark.parametrize("pipeline", [True, False])
def test_admission_is_fifo_and_within_budget(pipeline):
    reqs = [Request(256, 256, 30 + i, seed=i, arrival=0.0, name=f"r{i}") for i in range(12)]
    per = FakeBatch.lattice_bytes(256, 256)
    budget = 3 * per + Server.staging_bytes(reqs[0]) + (64 << 10)
    fake = FakeBatch(budget)
    with Server(budget, quantum_max=8, quantum_min=8, batch=fake, pipeline=pipeline) as srv:
        done = srv.serve(reqs, realtime=False)
        assert srv.stats.admissions_deferred > 0
        assert srv.stats.peak_resident <= 3
        assert srv.stats.peak_resident_bytes <= budget
    adds = [s for op, s in fake.log if op == "add"]
    assert adds == sorted(adds)                                     # first come, first admitted
    assert fake.staging_peak <= budget
    assert len(done) == 12


def test_quantum_follows_the_shortest_remaining_budget():
    reqs = [Request(64, 64, 5, seed=1, arrival=0.0), Request(64, 64, 100, seed=2, arrival=0.0)]
    fake = FakeBatch(1 << 24)
    with Server(1 << 24, quantum_max=64, quantum_min=2, batch=fake) as srv:
        done = srv.serve(reqs, realtime=False)
    assert fake.step_calls[0] == 5                    # the short request ends on a tick boundary
    assert [c.request.seed for c in sorted(done, key=lambda c: c.finished)] == [1, 2]


def test_rejects_requests_that_never_fit():
    fake = FakeBatch(1 << 20)
    with Server(1 << 20, batch=fake) as srv:
        with pytest.raises(ValueError):
            srv.submit(Request(4096, 4096, 10))
        with pytest.raises(ValueError):
            srv.submit(Request(48, 64, 10))
        with pytest.raises(ValueError):
            srv.submit(Request(96, 64, 10, cg_block=64))


def test_summary_percentiles():
    reqs = make_requests(10, seed=3)
    fake = FakeBatch(64 << 20)
    with Server(64 << 20, batch=fake) as srv:
        done = srv.serve(reqs, realtime=False)
    s = summarize(done)
    lat = sorted(c.latency for c in done)
    assert s["completed"] == 10
    assert s["p50_ms"] == pytest.approx(np.percentile(lat, 50) * 1e3)
    assert s["p99_ms"] <= s["max_ms"] + 1e-9


def test_pipelined_ticks_keep_one_quantum_queued():
    """With pipelining a tick queues the next quantum before the previous
    one's lattices are read back: a lattice finishing in quantum k is read
    back in tick k + 1, after quantum k + 1 was issued."""
    reqs = [Request(64, 64, 8, seed=1, arrival=0.0), Request(64, 64, 40, seed=2, arrival=0.0)]
    fake = FakeBatch(1 << 24)
    with Server(1 << 24, quantum_max=8, quantum_min=8, batch=fake, pipeline=True) as srv:
        done = srv.serve(reqs, realtime=False)
    assert len(done) == 2
    steps = [i for i, e in enumerate(fake.log) if e[0] == "step"]
    read1 = fake.log.index(("read", 1))
    assert steps[0] < steps[1] < read1          # quantum 2 was queued before request 1 was read back
    assert ("remove", 1) in fake.log[read1:]
    assert [c.request.seed for c in sorted(done, key=lambda c: c.finished)] == [1, 2]


def test_server_sets_the_batch_temporal_block():
    """Blocking stays off unless asked for: quanta are too short for a tuning
    trial over the blocked passes."""
    b = FakeBatch(1 << 20)
    Server(1 << 20, batch=b)
    assert b.temporal_block == 1
    b4 = FakeBatch(1 << 20)
    Server(1 << 20, batch=b4, temporal_block=4)
    assert b4.temporal_block == 4
