"""Serving by continuous batching on the device: every request's result in the
mix equals the same request served alone (a single lattice through the C
ABI) and the CPU oracle, bit for bit; admission respects the memory budget."""
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


def mixed_requests(serving, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for i in range(n):
        W = int(rng.choice(np.arange(64, 449, 64)))
        H = int(rng.choice(np.arange(64, 321, 64)))
        cyl = i % 2 == 0
        shapes = cyl and i % 4 == 0            # half of the cylinders generated on the device
        reqs.append(serving.Request(
            W, H, int(rng.integers(0, 70)), seed=880_000 + 7 * i, density=float(rng.uniform(0.1, 0.4)),
            forcing_p=5e-4 if cyl else 0.0,
            obstacles=(lambda W=W, H=H: workloads.cylinder_mask(W, H)) if cyl and not shapes else None,
            obstacle_shapes=workloads.cylinder_shapes(W, H) if shapes else None,
            cg_block=32, arrival=float(rng.integers(0, 12)), name=f"q{i}", keep_state=True))
    return reqs


def request_mask(req):
    if req.obstacle_shapes:
        return workloads.cylinder_mask(req.width, req.height)   # the shapes used here are the cylinder's
    return req.obstacles() if callable(req.obstacles) else req.obstacles


def alone(pkg, req):
    with pkg.Lattice(req.width, req.height, seed=req.seed, forcing_p=req.forcing_p) as lat:
        mask = request_mask(req)
        if mask is not None:
            lat.load_obstacles(mask)
        lat.init_random(req.density)
        lat.step(req.steps)
        return lat.get_state(), lat.coarse_grain(req.cg_block)


def oracle_result(oracle_mod, req):
    mask = request_mask(req)
    s0 = oracle_mod.init_random(req.width, req.height, req.seed, req.density, mask)
    out, _ = oracle_mod.run(s0, req.seed, 0, req.steps, req.forcing_p)
    return out


def check_against_alone_and_oracle(pkg, oracle_mod, done, reqs):
    assert sorted(c.request.name for c in done) == sorted(r.name for r in reqs)
    for c in done:
        req = c.request
        want_state, (wc, wr, wx, wy) = alone(pkg, req)
        assert np.array_equal(c.state, want_state), req.name
        assert np.array_equal(c.counts, wc), req.name
        assert np.array_equal(c.rho, wr) and np.array_equal(c.ux, wx) and np.array_equal(c.uy, wy), req.name
        assert np.array_equal(c.state, oracle_result(oracle_mod, req)), req.name
        ref_counts, _, _, _ = oracle_mod.coarse_grain(c.state, req.cg_block)
        assert np.array_equal(c.counts, ref_counts), req.name


def test_results_in_the_mix_equal_results_alone(pkg, oracle_mod):
    from paper_1208_2428_gb300 import serving
    reqs = mixed_requests(serving, 18, 1)
    with serving.Server(256 << 20, quantum_max=8, quantum_min=2, graph_steps=4) as srv:
        done = srv.serve(reqs, realtime=False)
        assert srv.stats.peak_resident >= 4            # requests really overlapped on the device
    check_against_alone_and_oracle(pkg, oracle_mod, done, reqs)


def test_admission_waits_for_memory(pkg, oracle_mod):
    from paper_1208_2428_gb300 import serving
    reqs = [serving.Request(512, 256, 20 + 3 * i, seed=990 + i, density=0.3, arrival=0.0, name=f"m{i}",
                            keep_state=True, obstacles=(lambda: workloads.cylinder_mask(512, 256)) if i % 2 else None,
                            forcing_p=1e-3 if i % 3 == 0 else 0.0)
            for i in range(8)]
    per = pkg.Batch.lattice_bytes(512, 256)
    # two lattices, the read-back reserve, and room for the descriptor tables
    budget = 2 * per + serving.Server.staging_bytes(reqs[0]) + (32 << 10)
    with serving.Server(budget, quantum_max=8, quantum_min=8, graph_steps=4) as srv:
        done = srv.serve(reqs, realtime=False)
        assert srv.stats.admissions_deferred > 0
        assert srv.stats.peak_resident == 2
    check_against_alone_and_oracle(pkg, oracle_mod, done, reqs)


def test_realtime_trace_and_sequential_comparison(pkg, oracle_mod):
    from paper_1208_2428_gb300 import serving
    reqs = mixed_requests(serving, 10, 2)
    for i, r in enumerate(reqs):
        r.arrival = 0.002 * i
    with serving.Server(256 << 20, quantum_max=16, quantum_min=4) as srv:
        done = srv.serve(reqs, realtime=True)
    seq = serving.serve_sequential(reqs, realtime=True)
    s1, s2 = serving.summarize(done), serving.summarize(seq)
    assert s1["completed"] == s2["completed"] == 10
    assert s1["p99_ms"] >= s1["p50_ms"] > 0
    by_name = {c.request.name: c for c in seq}
    for c in done:
        assert np.array_equal(c.state, by_name[c.request.name].state), c.request.name
        assert np.array_equal(c.counts, by_name[c.request.name].counts)
