"""Row strips on the device: strips of one lattice (row offsets, ghost-row
exchange through device buffers) equal the undivided lattice and the oracle,
bit for bit, for every step kernel."""
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


@pytest.mark.parametrize("parts,halo,kernel,k", [(2, 2, 0, 1), (3, 4, 1, 1), (4, 2, 2, 1), (2, 8, 3, 1),
                                                 (3, 4, 0, 2), (2, 8, 0, 4), (1, 2, 0, 1)])
def test_device_strips_equal_the_whole_lattice(pkg, oracle_mod, parts, halo, kernel, k):
    from paper_1208_2428_gb300.strips import DeviceStrip, LocalExchange, StripDomain, StripPlan
    W, H, seed, p, steps = 512, 96, 1234, 2e-3, 23
    s0 = workloads.Lattice("s", W, H, 0.3, seed, p, 0, obstacle="cylinder").initial_state()
    plan = StripPlan(W, H, parts, halo)
    strips = [DeviceStrip(plan, r, seed, p) for r in range(parts)]
    try:
        for s in strips:
            s.set_from_global(s0)
            s.set_time(3)
            s.lattice.set_step_kernel(kernel)
            s.lattice.set_temporal_block(k)
        StripDomain(plan, strips, LocalExchange()).step(steps)
        got = np.concatenate([s.owned_state() for s in strips])
    finally:
        for s in strips:
            s.close()
    want, _ = oracle_mod.run(s0, seed, 3, steps, p)
    assert np.array_equal(got, want)
    with pkg.Lattice(W, H, seed=seed, forcing_p=p) as whole:
        whole.set_state(s0)
        whole.set_time(3)
        whole.step(steps)
        assert np.array_equal(whole.get_state(), got)


def test_rows_roundtrip_and_bounds(pkg):
    import torch
    with pkg.Lattice(160, 8, seed=1) as lat:
        s = workloads.bernoulli_lattice(160, 8, 0.5, 2)
        lat.set_state(s)
        rows = lat.get_rows_tensor(2, 3)
        assert rows.shape == (7, 3, lat.row_pitch_words) and lat.row_pitch_words == 8
        lat.set_rows_tensor(5, rows)
        got = lat.get_state()
        assert np.array_equal(got[5:8] & 0x7F, s[2:5] & 0x7F)
        assert np.array_equal(got[:5], s[:5])
        with pytest.raises(pkg.FhpError):
            lat.get_rows_tensor(6, 3)
        with pytest.raises(pkg.FhpError):
            lat.set_row_offset(3)
        del torch
