"""Row strips across processes on the device: each of two ranks (spawned
processes of a gloo group, both on cuda:0) advances a DeviceStrip with the
library's kernels, and the strips trade ghost rows through DistExchange
(rows staged through host memory, as gloo carries host tensors).  The owned
rows of the two ranks, put together, equal the oracle's run of the undivided
lattice bit for bit -- the paper's two-GPU decomposition (Table 1, mGPU) with
the product's stepper and exchange in separate processes.

The strips use step kernels without waits between CTAs (direct and
single-step ring); no kernel of one rank waits on the other rank's work:
the ranks meet only on the host, between steps."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

W, H, SEED, P, STEPS = 1024, 72, 4321, 3e-3, 19


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _initial():
    return workloads.Lattice("dist", W, H, 0.3, SEED, P, 0, obstacle="cylinder").initial_state()


def _rank_main(rank, world, port, out_dir, halo, kernel):
    import torch
    import torch.distributed as dist

    from paper_1208_2428_gb300.strips import DeviceStrip, DistExchange, StripDomain, StripPlan
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    strip = None
    try:
        plan = StripPlan(W, H, world, halo)
        strip = DeviceStrip(plan, rank, SEED, P, device="cuda:0")
        strip.set_from_global(_initial())
        strip.set_time(2)
        strip.lattice.set_step_kernel(kernel)
        ex = DistExchange()
        assert ex.via_host
        dom = StripDomain(plan, [strip], ex)
        dom.step(STEPS)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), strip.owned_state())
        np.save(os.path.join(out_dir, f"kernel{rank}.npy"), np.array([strip.lattice.step_kernel]))
        dist.barrier()
    finally:
        if strip is not None:
            strip.close()
        dist.destroy_process_group()


@pytest.mark.parametrize("halo,kernel", [(2, 1), (4, 2), (8, 1)])
def test_two_processes_equal_the_whole_lattice(oracle_mod, tmp_path, halo, kernel):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2428_gb300 import build as cuda_build
    cuda_build.build()
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), halo, kernel), nprocs=world, join=True)
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)])
    for r in range(world):
        assert int(np.load(tmp_path / f"kernel{r}.npy")[0]) == kernel
    want, _ = oracle_mod.run(_initial(), SEED, 2, STEPS, P)
    assert np.array_equal(got, want)
