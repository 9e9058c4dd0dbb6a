"""Run in a subprocess with FHP_DEBUG=1 by test_gpu_debug.py: tiny lattices
and batches through every kernel of the debug build (device-side index
checks, canary blocks), each compared bit for bit with the oracle, with no
failed check and every canary intact.  Prints one JSON line."""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402
from paper_1208_2428_gb300 import Batch, Lattice, fhp  # noqa: E402

# (step kernel, temporal block, temporal-block kernel): direct, ring,
# multi-step, resident (one-row and two-row exchange), 2-D tiles, wavefronts
CONFIGS = [(1, 1, 0), (2, 1, 0), (3, 1, 0), (4, 1, 0), (4, 2, 0), (0, 2, 2), (0, 4, 2), (0, 8, 2), (0, 2, 1),
           (0, 3, 1), (0, 4, 1)]
SHAPES = [(32, 2), (32, 6), (64, 4), (96, 8), (128, 2), (160, 6), (256, 8), (512, 18), (640, 20), (4128, 4)]


def main() -> int:
    assert os.environ.get("FHP_DEBUG") == "1"
    lib = fhp.load()
    assert lib.fhp_debug_build() == 1, "FHP_DEBUG=1 must load the debug build"
    word = fhp.ctypes.c_uint32(0)
    assert lib.fhp_debug_selftest(fhp.ctypes.byref(word)) == 0
    selftest = {"bounds_bit": bool(word.value & 2), "site": (word.value >> 8) & 0xFF}
    cases = 0
    for W, H in SHAPES:
        for variant in ("periodic", "points_forcing"):
            seed = 5 + W + H
            rng = np.random.Generator(np.random.PCG64(seed))
            solid = None if variant == "periodic" else workloads.random_points(W, H, 0.08, rng)
            p = 0.0 if variant == "periodic" else 0.3
            s0 = workloads.bernoulli_lattice(W, H, 0.4, seed, solid)
            steps = 9
            want, _ = oracle.run(s0, seed, 2, steps, p)
            for kernel, k, bk in CONFIGS:
                with Lattice(W, H, seed=seed, forcing_p=p, step_kernel=kernel) as lat:
                    lat.set_temporal_block(k)
                    lat.set_temporal_block_kernel(bk)
                    lat.set_state(s0)
                    lat.set_time(2)
                    lat.step(steps)
                    lat.synchronize()          # FHP_EDEBUG if an index check failed
                    got = lat.get_state()
                    checked, corrupted = lat.debug_canaries()
                if not np.array_equal(got, want):
                    print(json.dumps({"ok": False, "case": [W, H, variant, kernel, k, bk], "why": "state"}))
                    return 1
                if checked != 6 or corrupted:
                    print(json.dumps({"ok": False, "case": [W, H, variant, kernel, k, bk],
                                      "why": f"canaries {checked} {corrupted}"}))
                    return 1
                cases += 1
    # coarse-graining
    W, H = 256, 64
    s0 = workloads.bernoulli_lattice(W, H, 0.3, 3, workloads.channel_walls(W, H))
    with Lattice(W, H, seed=3) as lat:
        lat.set_state(s0)
        counts, rho, ux, uy = lat.coarse_grain(32)
        assert lat.debug_canaries() == (6, 0)
    c_ref, _, _, _ = oracle.coarse_grain(s0, 32)
    assert np.array_equal(counts, c_ref)
    # batches: both kernels, two tile sizes, and blocked passes of 2 and 4 steps
    jobs = [(96, 6, 0.0), (160, 10, 0.2), (512, 4, 0.05), (4128, 8, 0.0), (64, 2, 0.3), (12288, 8, 0.1)]
    for kind, quads, block in ((1, 64, 1), (1, 256, 1), (2, 64, 1), (2, 256, 1), (1, 256, 2), (1, 256, 4),
                               (2, 64, 4)):
        arena = sum(Batch.lattice_bytes(w, h) for w, h, _ in jobs) + (8 << 20)
        with Batch(arena) as b:
            b.set_step_kernel(kind)
            b.set_tile_quads(quads)
            b.set_temporal_block(block)
            slots, states = [], []
            for i, (w, h, pp) in enumerate(jobs):
                rng = np.random.Generator(np.random.PCG64(70 + i))
                s = workloads.bernoulli_lattice(w, h, 0.35, 70 + i, workloads.random_points(w, h, 0.05, rng))
                slot = b.add(w, h, 70 + i, pp)
                b.set_state(slot, s)
                slots.append(slot)
                states.append(s)
            b.step(7)
            b.synchronize()
            for i, (w, h, pp) in enumerate(jobs):
                want, _ = oracle.run(states[i], 70 + i, 0, 7, pp)
                if not np.array_equal(b.get_state(slots[i]), want):
                    print(json.dumps({"ok": False, "case": ["batch", kind, quads, block, w, h], "why": "state"}))
                    return 1
            checked, corrupted = b.debug_canaries()
            if checked != len(jobs) or corrupted:
                print(json.dumps({"ok": False, "case": ["batch", kind, quads, block], "why": "canaries"}))
                return 1
            cases += 1
    print(json.dumps({"ok": True, "cases": cases, "selftest": selftest}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
