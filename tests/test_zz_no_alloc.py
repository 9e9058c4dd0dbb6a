"""fhp_run_static, the entry point that allocates no device memory.

It serves callers that cannot allocate device memory (plugins whose host
application owns all GPU memory, services with a fixed memory cap, loops that
must not allocate).  Its output must equal the CPU oracle's run and what the ordinary lattice
calls (fhp_create, fhp_set_state, fhp_set_time, fhp_step, fhp_get_state) give
-- bit-exact, the tolerance of every lattice-state test here -- on
consecutive calls that reuse the same static scratch array: with and without
obstacles, in place (input and output the same buffer) and at the largest
size the header documents.  This file is collected last
so that a run that stops at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_2428_gb300 import build as cuda_build
    from paper_1208_2428_gb300 import fhp
    cuda_build.build()
    lib = fhp.load()
    lib.fhp_run_static.restype = ctypes.c_int
    lib.fhp_run_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_void_p]
    return lib


def run_static(lib, s0, seed, t0, n, p, in_place=False):
    import torch
    H, W = s0.shape
    din = torch.from_numpy(s0).cuda()
    dout = din if in_place else torch.full_like(din, 0x5A)
    stream = torch.cuda.current_stream()
    rc = lib.fhp_run_static(ctypes.c_void_p(din.data_ptr()), ctypes.c_void_p(dout.data_ptr()), W, H,
                            seed, t0, n, p, ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.fhp_last_error(None)
    torch.cuda.synchronize()
    return dout.cpu().numpy()


def run_lattice(s0, seed, t0, n, p):
    from paper_1208_2428_gb300 import Lattice
    H, W = s0.shape
    with Lattice(W, H, seed=seed, forcing_p=p) as lat:
        lat.set_state(s0)
        lat.set_time(t0)
        lat.step(n)
        return lat.get_state()


def run_oracle(s0, seed, t0, n, p):
    import oracle
    return oracle.run(s0, seed, t0, n, p)[0]


def test_run_static_matches_lattice_calls_and_oracle(lib):
    W1, H1 = 4160, 64
    a = workloads.bernoulli_lattice(W1, H1, 0.3, 31, workloads.cylinder_mask(W1, H1))
    rng = np.random.Generator(np.random.PCG64(32))
    W2, H2 = 224, 30
    b = workloads.bernoulli_lattice(W2, H2, 0.4, 33, workloads.random_points(W2, H2, 0.05, rng))
    W3, H3 = 640, 48
    c = workloads.bernoulli_lattice(W3, H3, 0.25, 34)     # no obstacles: the solid plane is all zero
    calls = [(a, 0xABCDEF0123, 7, 21, 0.02, False), (b, 99, 0, 13, 0.0, False), (c, 5, 3, 17, 0.01, False),
             (b, 99, 0, 13, 0.0, True), (a, 0xABCDEF0123, 7, 21, 0.02, False)]
    outs = []
    for s0, seed, t0, n, p, in_place in calls:   # consecutive calls share the static scratch array
        got = run_static(lib, s0, seed, t0, n, p, in_place=in_place)
        assert np.array_equal(got, run_oracle(s0, seed, t0, n, p))
        assert np.array_equal(got, run_lattice(s0, seed, t0, n, p))
        outs.append(got)
    assert np.array_equal(outs[0], outs[4])
    assert np.array_equal(outs[1], outs[3])     # in place == separate buffers


def test_run_static_largest_documented_lattice(lib):
    W, H = 4096, 2048                            # the size limit stated in the header
    s0 = workloads.bernoulli_lattice(W, H, 0.2, 35, workloads.channel_walls(W, H))
    got = run_static(lib, s0, 41, 0, 2, 1e-3)
    assert np.array_equal(got, run_oracle(s0, 41, 0, 2, 1e-3))


def test_run_static_rejects_oversized_lattice(lib):
    import torch
    from paper_1208_2428_gb300 import fhp
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = lib.fhp_run_static(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), 4096, 4096,
                            1, 0, 1, 0.0, None)
    assert rc == fhp.FHP_EINVAL
    assert b"scratch" in lib.fhp_last_error(None)
