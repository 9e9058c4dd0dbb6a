"""fhp_run_static, the entry point that allocates no device memory.

It serves callers that cannot allocate device memory (plugins whose host
application owns all GPU memory, services with a fixed memory cap, loops that
must not allocate).  Its output must equal what the ordinary lattice calls
(fhp_create, fhp_set_state, fhp_set_time, fhp_step, fhp_get_state) give --
bit-exact, the tolerance of every lattice-state test here -- on consecutive
calls that reuse the same static scratch array.  This file is collected last
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


def run_static(lib, s0, seed, t0, n, p):
    import torch
    H, W = s0.shape
    din = torch.from_numpy(s0).cuda()
    dout = torch.full_like(din, 0x5A)
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


def test_run_static_matches_lattice_calls(lib):
    W1, H1 = 4160, 64
    a = workloads.bernoulli_lattice(W1, H1, 0.3, 31, workloads.cylinder_mask(W1, H1))
    rng = np.random.Generator(np.random.PCG64(32))
    W2, H2 = 224, 30
    b = workloads.bernoulli_lattice(W2, H2, 0.4, 33, workloads.random_points(W2, H2, 0.05, rng))
    calls = [(a, 0xABCDEF0123, 7, 21, 0.02), (b, 99, 0, 13, 0.0), (a, 0xABCDEF0123, 7, 21, 0.02)]
    outs = []
    for s0, seed, t0, n, p in calls:   # consecutive calls share the static scratch array
        got = run_static(lib, s0, seed, t0, n, p)
        want = run_lattice(s0, seed, t0, n, p)
        assert np.array_equal(got, want)
        outs.append(got)
    assert np.array_equal(outs[0], outs[2])


def test_run_static_rejects_oversized_lattice(lib):
    import torch
    from paper_1208_2428_gb300 import fhp
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    rc = lib.fhp_run_static(ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), 4096, 4096,
                            1, 0, 1, 0.0, None)
    assert rc == fhp.FHP_EINVAL
    assert b"scratch" in lib.fhp_last_error(None)
