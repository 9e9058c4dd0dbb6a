"""The C-ABI library builds, loads and exports every function of include/fhp.h.

No compute call is made (these run without a GPU)."""
import ctypes

import pytest

from paper_1208_2428_gb300 import build as cuda_build
from paper_1208_2428_gb300 import fhp


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return fhp.load()


def test_header_declares_the_boundary():
    names = fhp.exported_names()
    for required in ("fhp_create", "fhp_load_obstacles", "fhp_step", "fhp_coarse_grain", "fhp_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in fhp.exported_names() if not hasattr(lib, n)]
    assert not missing, missing


def test_required_bytes_and_validation_without_gpu(lib):
    # pure host arithmetic: no CUDA call behind these
    assert lib.fhp_required_bytes(31, 4) == 0
    assert lib.fhp_required_bytes(64, 3) == 0
    assert lib.fhp_required_bytes(32, 0) == 0
    n = lib.fhp_required_bytes(16384, 4096)
    planes = 15 * 16384 * 4096 // 8
    assert planes <= n <= planes + 16384 * 4096 + 4 * 4096 + 4096
    # ragged rows are padded to whole 16-byte quads
    assert lib.fhp_required_bytes(96, 2) >= 15 * 2 * 16 + 96 * 2
    # the staging area also holds the two-ghost-row exchange (144 bytes per row
    # quad for each of up to min(H/4, 256) strips) where that exceeds W*H
    for W, H in ((4096, 1024), (512, 608), (4128, 640), (16384, 4096)):
        Pq = 4 * ((W // 32 + 3) // 4)
        staging = max(W * H, 144 * min(H // 4, 256) * Pq)
        n = lib.fhp_required_bytes(W, H)
        assert 15 * H * Pq * 4 + staging <= n <= 15 * H * Pq * 4 + staging + 4 * H + 4096, (W, H)
    out = ctypes.c_void_p(123)
    rc = lib.fhp_create(ctypes.byref(out), None)
    assert rc == fhp.FHP_EINVAL and out.value is None
    assert b"params" in lib.fhp_last_error(None)
    p = fhp._Params(100, 4, 0, 0.0, None, None, 0)
    assert lib.fhp_create(ctypes.byref(out), ctypes.byref(p)) == fhp.FHP_EINVAL
    p = fhp._Params(64, 4, 0, 1.5, None, None, 0)
    assert lib.fhp_create(ctypes.byref(out), ctypes.byref(p)) == fhp.FHP_EINVAL
    assert lib.fhp_step(None, 1) == fhp.FHP_EINVAL
    lib.fhp_destroy(None)


def test_debug_build_exports_every_declared_symbol():
    path = cuda_build.build(debug=True)
    dbg = ctypes.CDLL(path)
    missing = [n for n in fhp.exported_names() if not hasattr(dbg, n)]
    assert not missing, missing
    dbg.fhp_debug_build.restype = ctypes.c_int
    assert dbg.fhp_debug_build() == 1
    # the debug layout adds six 256-byte canary blocks to a lattice's bytes
    dbg.fhp_required_bytes.restype = ctypes.c_size_t
    dbg.fhp_required_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32]
    rel = fhp.load()
    assert dbg.fhp_required_bytes(256, 64) == rel.fhp_required_bytes(256, 64) + 6 * 256


def test_batch_block_rows_without_gpu(lib):
    """Blocked tiles inside batches (host arithmetic only): R_out + 2k staged
    rows of the member's row pitch fill at most one 3,072-word plane, R_out is
    even (or the whole lattice), at most H, and at least 4k rows -- else the
    member takes no blocked passes."""
    for W in range(32, 16385, 32):
        Pq = 4 * ((W // 32 + 3) // 4)
        for H in (2, 4, 8, 20, 64, 130, 1030, 2048):
            for k in (2, 4):
                R = lib.fhp_batch_block_rows(W, H, k)
                if R == 0:
                    full = (3072 // Pq - 2 * k) & ~1
                    assert min(full, H) < 4 * k and min(full, H) != H or full <= 0, (W, H, k)
                    continue
                assert (min(R, H) + 2 * k) * Pq <= 3072, (W, H, k, R)
                assert R <= H and (R % 2 == 0 or R == H) and (R >= 4 * k or R == H), (W, H, k, R)
                # the largest such R: two more rows would not fit (or exceed H)
                assert R == H or (R + 2 + 2 * k) * Pq > 3072, (W, H, k, R)
    assert lib.fhp_batch_block_rows(2048, 2048, 4) == 40
    assert lib.fhp_batch_block_rows(16384, 4096, 2) == 0
    assert lib.fhp_batch_block_rows(2048, 512, 3) == 0
    assert lib.fhp_batch_block_rows(100, 64, 2) == 0
