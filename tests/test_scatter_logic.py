"""The bit-sliced scattering expressions of the CUDA path, compiled for the
host, against the oracle's 256-entry tables: every node byte x both
chiralities (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def host_scatter(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("hs") / "libhost_scatter.so"
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-std=c++17", "-o", str(out),
                    os.path.join(HERE, "csrc", "host_scatter.cu")], check=True)
    lib = ctypes.CDLL(str(out))
    lib.host_scatter_words.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_void_p]
    lib.host_scatter_words.restype = None
    lib.host_scatter_saturated_words.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p]
    lib.host_scatter_saturated_words.restype = None
    return lib


@pytest.mark.parametrize("rules,mask", [(2, 0xFFFFFFFF), (1, 0), (3, None)])
def test_bitsliced_scatter_equals_table(host_scatter, oracle_mod, rules, mask):
    tables = [oracle_mod.table(0, rules=rules), oracle_mod.table(1, rules=rules)]
    states = np.arange(256, dtype=np.uint32)
    # 8 words x 32 nodes cover all 256 bytes; a chirality pattern per run
    for chi_pattern in (0x00000000, 0xFFFFFFFF, 0xA5A5A5A5, 0x0F0F33CC):
        for wi in range(8):
            nodes = states[32 * wi:32 * wi + 32]
            planes = np.array([int(((nodes >> k) & 1) @ (1 << np.arange(32, dtype=np.uint64)))
                               for k in range(7)], dtype=np.uint32)
            solid = np.uint32(int(((nodes >> 7) & 1) @ (1 << np.arange(32, dtype=np.uint64))))
            out = np.zeros(7, dtype=np.uint32)
            if rules == 3:
                host_scatter.host_scatter_saturated_words(planes.ctypes.data, int(solid), chi_pattern, out.ctypes.data)
            else:
                host_scatter.host_scatter_words(planes.ctypes.data, int(solid), chi_pattern, mask, out.ctypes.data)
            for j in range(32):
                b = int(nodes[j])
                chi = (chi_pattern >> j) & 1
                got = sum(((int(out[k]) >> j) & 1) << k for k in range(7)) | (b & 0x80)
                assert got == int(tables[chi][b]), (b, chi)
