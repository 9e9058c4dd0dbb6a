"""CPU oracle for the FHP lattice-gas step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library
in ``paper_1208_2428_gb300`` and its binding) never loads it; it shares no
code with it.

The arithmetic lives in ``fhp_oracle.c`` (plain C, byte per node, a
256-entry look-up table per chirality value, neighbour-pull motion, per-word
forcing).  This module compiles it with gcc and wraps it with ctypes.

Paper: Szkoda, Koza & Tykierko, arXiv:1208.2428, Section 2 (the model).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fhp_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fvisibility=hidden", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_rng_word.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_uint32]
        lib.oracle_rng_word.restype = ctypes.c_uint32
        lib.oracle_build_table.argtypes = [ctypes.c_int, u8p]
        lib.oracle_build_table.restype = None
        lib.oracle_build_table_rules.argtypes = [ctypes.c_int, ctypes.c_int, u8p]
        lib.oracle_build_table_rules.restype = None
        lib.oracle_run_rules.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_int]
        lib.oracle_run_rules.restype = ctypes.c_int64
        lib.oracle_neighbour.argtypes = [ctypes.c_int] * 5 + [ip, ip]
        lib.oracle_neighbour.restype = None
        lib.oracle_forcing_thresholds.argtypes = [ctypes.c_double, u64p]
        lib.oracle_forcing_thresholds.restype = None
        lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_int64, ctypes.c_double]
        lib.oracle_run.restype = ctypes.c_int64
        lib.oracle_run_rows.argtypes = [ctypes.c_int, ctypes.c_int, u8p, u8p, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_int64, ctypes.c_double, ctypes.c_int64, ctypes.c_int]
        lib.oracle_run_rows.restype = ctypes.c_int64
        lib.oracle_coarse_grain.argtypes = [ctypes.c_int, ctypes.c_int, u8p, ctypes.c_int,
                                            i32p, f64p, f64p, f64p]
        lib.oracle_coarse_grain.restype = None
        lib.oracle_init_random.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                                           u8p, u8p]
        lib.oracle_init_random.restype = None
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and a 2-word key (SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                                 _ptr(out, ctypes.c_uint32))
    return out


def rng_word(seed: int, t: int, y: int, w: int, stream: int) -> int:
    """Random word of (row y, word w, step t, stream) for a lattice seed."""
    return int(_load().oracle_rng_word(seed, t, y, w, stream))


def table(chirality: int, rules: int = 2) -> np.ndarray:
    """The 256-entry scattering table for chirality 0 or 1 (uint8[256]) of
    rule set 2 (FHP-II), 1 (FHP-I) or 3 (FHP-III, collision-saturated)."""
    out = np.zeros(256, dtype=np.uint8)
    if rules == 2:
        _load().oracle_build_table(int(chirality), _ptr(out, ctypes.c_uint8))
    else:
        _load().oracle_build_table_rules(int(rules), int(chirality), _ptr(out, ctypes.c_uint8))
    return out


def neighbour(W: int, H: int, x: int, y: int, i: int):
    nx, ny = ctypes.c_int(), ctypes.c_int()
    _load().oracle_neighbour(W, H, x, y, i, ctypes.byref(nx), ctypes.byref(ny))
    return nx.value, ny.value


def forcing_thresholds(p: float) -> np.ndarray:
    """Q_0..Q_32 of the forcing sampler, uint64[33] in units of 2^-32."""
    q = np.zeros(33, dtype=np.uint64)
    _load().oracle_forcing_thresholds(float(p), _ptr(q, ctypes.c_uint64))
    return q


def run(state: np.ndarray, seed: int, t0: int, n: int, p: float = 0.0, rules: int = 2) -> tuple[np.ndarray, int]:
    """Advance an H x W uint8 lattice by n steps from step t0 (rule set 2 =
    FHP-II, 1 = FHP-I, 3 = FHP-III).

    Returns (new state, number of forcing events)."""
    s = np.array(state, dtype=np.uint8, order="C", copy=True)
    if s.ndim != 2:
        raise ValueError("state must be H x W")
    H, W = s.shape
    if W % 32 or W < 32 or H % 2 or H < 2:
        raise ValueError("W must be a positive multiple of 32 and H even")
    scratch = np.empty_like(s)
    if rules == 2:
        ev = _load().oracle_run(W, H, _ptr(s, ctypes.c_uint8), _ptr(scratch, ctypes.c_uint8),
                                int(seed), int(t0), int(n), float(p))
    else:
        ev = _load().oracle_run_rules(W, H, _ptr(s, ctypes.c_uint8), _ptr(scratch, ctypes.c_uint8),
                                      int(seed), int(t0), int(n), float(p), int(rules))
        if ev < 0:
            raise ValueError("rules must be 1, 2 or 3")
    return s, int(ev)


def run_rows(rows: np.ndarray, seed: int, t0: int, n: int, p: float, row_base: int, global_height: int):
    """Advance an h x W array whose row y is row (row_base + y) mod
    global_height of a larger lattice, n steps, periodic in its own rows
    (a strip with ghost rows: rows within n of its edges become invalid)."""
    s = np.array(rows, dtype=np.uint8, order="C", copy=True)
    H, W = s.shape
    if W % 32 or W < 32 or H % 2 or H < 2 or row_base % 2:
        raise ValueError("W must be a positive multiple of 32, H and row_base even")
    scratch = np.empty_like(s)
    ev = _load().oracle_run_rows(W, H, _ptr(s, ctypes.c_uint8), _ptr(scratch, ctypes.c_uint8), int(seed), int(t0),
                                 int(n), float(p), int(row_base), int(global_height))
    if ev < 0:
        raise ValueError("invalid strip")
    return s, int(ev)


def coarse_grain(state: np.ndarray, B: int):
    """Block counts int32[H/B, W/B, 9] and float64 rho, ux, uy [H/B, W/B]."""
    s = np.ascontiguousarray(state, dtype=np.uint8)
    H, W = s.shape
    if H % B or W % B:
        raise ValueError("B must divide W and H")
    counts = np.zeros((H // B, W // B, 9), dtype=np.int32)
    rho = np.zeros((H // B, W // B), dtype=np.float64)
    ux = np.zeros_like(rho)
    uy = np.zeros_like(rho)
    _load().oracle_coarse_grain(W, H, _ptr(s, ctypes.c_uint8), int(B),
                                _ptr(counts, ctypes.c_int32), _ptr(rho, ctypes.c_double),
                                _ptr(ux, ctypes.c_double), _ptr(uy, ctypes.c_double))
    return counts, rho, ux, uy


def init_random(W: int, H: int, seed: int, density: float, solid=None) -> np.ndarray:
    """Generated initial state (each of bits 0..6 of a fluid node set with
    probability round(density * 2^16) / 2^16 from counter-based draws)."""
    out = np.empty((H, W), dtype=np.uint8)
    mask = None
    if solid is not None:
        mask = np.ascontiguousarray(solid, dtype=np.uint8)
    _load().oracle_init_random(int(W), int(H), int(seed), float(density),
                               _ptr(mask, ctypes.c_uint8) if mask is not None else None,
                               _ptr(out, ctypes.c_uint8))
    return out


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())
