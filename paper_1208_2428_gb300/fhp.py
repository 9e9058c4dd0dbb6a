"""ctypes binding of the C ABI in ``include/fhp.h`` (libfhp_gb300.so).

Argument marshalling only: every step of the FHP update runs in the CUDA
library.  PyTorch supplies device memory (the lattice buffers are a torch
allocation handed to ``fhp_create``) and the CUDA stream (torch's current
stream).  If the library is missing this module raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libfhp_gb300.so")
# The debug build (device-side index checks, canary blocks; see fhp.h) is
# loaded instead when the environment sets FHP_DEBUG=1.
DEBUG_LIB_PATH = os.path.join(_PKG, "_lib", "libfhp_gb300_debug.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "fhp.h")

FHP_OK, FHP_EINVAL, FHP_ENOMEM, FHP_ECUDA, FHP_ETIMEOUT, FHP_EBUSY, FHP_EDEBUG = range(7)
_ERRNAMES = {1: "FHP_EINVAL", 2: "FHP_ENOMEM", 3: "FHP_ECUDA", 4: "FHP_ETIMEOUT", 5: "FHP_EBUSY",
             6: "FHP_EDEBUG"}

_lib = None


class FhpError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {message}")
        self.code = code


class _Shape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("a", ctypes.c_int32), ("b", ctypes.c_int32), ("c", ctypes.c_int32)]


SHAPE_DISC = 1   # (x - a)^2 + (y - b)^2 <= c^2
SHAPE_ROWS = 2   # a <= y < b


def _shapes(shapes):
    arr = (_Shape * max(1, len(shapes)))()
    for i, (kind, a, b, c) in enumerate(shapes):
        arr[i] = _Shape(int(kind), int(a), int(b), int(c))
    return arr, len(shapes)


class _Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("forcing_p", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("device_memory", ctypes.c_void_p), ("device_memory_bytes", ctypes.c_size_t)]


def exported_names() -> list[str]:
    """Function names declared in include/fhp.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fhp_[a-z0-9_]+)\s*\(", text)))


def load(path: str | None = None):
    """Load libfhp_gb300.so, or its debug build when FHP_DEBUG=1 is set
    (raises if the library has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or (DEBUG_LIB_PATH if os.environ.get("FHP_DEBUG") == "1" else LIB_PATH)
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    vp, i32, i64, u8p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "fhp_required_bytes": (ctypes.c_size_t, [i32, i32]),
        "fhp_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(_Params)]),
        "fhp_destroy": (None, [vp]),
        "fhp_last_error": (ctypes.c_char_p, [vp]),
        "fhp_set_state": (ctypes.c_int, [vp, u8p]),
        "fhp_get_state": (ctypes.c_int, [vp, u8p]),
        "fhp_set_state_device": (ctypes.c_int, [vp, u8p]),
        "fhp_get_state_device": (ctypes.c_int, [vp, u8p]),
        "fhp_load_obstacles": (ctypes.c_int, [vp, u8p]),
        "fhp_step": (ctypes.c_int, [vp, i64]),
        "fhp_coarse_grain": (ctypes.c_int, [vp, i32, vp, vp, vp, vp]),
        "fhp_coarse_grain_device": (ctypes.c_int, [vp, i32, vp, vp, vp, vp]),
        "fhp_get_time": (i64, [vp]),
        "fhp_set_time": (ctypes.c_int, [vp, i64]),
        "fhp_set_forcing": (ctypes.c_int, [vp, ctypes.c_double]),
        "fhp_set_temporal_block": (ctypes.c_int, [vp, i32]),
        "fhp_set_temporal_block_kernel": (ctypes.c_int, [vp, i32]),
        "fhp_get_temporal_block_kernel": (ctypes.c_int, [vp]),
        "fhp_synchronize": (ctypes.c_int, [vp]),
        "fhp_set_step_kernel": (ctypes.c_int, [vp, i32]),
        "fhp_get_step_kernel": (ctypes.c_int, [vp]),
        "fhp_kernel_launches": (i64, [vp]),
        "fhp_philox4x32_10_device": (ctypes.c_int, [vp, vp, vp, i64, vp]),
        "fhp_init_random": (ctypes.c_int, [vp, ctypes.c_double]),
        "fhp_selftest_wait_limits": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
        "fhp_load_obstacle_shapes": (ctypes.c_int, [vp, ctypes.POINTER(_Shape), i32]),
        "fhp_batch_load_obstacle_shapes": (ctypes.c_int, [vp, i32, ctypes.POINTER(_Shape), i32]),
        "fhp_get_temporal_block": (ctypes.c_int, [vp]),
        "fhp_set_row_offset": (ctypes.c_int, [vp, i32]),
        "fhp_set_rules": (ctypes.c_int, [vp, i32]),
        "fhp_get_rules": (ctypes.c_int, [vp]),
        "fhp_batch_set_rules": (ctypes.c_int, [vp, i32, i32]),
        "fhp_row_pitch_words": (i32, [vp]),
        "fhp_get_rows_device": (ctypes.c_int, [vp, i32, i32, vp]),
        "fhp_set_rows_device": (ctypes.c_int, [vp, i32, i32, vp]),
        "fhp_autotune": (ctypes.c_int, [vp, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "fhp_batch_init_random": (ctypes.c_int, [vp, i32, ctypes.c_double]),
        "fhp_batch_set_step_kernel": (ctypes.c_int, [vp, i32]),
        "fhp_batch_remove_async": (ctypes.c_int, [vp, i32]),
        "fhp_batch_coarse_grain_device": (ctypes.c_int, [vp, i32, i32, vp, vp, vp, vp, vp]),
        "fhp_batch_get_step_kernel": (ctypes.c_int, [vp]),
        "fhp_batch_get_tuned_kernel": (ctypes.c_int, [vp, i32]),
        "fhp_batch_get_tuned_tile_quads": (ctypes.c_int, [vp, i32]),
        "fhp_batch_set_tile_quads": (ctypes.c_int, [vp, i32]),
        "fhp_batch_get_tile_quads": (ctypes.c_int, [vp]),
        "fhp_batch_set_temporal_block": (ctypes.c_int, [vp, i32]),
        "fhp_batch_get_temporal_block": (ctypes.c_int, [vp]),
        "fhp_batch_get_tuned_temporal_block": (ctypes.c_int, [vp, i32]),
        "fhp_batch_block_rows": (ctypes.c_int, [i32, i32, i32]),
        "fhp_batch_tile_count": (i32, [vp]),
        "fhp_batch_load_obstacles": (ctypes.c_int, [vp, i32, u8p]),
        "fhp_batch_lattice_bytes": (ctypes.c_size_t, [i32, i32]),
        "fhp_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_size_t, vp, vp]),
        "fhp_batch_destroy": (None, [vp]),
        "fhp_batch_last_error": (ctypes.c_char_p, [vp]),
        "fhp_batch_add": (ctypes.c_int, [vp, i32, i32, ctypes.c_uint64, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int32)]),
        "fhp_batch_remove": (ctypes.c_int, [vp, i32]),
        "fhp_batch_set_state": (ctypes.c_int, [vp, i32, u8p]),
        "fhp_batch_get_state": (ctypes.c_int, [vp, i32, u8p]),
        "fhp_batch_set_time": (ctypes.c_int, [vp, i32, i64]),
        "fhp_batch_get_time": (i64, [vp, i32]),
        "fhp_batch_set_steps_left": (ctypes.c_int, [vp, i32, i64]),
        "fhp_batch_get_steps_left": (i64, [vp, i32]),
        "fhp_batch_step": (ctypes.c_int, [vp, i64]),
        "fhp_batch_set_graph_steps": (ctypes.c_int, [vp, i32]),
        "fhp_batch_coarse_grain": (ctypes.c_int, [vp, i32, i32, vp, vp, vp, vp]),
        "fhp_batch_synchronize": (ctypes.c_int, [vp]),
        "fhp_batch_count": (i32, [vp]),
        "fhp_batch_free_bytes": (ctypes.c_size_t, [vp]),
        "fhp_batch_kernel_launches": (i64, [vp]),
        "fhp_debug_build": (ctypes.c_int, []),
        "fhp_debug_canaries": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "fhp_batch_debug_canaries": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32),
                                                    ctypes.POINTER(ctypes.c_int32)]),
        "fhp_debug_selftest": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def required_bytes(width: int, height: int) -> int:
    return int(load().fhp_required_bytes(width, height))


class Lattice:
    """One FHP lattice resident on a CUDA device.

    ``width`` x ``height`` nodes (width a multiple of 32, height even),
    counter-based random stream keyed by ``seed``, forcing probability
    ``forcing_p``.  Device memory comes from torch on ``device``; work is
    enqueued on ``stream`` (a torch.cuda.Stream, default: the current stream).
    """

    def __init__(self, width: int, height: int, seed: int = 0, forcing_p: float = 0.0,
                 device=None, stream=None, step_kernel: int = 0):
        torch = _torch()
        self._lib = load()
        self.width, self.height = int(width), int(height)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        nbytes = self._lib.fhp_required_bytes(self.width, self.height)
        if nbytes == 0:
            raise FhpError(FHP_EINVAL, f"invalid lattice {width} x {height}")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self._mem.data_ptr()
            aligned = (base + 255) & ~255
            p = _Params(self.width, self.height, int(seed) & (2**64 - 1), float(forcing_p),
                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.c_void_p(aligned), nbytes)
            h = ctypes.c_void_p()
            rc = self._lib.fhp_create(ctypes.byref(h), ctypes.byref(p))
        if rc != FHP_OK:
            raise FhpError(rc, self._lib.fhp_last_error(None).decode())
        self._h = h
        self.seed = int(seed)
        self.forcing_p = float(forcing_p)
        if step_kernel:
            self.set_step_kernel(step_kernel)

    # -- plumbing -------------------------------------------------------------
    def _check(self, rc: int):
        if rc != FHP_OK:
            raise FhpError(rc, self._lib.fhp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fhp_destroy(self._h)
            self._h = None
            self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self):
        return (self.height, self.width)

    # -- state ----------------------------------------------------------------
    def set_state(self, state: np.ndarray):
        s = np.ascontiguousarray(state, dtype=np.uint8)
        if s.shape != self.shape:
            raise ValueError(f"state must be {self.shape}, got {s.shape}")
        self._check(self._lib.fhp_set_state(self._h, _ptr(s)))

    def get_state(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.uint8)
        self._check(self._lib.fhp_get_state(self._h, _ptr(out)))
        return out

    def set_state_tensor(self, t):
        torch = _torch()
        if t.dtype != torch.uint8 or tuple(t.shape) != self.shape or not t.is_contiguous() \
                or t.device != self.device:
            raise ValueError("expected a contiguous uint8 tensor of shape (H, W) on the lattice's device")
        self._check(self._lib.fhp_set_state_device(self._h, ctypes.c_void_p(t.data_ptr())))

    def get_state_tensor(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.uint8, device=self.device)
        self._check(self._lib.fhp_get_state_device(self._h, ctypes.c_void_p(out.data_ptr())))
        return out

    def load_obstacles(self, mask: np.ndarray):
        m = np.ascontiguousarray(mask).astype(np.uint8, copy=False)
        if m.shape != self.shape:
            raise ValueError(f"mask must be {self.shape}")
        self._check(self._lib.fhp_load_obstacles(self._h, _ptr(m)))

    def load_obstacle_shapes(self, shapes):
        """Obstacles generated on the device from (kind, a, b, c) shapes:
        SHAPE_DISC (x-a)^2 + (y-b)^2 <= c^2, SHAPE_ROWS a <= y < b."""
        arr, n = _shapes(shapes)
        self._check(self._lib.fhp_load_obstacle_shapes(self._h, arr, n))

    def init_random(self, density: float):
        """Generated Bernoulli(density) occupation of every fluid node."""
        self._check(self._lib.fhp_init_random(self._h, float(density)))

    # -- dynamics -------------------------------------------------------------
    def step(self, n: int = 1):
        self._check(self._lib.fhp_step(self._h, int(n)))

    @property
    def t(self) -> int:
        return int(self._lib.fhp_get_time(self._h))

    def set_time(self, t: int):
        self._check(self._lib.fhp_set_time(self._h, int(t)))

    def set_forcing(self, p: float):
        self._check(self._lib.fhp_set_forcing(self._h, float(p)))
        self.forcing_p = float(p)

    def set_temporal_block(self, k: int):
        self._check(self._lib.fhp_set_temporal_block(self._h, int(k)))

    def set_temporal_block_kernel(self, kind: int):
        """0: automatic; 1: row wavefronts; 2: 2-D tiles (see fhp.h)."""
        self._check(self._lib.fhp_set_temporal_block_kernel(self._h, int(kind)))

    @property
    def temporal_block_kernel(self) -> int:
        """Kernel of the blocked passes fhp_step runs: 1 wavefronts, 2 tiles, 0 none."""
        return int(self._lib.fhp_get_temporal_block_kernel(self._h))

    def set_step_kernel(self, kind: int):
        """0 automatic, 1 direct register loads, 2 bulk-copy shared-memory ring, 3 multi-step ring,
        4 shared-memory resident lattice."""
        self._check(self._lib.fhp_set_step_kernel(self._h, int(kind)))

    # -- collision rules -------------------------------------------------------------
    def set_rules(self, rules: int):
        """2: FHP-II (default); 1: FHP-I (no rest-particle collisions); 3: FHP-III
        (collision-saturated; steps with the direct and ring kernels)."""
        self._check(self._lib.fhp_set_rules(self._h, int(rules)))

    @property
    def rules(self) -> int:
        return int(self._lib.fhp_get_rules(self._h))

    # -- strips of a larger lattice ------------------------------------------------
    def set_row_offset(self, row_base: int):
        """Array row y is row row_base + y of a larger lattice (even row_base)."""
        self._check(self._lib.fhp_set_row_offset(self._h, int(row_base)))

    @property
    def row_pitch_words(self) -> int:
        return int(self._lib.fhp_row_pitch_words(self._h))

    def get_rows_tensor(self, y0: int, n: int, out=None):
        """Rows [y0, y0+n) of the 7 state planes as an int32 CUDA tensor [7, n, pitch]."""
        torch = _torch()
        if out is None:
            out = torch.empty((7, int(n), self.row_pitch_words), dtype=torch.int32, device=self.device)
        self._check(self._lib.fhp_get_rows_device(self._h, int(y0), int(n), ctypes.c_void_p(out.data_ptr())))
        return out

    def set_rows_tensor(self, y0: int, rows):
        """Inverse of get_rows_tensor (an int32 CUDA tensor [7, n, pitch])."""
        if rows.dim() != 3 or rows.shape[0] != 7 or rows.shape[2] != self.row_pitch_words or not rows.is_contiguous():
            raise ValueError("rows must be a contiguous [7, n, pitch] tensor")
        self._check(self._lib.fhp_set_rows_device(self._h, int(y0), int(rows.shape[1]),
                                                  ctypes.c_void_p(rows.data_ptr())))

    @property
    def temporal_block(self) -> int:
        return int(self._lib.fhp_get_temporal_block(self._h))

    def autotune(self, trial_steps: int = 64) -> tuple[int, int]:
        """Time the step configurations on this lattice and record the
        fastest for its shape; returns (kernel, temporal block)."""
        kern, k = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self._lib.fhp_autotune(self._h, int(trial_steps), ctypes.byref(kern), ctypes.byref(k)))
        return kern.value, k.value

    @property
    def step_kernel(self) -> int:
        return int(self._lib.fhp_get_step_kernel(self._h))

    def synchronize(self):
        self._check(self._lib.fhp_synchronize(self._h))

    def debug_canaries(self) -> tuple[int, int]:
        """(canary blocks checked, blocks corrupted); (0, 0) in the release build."""
        checked, corrupted = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self._lib.fhp_debug_canaries(self._h, ctypes.byref(checked), ctypes.byref(corrupted)))
        return checked.value, corrupted.value

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.fhp_kernel_launches(self._h))

    # -- observables ----------------------------------------------------------
    def coarse_grain(self, block: int = 32):
        nby, nbx = self.height // block, self.width // block
        counts = np.empty((nby, nbx, 9), dtype=np.int32)
        rho = np.empty((nby, nbx), dtype=np.float32)
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        self._check(self._lib.fhp_coarse_grain(self._h, int(block), _ptr(counts), _ptr(rho),
                                               _ptr(ux), _ptr(uy)))
        return counts, rho, ux, uy

    def coarse_grain_into(self, block: int, counts, rho, ux, uy):
        """Coarse-grain into preallocated device tensors (asynchronous)."""
        self._check(self._lib.fhp_coarse_grain_device(
            self._h, int(block), ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
            ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(uy.data_ptr())))

    def coarse_grain_host_into(self, block: int, counts: np.ndarray, rho: np.ndarray,
                               ux: np.ndarray, uy: np.ndarray):
        """Coarse-grain into preallocated host arrays (synchronous)."""
        self._check(self._lib.fhp_coarse_grain(self._h, int(block), _ptr(counts), _ptr(rho),
                                               _ptr(ux), _ptr(uy)))

    def coarse_grain_tensor(self, block: int = 32):
        torch = _torch()
        nby, nbx = self.height // block, self.width // block
        counts = torch.empty((nby, nbx, 9), dtype=torch.int32, device=self.device)
        rho = torch.empty((nby, nbx), dtype=torch.float32, device=self.device)
        ux = torch.empty_like(rho)
        uy = torch.empty_like(rho)
        self._check(self._lib.fhp_coarse_grain_device(
            self._h, int(block), ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
            ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(uy.data_ptr())))
        return counts, rho, ux, uy


class Batch:
    """Many independent FHP lattices advanced by shared kernel launches.

    Members are added and removed while the batch lives (continuous
    batching); each keeps its own seed, forcing probability, obstacles, step
    counter and optional step budget, and evolves exactly as it would alone.
    The batch's device arena is a torch allocation of ``arena_bytes``.
    """

    def __init__(self, arena_bytes: int, device=None, stream=None):
        torch = _torch()
        self._lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._mem = torch.empty(int(arena_bytes) + 256, dtype=torch.uint8, device=self.device)
            aligned = (self._mem.data_ptr() + 255) & ~255
            h = ctypes.c_void_p()
            rc = self._lib.fhp_batch_create(ctypes.byref(h), int(arena_bytes), ctypes.c_void_p(aligned),
                                            ctypes.c_void_p(self.stream.cuda_stream))
        if rc != FHP_OK:
            raise FhpError(rc, self._lib.fhp_last_error(None).decode())
        self._h = h
        self.shapes = {}

    def _check(self, rc: int):
        if rc != FHP_OK:
            raise FhpError(rc, self._lib.fhp_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fhp_batch_destroy(self._h)
            self._h = None
            self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def lattice_bytes(width: int, height: int) -> int:
        return int(load().fhp_batch_lattice_bytes(int(width), int(height)))

    @staticmethod
    def block_rows(width: int, height: int, k: int) -> int:
        """Output rows per blocked tile of a member at temporal block k (0: it takes no blocked passes)."""
        return int(load().fhp_batch_block_rows(int(width), int(height), int(k)))

    def add(self, width: int, height: int, seed: int = 0, forcing_p: float = 0.0) -> int:
        slot = ctypes.c_int32(-1)
        self._check(self._lib.fhp_batch_add(self._h, int(width), int(height), int(seed) & (2**64 - 1),
                                            float(forcing_p), ctypes.byref(slot)))
        self.shapes[slot.value] = (int(height), int(width))
        return slot.value

    def remove(self, slot: int, wait: bool = True):
        """Return a member's memory to the arena.  wait=False does not wait for
        queued work (see fhp_batch_remove_async)."""
        fn = self._lib.fhp_batch_remove if wait else self._lib.fhp_batch_remove_async
        self._check(fn(self._h, int(slot)))
        self.shapes.pop(int(slot), None)

    def coarse_grain_begin(self, slot: int, block: int, after_event=None):
        """Start reading back a member's coarse-grained fields on a side stream
        (optionally after a torch.cuda.Event recorded on the batch's stream);
        returns a handle for coarse_grain_finish.  Device outputs go to pinned
        host buffers without blocking the batch's stream."""
        torch = _torch()
        if getattr(self, "_side", None) is None:
            self._side = torch.cuda.Stream(device=self.device)
        s = self._side
        H, W = self.shapes[slot]
        nby, nbx = H // block, W // block
        if after_event is not None:
            s.wait_event(after_event)
        with torch.cuda.stream(s):
            dev = [torch.empty((nby, nbx, 9), dtype=torch.int32, device=self.device)] + \
                  [torch.empty((nby, nbx), dtype=torch.float32, device=self.device) for _ in range(3)]
            self._check(self._lib.fhp_batch_coarse_grain_device(
                self._h, int(slot), int(block), *[ctypes.c_void_p(t.data_ptr()) for t in dev],
                ctypes.c_void_p(s.cuda_stream)))
            host = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in dev]
            for hsrc, dsrc in zip(host, dev):
                hsrc.copy_(dsrc, non_blocking=True)
        return (s, dev, host)

    @staticmethod
    def coarse_grain_finish(handle):
        """Wait for a read-back started by coarse_grain_begin; returns
        (counts, rho, ux, uy) as numpy arrays."""
        s, dev, host = handle
        s.synchronize()
        return tuple(h.numpy() for h in host)

    def set_state(self, slot: int, state: np.ndarray):
        s = np.ascontiguousarray(state, dtype=np.uint8)
        if s.shape != self.shapes[slot]:
            raise ValueError(f"state must be {self.shapes[slot]}")
        self._check(self._lib.fhp_batch_set_state(self._h, int(slot), _ptr(s)))

    def init_random(self, slot: int, density: float):
        self._check(self._lib.fhp_batch_init_random(self._h, int(slot), float(density)))

    def set_rules(self, slot: int, rules: int):
        self._check(self._lib.fhp_batch_set_rules(self._h, int(slot), int(rules)))

    def load_obstacle_shapes(self, slot: int, shapes):
        arr, n = _shapes(shapes)
        self._check(self._lib.fhp_batch_load_obstacle_shapes(self._h, int(slot), arr, n))

    def load_obstacles(self, slot: int, mask: np.ndarray):
        m = np.ascontiguousarray(mask).astype(np.uint8, copy=False)
        if m.shape != self.shapes[slot]:
            raise ValueError(f"mask must be {self.shapes[slot]}")
        self._check(self._lib.fhp_batch_load_obstacles(self._h, int(slot), _ptr(m)))

    def get_state(self, slot: int) -> np.ndarray:
        out = np.empty(self.shapes[slot], dtype=np.uint8)
        self._check(self._lib.fhp_batch_get_state(self._h, int(slot), _ptr(out)))
        return out

    def set_time(self, slot: int, t: int):
        self._check(self._lib.fhp_batch_set_time(self._h, int(slot), int(t)))

    def time(self, slot: int) -> int:
        return int(self._lib.fhp_batch_get_time(self._h, int(slot)))

    def set_steps_left(self, slot: int, n: int):
        self._check(self._lib.fhp_batch_set_steps_left(self._h, int(slot), int(n)))

    def steps_left(self, slot: int) -> int:
        return int(self._lib.fhp_batch_get_steps_left(self._h, int(slot)))

    def step(self, n: int = 1):
        self._check(self._lib.fhp_batch_step(self._h, int(n)))

    def set_step_kernel(self, kind: int):
        """0 automatic, 1 one launch per step (CUDA graphs), 2 all steps of a
        call in one cooperative launch."""
        self._check(self._lib.fhp_batch_set_step_kernel(self._h, int(kind)))

    @property
    def step_kernel(self) -> int:
        return int(self._lib.fhp_batch_get_step_kernel(self._h))

    @property
    def tile_count(self) -> int:
        return int(self._lib.fhp_batch_tile_count(self._h))

    def tuned_kernel(self, ntiles: int | None = None) -> int:
        """Kernel the automatic choice recorded for this many tiles at the
        default tile size (None: the current members; 0: none yet)."""
        n = 0 if ntiles is None else int(ntiles)
        return int(self._lib.fhp_batch_get_tuned_kernel(self._h, n))

    def tuned_tile_quads(self, ntiles: int | None = None) -> int:
        """Tile size recorded with the tuned kernel (0: none yet)."""
        n = 0 if ntiles is None else int(ntiles)
        return int(self._lib.fhp_batch_get_tuned_tile_quads(self._h, n))

    def set_tile_quads(self, quads: int):
        """Quads (128-node units) per tile: 64, 128, 256, or 0 = tuned online."""
        self._check(self._lib.fhp_batch_set_tile_quads(self._h, int(quads)))

    @property
    def tile_quads(self) -> int:
        """Tile size of the current tile list."""
        return int(self._lib.fhp_batch_get_tile_quads(self._h))

    def set_graph_steps(self, n: int):
        self._check(self._lib.fhp_batch_set_graph_steps(self._h, int(n)))

    def set_temporal_block(self, k: int):
        """Steps per blocked pass: 2 or 4, 1 = none, 0 = tuned online with the kernel."""
        self._check(self._lib.fhp_batch_set_temporal_block(self._h, int(k)))

    @property
    def temporal_block(self) -> int:
        """The temporal-block setting (0: automatic)."""
        return int(self._lib.fhp_batch_get_temporal_block(self._h))

    def tuned_temporal_block(self, ntiles: int | None = None) -> int:
        """Temporal block the automatic choice recorded for this batch's size class (0: not yet)."""
        n = 0 if ntiles is None else int(ntiles)
        return int(self._lib.fhp_batch_get_tuned_temporal_block(self._h, n))

    def coarse_grain(self, slot: int, block: int = 32):
        H, W = self.shapes[slot]
        nby, nbx = H // block, W // block
        counts = np.empty((nby, nbx, 9), dtype=np.int32)
        rho = np.empty((nby, nbx), dtype=np.float32)
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        self._check(self._lib.fhp_batch_coarse_grain(self._h, int(slot), int(block), _ptr(counts), _ptr(rho),
                                                     _ptr(ux), _ptr(uy)))
        return counts, rho, ux, uy

    def synchronize(self):
        self._check(self._lib.fhp_batch_synchronize(self._h))

    def debug_canaries(self) -> tuple[int, int]:
        """(canary blocks checked, blocks corrupted) over the members; (0, 0) in the release build."""
        checked, corrupted = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self._lib.fhp_batch_debug_canaries(self._h, ctypes.byref(checked), ctypes.byref(corrupted)))
        return checked.value, corrupted.value

    @property
    def count(self) -> int:
        return int(self._lib.fhp_batch_count(self._h))

    @property
    def free_bytes(self) -> int:
        return int(self._lib.fhp_batch_free_bytes(self._h))

    @property
    def kernel_launches(self) -> int:
        return int(self._lib.fhp_batch_kernel_launches(self._h))


def selftest_wait_limits() -> int:
    """Run the bounded device-side waits on conditions that never hold;
    returns the status bits (3: both waits gave up as designed)."""
    lib = load()
    st = ctypes.c_uint32(0)
    rc = lib.fhp_selftest_wait_limits(ctypes.byref(st))
    if rc != FHP_OK:
        raise FhpError(rc, "wait self-test failed")
    return int(st.value)


def philox4x32_10_device(ctr, key, stream=None):
    """Philox4x32-10 blocks computed by the library's device code.

    ``ctr``: uint32-valued int64/int32 tensor (n, 4) on the GPU; ``key``: (n, 2)."""
    torch = _torch()
    lib = load()
    c = ctr.to(torch.int32).contiguous()
    k = key.to(torch.int32).contiguous()
    out = torch.empty_like(c)
    s = stream if stream is not None else torch.cuda.current_stream(c.device)
    rc = lib.fhp_philox4x32_10_device(ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(k.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), c.shape[0],
                                      ctypes.c_void_p(s.cuda_stream))
    if rc != FHP_OK:
        raise FhpError(rc, lib.fhp_last_error(None).decode())
    return out
