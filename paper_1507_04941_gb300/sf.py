"""Python binding of libsf.so (include/sf.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; PyTorch only
provides device memory and the current stream.  Importing works without a
GPU; any call that needs the library raises when it is not built or cannot be
loaded (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SF_OK, SF_EINVAL, SF_ENOMEM, SF_EBUDGET, SF_ECUDA, SF_ETIMEOUT, SF_ESTATE, SF_EJIT, SF_ECANCELED = range(9)
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}

_lock = threading.Lock()
_lib = None


class SfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_str(status)}: {message}")
        self.status = status


class FilterSpec(ctypes.Structure):
    _fields_ = [("sigma_xy", ctypes.c_float), ("sigma_z", ctypes.c_float)]


class Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("n_filters", ctypes.c_int32), ("filters", ctypes.POINTER(FilterSpec)),
                ("truncation", ctypes.c_float), ("wx", ctypes.c_int32), ("wy", ctypes.c_int32),
                ("wz", ctypes.c_int32), ("k", ctypes.c_float), ("storage", ctypes.c_int32),
                ("stats_fp64", ctypes.c_int32), ("device", ctypes.c_int32),
                ("std_ddof", ctypes.c_int32)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64

# name -> (restype, argtypes); every function declared in include/sf.h
SIGNATURES = {
    "sf_create": (_i32, [ctypes.POINTER(Config), ctypes.POINTER(_vp)]),
    "sf_destroy": (_i32, [_vp]),
    "sf_status_str": (ctypes.c_char_p, [_i32]),
    "sf_last_error": (ctypes.c_char_p, [_vp]),
    "sf_taps": (_i32, [_vp, _i32, _i32, ctypes.POINTER(ctypes.c_float), _i32,
                       ctypes.POINTER(_i32)]),
    "sf_window_grid": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                              ctypes.POINTER(_i32)]),
    "sf_mask_words": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "sf_filter": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "sf_stats": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "sf_threshold": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _vp]),
    "sf_detect": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "sf_detect_host": (_i32, [_vp, _vp, _vp, _vp]),
    "sf_detect_slab": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "sf_synchronize": (_i32, [_vp, _vp]),
    "sf_create_sectioned": (_i32, [ctypes.POINTER(Config), _i64, ctypes.POINTER(_vp)]),
    "sf_create_batch": (_i32, [ctypes.POINTER(Config), _i32, ctypes.POINTER(_i64),
                               ctypes.POINTER(_vp)]),
    "sf_detect_batch": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                               ctypes.POINTER(_vp), _vp]),
    "sf_tune": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    "sf_tune_report": (_i32, [_vp, ctypes.c_char_p, _i32]),
    "sf_server_create": (_i32, [ctypes.POINTER(Config), _i64, _i32, ctypes.POINTER(_vp)]),
    "sf_server_submit": (_i32, [_vp, _vp, _i64, _i64, _i64, _vp, ctypes.POINTER(_i64)]),
    "sf_server_cancel": (_i32, [_vp, _i64]),
    "sf_server_poll": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i64),
                              _i32, _i32, ctypes.POINTER(_i32)]),
    "sf_server_stats": (_i32, [_vp, ctypes.POINTER(_i64), _i32]),
    "sf_server_destroy": (_i32, [_vp]),
    "sf_filter_noalloc": (_i32, [_vp, _i64, _i64, _i64, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, _vp, _vp]),
    "sf_local_stats": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp]),
    "sf_local_detect": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "sf_local_zscore": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "sf_weighted_filter": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    "sf_weighted_detect": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "sf_profile_enable": (_i32, [_vp, _i32]),
    "sf_profile_read": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]),
    "sf_set_wait_limit": (_i32, [_vp, _i64]),
    "sf_test_stall_batch": (_i32, [_vp, _i32]),
    "sf_fp32_peak": (_i32, [_i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "sf_fp32_peak_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libsf.so (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built: call __graft_entry__.build() first")
        handle = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
        return handle


def status_str(status: int) -> str:
    try:
        return lib().sf_status_str(int(status)).decode()
    except Exception:  # noqa: BLE001 - library missing: plain number
        return f"status {int(status)}"


def _check(status: int, ctx=None):
    if status != SF_OK:
        msg = lib().sf_last_error(ctx).decode(errors="replace")
        raise SfError(status, msg)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(device):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class SourceFinder:
    """One planned filter bank over cubes of one shape (wraps an sf_ctx)."""

    def __init__(self, shape, bank, truncation: float = 3.0, window=(32, 32, 64), k: float = 4.0,
                 storage: str = "f32", device=None, stats_fp64: bool = False, std_ddof: int = 0):
        import torch
        self.shape = tuple(int(s) for s in shape)
        self.bank = tuple((float(a), float(b)) for a, b in bank)
        self.truncation = float(truncation)
        self.window = tuple(int(w) for w in window)
        self.k = float(k)
        self.storage = storage
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        specs = (FilterSpec * len(self.bank))(*[FilterSpec(a, b) for a, b in self.bank])
        self._specs = specs
        cfg = Config(self.shape[0], self.shape[1], self.shape[2], len(self.bank), specs,
                     self.truncation, self.window[0], self.window[1], self.window[2], self.k,
                     STORAGE[storage], 1 if stats_fp64 else 0,
                     self.device.index if self.device.index is not None else -1, int(std_ddof))
        h = _vp()
        _check(lib().sf_create(ctypes.byref(cfg), ctypes.byref(h)), None)
        self._h = h
        nwx, nwy, nwz = _i32(), _i32(), _i32()
        _check(lib().sf_window_grid(h, ctypes.byref(nwx), ctypes.byref(nwy), ctypes.byref(nwz)), h)
        self.grid = (nwx.value, nwy.value, nwz.value)
        words = _i64()
        _check(lib().sf_mask_words(h, ctypes.byref(words)), h)
        self.mask_words = words.value

    # -- helpers --------------------------------------------------------------------
    @property
    def handle(self):
        return self._h

    @property
    def n_windows(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def mask_shape(self):
        return (self.shape[0], self.shape[1], -(-self.shape[2] // 32))

    def _torch_dtype(self):
        import torch
        return {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.storage]

    def _check_cube(self, cube):
        if tuple(cube.shape) != self.shape or cube.dtype != self._torch_dtype() \
                or not cube.is_contiguous() or cube.device != self.device:
            raise ValueError(f"cube must be a contiguous {self._torch_dtype()} tensor of shape "
                             f"{self.shape} on {self.device}")

    def _check_f32(self, t, shape, name):
        import torch
        if tuple(t.shape) != tuple(shape) or t.dtype != torch.float32 or not t.is_contiguous() \
                or t.device != self.device:
            raise ValueError(f"{name} must be a contiguous float32 tensor of shape {shape} "
                             f"on {self.device}")

    def taps(self, filter_index: int, axis: int) -> np.ndarray:
        r = _i32()
        _check(lib().sf_taps(self._h, filter_index, axis, None, 0, ctypes.byref(r)), self._h)
        out = np.empty(2 * r.value + 1, dtype=np.float32)
        _check(lib().sf_taps(self._h, filter_index, axis,
                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size,
                             ctypes.byref(r)), self._h)
        return out

    # -- entry points --------------------------------------------------------------------
    def filter(self, cube, filter_index: int, out=None):
        import torch
        self._check_cube(cube)
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        self._check_f32(out, self.shape, "out")
        _check(lib().sf_filter(self._h, _ptr(cube), int(filter_index), _ptr(out),
                               _stream(self.device)), self._h)
        return out

    def stats(self, filtered, mean=None, std=None):
        import torch
        self._check_f32(filtered, self.shape, "filtered")
        if mean is None:
            mean = torch.empty(self.grid, dtype=torch.float32, device=self.device)
        if std is None:
            std = torch.empty(self.grid, dtype=torch.float32, device=self.device)
        self._check_f32(mean, self.grid, "mean")
        self._check_f32(std, self.grid, "std")
        _check(lib().sf_stats(self._h, _ptr(filtered), _ptr(mean), _ptr(std),
                              _stream(self.device)), self._h)
        return mean, std

    def threshold(self, filtered, mean, std, mask=None, accumulate: bool = False):
        import torch
        self._check_f32(filtered, self.shape, "filtered")
        self._check_f32(mean, self.grid, "mean")
        self._check_f32(std, self.grid, "std")
        if mask is None:
            mask = torch.zeros(self.mask_shape, dtype=torch.int32, device=self.device)
        _check(lib().sf_threshold(self._h, _ptr(filtered), _ptr(mean), _ptr(std), _ptr(mask),
                                  int(bool(accumulate)), _stream(self.device)), self._h)
        return mask

    def detect(self, cube, mask=None, stats: bool = False):
        """Packed mask (int32 view of the uint32 words); with stats=True also
        (mean, std) as float32 [n_filters][nwx][nwy][nwz]."""
        import torch
        self._check_cube(cube)
        if mask is None:
            mask = torch.empty(self.mask_shape, dtype=torch.int32, device=self.device)
        mean = std = None
        if stats:
            shp = (len(self.bank),) + self.grid
            mean = torch.empty(shp, dtype=torch.float32, device=self.device)
            std = torch.empty(shp, dtype=torch.float32, device=self.device)
        _check(lib().sf_detect(self._h, _ptr(cube), _ptr(mask), _ptr(mean), _ptr(std),
                               _stream(self.device)), self._h)
        return (mask, mean, std) if stats else mask

    def detect_slab(self, ext, halo: int, mask=None, stats: bool = False):
        """sf_detect_slab: `ext` is this context's cube, an x slab with `halo`
        neighbour planes on each side; returns the slab's mask words
        [nx - 2 halo][ny][ceil(nz/32)] (and with stats=True its windows'
        mean, std [n_filters][ceil(S/wx)][nwy][nwz])."""
        import torch
        self._check_cube(ext)
        halo = int(halo)
        S = self.shape[0] - 2 * halo
        if S < 1:
            raise ValueError("the slab needs at least one plane between its halos")
        if mask is None:
            mask = torch.empty((S,) + self.mask_shape[1:], dtype=torch.int32, device=self.device)
        mean = std = None
        if stats:
            shp = (len(self.bank), -(-S // self.window[0])) + self.grid[1:]
            mean = torch.empty(shp, dtype=torch.float32, device=self.device)
            std = torch.empty(shp, dtype=torch.float32, device=self.device)
        _check(lib().sf_detect_slab(self._h, _ptr(ext), halo, _ptr(mask), _ptr(mean), _ptr(std),
                                    _stream(self.device)), self._h)
        return (mask, mean, std) if stats else mask

    def local_stats(self, filtered, half, mean=None, std=None):
        """Per-voxel mean and std of a filtered cube over the box of
        half-widths half = (sx, sy, sz) clipped to the cube (float32, the
        cube's shape)."""
        import torch
        self._check_f32(filtered, self.shape, "filtered")
        if mean is None:
            mean = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        if std is None:
            std = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        self._check_f32(mean, self.shape, "mean")
        self._check_f32(std, self.shape, "std")
        sx, sy, sz = (int(v) for v in half)
        _check(lib().sf_local_stats(self._h, _ptr(filtered), sx, sy, sz, _ptr(mean), _ptr(std),
                                    _stream(self.device)), self._h)
        return mean, std

    def local_zscore(self, filtered, half, out=None):
        """Per-voxel z-score (c - mean) / std over the box of half-widths
        half = (sx, sy, sz), 0 where std = 0 (float32, the cube's shape)."""
        import torch
        self._check_f32(filtered, self.shape, "filtered")
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        self._check_f32(out, self.shape, "out")
        sx, sy, sz = (int(v) for v in half)
        _check(lib().sf_local_zscore(self._h, _ptr(filtered), sx, sy, sz, _ptr(out),
                                     _stream(self.device)), self._h)
        return out

    def local_detect(self, cube, half, mask=None):
        """Packed mask of the detect with per-voxel local statistics over the
        box of half-widths half = (sx, sy, sz)."""
        import torch
        self._check_cube(cube)
        if mask is None:
            mask = torch.empty(self.mask_shape, dtype=torch.int32, device=self.device)
        sx, sy, sz = (int(v) for v in half)
        _check(lib().sf_local_detect(self._h, _ptr(cube), sx, sy, sz, _ptr(mask),
                                     _stream(self.device)), self._h)
        return mask

    DEN = {"fw": 0, "w": 1}

    def weighted_filter(self, cube, weights, filter_index: int, den: str = "fw", out=None):
        """Eq. 1 for one filter: sum d f w / D, D = sum f w (den="fw") or
        sum w (den="w", as printed); float32 cube of the context's shape."""
        import torch
        self._check_f32(cube, self.shape, "cube")
        self._check_f32(weights, self.shape, "weights")
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        self._check_f32(out, self.shape, "out")
        _check(lib().sf_weighted_filter(self._h, _ptr(cube), _ptr(weights), int(filter_index),
                                        self.DEN[den], _ptr(out), _stream(self.device)), self._h)
        return out

    def weighted_detect(self, cube, weights, den: str = "fw", mask=None, stats: bool = False):
        """Packed mask of the method with Eq. 1 filtering; with stats=True also
        (mean, std) as float32 [n_filters][nwx][nwy][nwz]."""
        import torch
        self._check_f32(cube, self.shape, "cube")
        self._check_f32(weights, self.shape, "weights")
        if mask is None:
            mask = torch.empty(self.mask_shape, dtype=torch.int32, device=self.device)
        mean = std = None
        if stats:
            shp = (len(self.bank),) + self.grid
            mean = torch.empty(shp, dtype=torch.float32, device=self.device)
            std = torch.empty(shp, dtype=torch.float32, device=self.device)
        _check(lib().sf_weighted_detect(self._h, _ptr(cube), _ptr(weights), self.DEN[den], _ptr(mask),
                                        _ptr(mean), _ptr(std), _stream(self.device)), self._h)
        return (mask, mean, std) if stats else mask

    def detect_host(self, cube_host, mask_host=None):
        """Host tensors in and out (pinned memory makes the copies DMA)."""
        import torch
        if tuple(cube_host.shape) != self.shape or cube_host.dtype != self._torch_dtype() \
                or cube_host.device.type != "cpu" or not cube_host.is_contiguous():
            raise ValueError("cube_host must be a contiguous CPU tensor of the cube shape/dtype")
        if mask_host is None:
            mask_host = torch.empty(self.mask_shape, dtype=torch.int32,
                                    pin_memory=cube_host.is_pinned())
        _check(lib().sf_detect_host(self._h, _ptr(cube_host), _ptr(mask_host),
                                    _stream(self.device)), self._h)
        return mask_host

    def tune(self, cube, mask=None):
        """Autotune the launch path on this cube (blocking); returns the timings report."""
        import torch
        self._check_cube(cube)
        if mask is None:
            mask = torch.empty(self.mask_shape, dtype=torch.int32, device=self.device)
        cubes = (_vp * 1)(cube.data_ptr())
        masks = (_vp * 1)(mask.data_ptr())
        _check(lib().sf_tune(self._h, cubes, masks, _stream(self.device)), self._h)
        return tune_report(self._h)

    def synchronize(self):
        """Wait for this context's work on the current stream; raise on kernel-side timeouts."""
        _check(lib().sf_synchronize(self._h, _stream(self.device)), self._h)

    def set_wait_limit(self, ns: int):
        """Limit of the kernels' bounded waits in ns (sf_set_wait_limit)."""
        _check(lib().sf_set_wait_limit(self._h, int(ns)), self._h)

    def profile(self, enable: bool = True):
        """Record CUDA events around the stages of every sf_detect."""
        _check(lib().sf_profile_enable(self._h, int(bool(enable))), self._h)

    def profile_read(self, n_stages: int = 2):
        """{stage: (milliseconds, launches)} since the last read (0: x pass, 1: window kernel)."""
        ms = (ctypes.c_double * n_stages)()
        nl = (_i64 * n_stages)()
        _check(lib().sf_profile_read(self._h, ms, nl, n_stages), self._h)
        return {i: (ms[i], nl[i]) for i in range(n_stages)}

    def close(self):
        if getattr(self, "_h", None):
            lib().sf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tune_report(handle) -> str:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().sf_tune_report(handle, buf, len(buf)), handle)
    return buf.value.decode()


class SectionedSourceFinder:
    """Detect on a cube held in host memory, section by section along x, with
    device memory bounded by the section size (wraps a sectioned sf_ctx)."""

    def __init__(self, shape, bank, truncation: float = 3.0, window=(32, 32, 64), k: float = 4.0,
                 section: int = 256, storage: str = "f32", device=None, std_ddof: int = 0):
        import torch
        self.shape = tuple(int(s) for s in shape)
        self.bank = tuple((float(a), float(b)) for a, b in bank)
        self.window = tuple(int(w) for w in window)
        self.storage = storage
        self.section = int(section)
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        specs = (FilterSpec * len(self.bank))(*[FilterSpec(a, b) for a, b in self.bank])
        self._specs = specs
        cfg = Config(self.shape[0], self.shape[1], self.shape[2], len(self.bank), specs,
                     float(truncation), self.window[0], self.window[1], self.window[2], float(k),
                     STORAGE[storage], 0, self.device.index if self.device.index is not None else -1,
                     int(std_ddof))
        h = _vp()
        _check(lib().sf_create_sectioned(ctypes.byref(cfg), self.section, ctypes.byref(h)), None)
        self._h = h

    @property
    def mask_shape(self):
        return (self.shape[0], self.shape[1], -(-self.shape[2] // 32))

    def detect_host(self, cube_host, mask_host=None):
        """Host tensors in and out (pinned memory makes the copies DMA)."""
        import torch
        dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.storage]
        if tuple(cube_host.shape) != self.shape or cube_host.dtype != dt \
                or cube_host.device.type != "cpu" or not cube_host.is_contiguous():
            raise ValueError("cube_host must be a contiguous CPU tensor of the cube shape/dtype")
        if mask_host is None:
            mask_host = torch.empty(self.mask_shape, dtype=torch.int32, pin_memory=cube_host.is_pinned())
        _check(lib().sf_detect_host(self._h, _ptr(cube_host), _ptr(mask_host), _stream(self.device)),
               self._h)
        return mask_host

    def close(self):
        if getattr(self, "_h", None):
            lib().sf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchSourceFinder:
    """Many cubes of different shapes, one filter bank (wraps a batched sf_ctx)."""

    def __init__(self, shapes, bank, truncation: float = 3.0, window=(32, 32, 64), k: float = 4.0,
                 storage: str = "f32", device=None, stats_fp64: bool = False, std_ddof: int = 0):
        import torch
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        self.bank = tuple((float(a), float(b)) for a, b in bank)
        self.window = tuple(int(w) for w in window)
        self.storage = storage
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        specs = (FilterSpec * len(self.bank))(*[FilterSpec(a, b) for a, b in self.bank])
        self._specs = specs
        cfg = Config(1, 1, 1, len(self.bank), specs, float(truncation), self.window[0],
                     self.window[1], self.window[2], float(k), STORAGE[storage], 1 if stats_fp64 else 0,
                     self.device.index if self.device.index is not None else -1, int(std_ddof))
        dims = (_i64 * (3 * len(self.shapes)))(*[v for sh in self.shapes for v in sh])
        h = _vp()
        _check(lib().sf_create_batch(ctypes.byref(cfg), len(self.shapes), dims, ctypes.byref(h)),
               None)
        self._h = h

    @property
    def handle(self):
        return self._h

    def mask_shape(self, i):
        nx, ny, nz = self.shapes[i]
        return (nx, ny, -(-nz // 32))

    def grid(self, i):
        return tuple(-(-n // w) for n, w in zip(self.shapes[i], self.window))

    def _arrays(self, cubes, masks, means=None, stds=None):
        n = len(self.shapes)
        if len(cubes) != n or len(masks) != n:
            raise ValueError(f"expected {n} cubes and masks")
        arr = lambda ts: (_vp * n)(*[_ptr(t) for t in ts])  # noqa: E731
        return (arr(cubes), arr(masks), arr(means) if means is not None else None,
                arr(stds) if stds is not None else None)

    def detect(self, cubes, masks=None, stats: bool = False):
        import torch
        dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.storage]
        for i, c in enumerate(cubes):
            if tuple(c.shape) != self.shapes[i] or c.dtype != dt or not c.is_contiguous() \
                    or c.device != self.device:
                raise ValueError(f"cube {i} must be a contiguous {dt} tensor of shape "
                                 f"{self.shapes[i]} on {self.device}")
        if masks is None:
            masks = [torch.empty(self.mask_shape(i), dtype=torch.int32, device=self.device)
                     for i in range(len(cubes))]
        means = stds = None
        if stats:
            means = [torch.empty((len(self.bank),) + self.grid(i), dtype=torch.float32,
                                 device=self.device) for i in range(len(cubes))]
            stds = [torch.empty_like(m) for m in means]
        c_arr, m_arr, me_arr, sd_arr = self._arrays(cubes, masks, means, stds)
        _check(lib().sf_detect_batch(self._h, c_arr, m_arr, me_arr, sd_arr, _stream(self.device)),
               self._h)
        return (masks, means, stds) if stats else masks

    def tune(self, cubes, masks=None):
        import torch
        if masks is None:
            masks = [torch.empty(self.mask_shape(i), dtype=torch.int32, device=self.device)
                     for i in range(len(cubes))]
        c_arr, m_arr, _, _ = self._arrays(cubes, masks)
        _check(lib().sf_tune(self._h, c_arr, m_arr, _stream(self.device)), self._h)
        return tune_report(self._h)

    def profile(self, enable: bool = True):
        _check(lib().sf_profile_enable(self._h, int(bool(enable))), self._h)

    def profile_read(self, n_stages: int = 2):
        ms = (ctypes.c_double * n_stages)()
        nl = (_i64 * n_stages)()
        _check(lib().sf_profile_read(self._h, ms, nl, n_stages), self._h)
        return {i: (ms[i], nl[i]) for i in range(n_stages)}

    def synchronize(self):
        _check(lib().sf_synchronize(self._h, _stream(self.device)), self._h)

    def set_wait_limit(self, ns: int):
        """Limit of the kernels' bounded waits in ns (sf_set_wait_limit)."""
        _check(lib().sf_set_wait_limit(self._h, int(ns)), self._h)

    def test_stall(self, extra: int):
        """Test hook of sf_test_stall_batch (bounded-wait path)."""
        _check(lib().sf_test_stall_batch(self._h, int(extra)), self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib().sf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


SERVER_STATS = ("submitted", "admitted", "completed", "rejected", "bytes_in_use", "peak_bytes",
                "idle_bytes", "evictions", "contexts_created", "busy", "queued", "budget", "cancelled")


class Server:
    """Continuous-batching detection server (wraps sf_server)."""

    def __init__(self, bank, truncation: float = 3.0, window=(32, 32, 64), k: float = 4.0,
                 storage: str = "f16", budget_bytes: int = 150 * 10 ** 9, max_inflight: int = 8,
                 device: int = 0):
        self.bank = tuple((float(a), float(b)) for a, b in bank)
        self.storage = storage
        specs = (FilterSpec * len(self.bank))(*[FilterSpec(a, b) for a, b in self.bank])
        self._specs = specs
        cfg = Config(1, 1, 1, len(self.bank), specs, float(truncation), int(window[0]),
                     int(window[1]), int(window[2]), float(k), STORAGE[storage], 0, int(device))
        h = _vp()
        st = lib().sf_server_create(ctypes.byref(cfg), int(budget_bytes), int(max_inflight),
                                    ctypes.byref(h))
        if st != SF_OK:
            raise SfError(st, "sf_server_create")
        self._h = h
        self._keep = {}

    def submit(self, cube_host, mask_host) -> int:
        """Queue a host cube (storage dtype, contiguous); mask_host receives the words."""
        nx, ny, nz = (int(v) for v in cube_host.shape)
        rid = _i64()
        st = lib().sf_server_submit(self._h, _ptr(cube_host), nx, ny, nz, _ptr(mask_host),
                                    ctypes.byref(rid))
        if st != SF_OK:
            raise SfError(st, "sf_server_submit")
        self._keep[rid.value] = (cube_host, mask_host)
        return rid.value

    def cancel(self, rid: int) -> bool:
        """Cancel a request still waiting for admission (it completes with
        SF_ECANCELED); False if it was already admitted or done."""
        st = lib().sf_server_cancel(self._h, int(rid))
        if st == SF_ESTATE:
            return False
        if st != SF_OK:
            raise SfError(st, "sf_server_cancel")
        return True

    def poll(self, cap: int = 256, timeout_ms: int = 0):
        """[(id, status, latency_seconds)] of requests completed since the last poll."""
        ids = (_i64 * cap)()
        sts = (_i32 * cap)()
        lat = (_i64 * cap)()
        n = _i32()
        st = lib().sf_server_poll(self._h, ids, sts, lat, cap, int(timeout_ms), ctypes.byref(n))
        if st != SF_OK:
            raise SfError(st, "sf_server_poll")
        out = []
        for i in range(n.value):
            self._keep.pop(ids[i], None)
            out.append((ids[i], sts[i], lat[i] * 1e-9))
        return out

    def stats(self) -> dict:
        vals = (_i64 * len(SERVER_STATS))()
        st = lib().sf_server_stats(self._h, vals, len(SERVER_STATS))
        if st != SF_OK:
            raise SfError(st, "sf_server_stats")
        return dict(zip(SERVER_STATS, list(vals)))

    def close(self):
        if getattr(self, "_h", None):
            lib().sf_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def fp32_peak(device: int = 0) -> tuple[float, float]:
    """Measured FP32 peak of the device in TFLOP/s: (scalar fma, packed f32x2 fma)."""
    a = ctypes.c_double()
    b = ctypes.c_double()
    st = lib().sf_fp32_peak(int(device), ctypes.byref(a), ctypes.byref(b))
    if st != SF_OK:
        raise SfError(st, lib().sf_fp32_peak_error().decode(errors="replace"))
    return a.value, b.value


def words_to_bits(words, nz: int) -> np.ndarray:
    """Unpack a packed mask (any integer dtype holding uint32 words) to bool [nx][ny][nz]."""
    w = np.asarray(words).view(np.uint32) if np.asarray(words).dtype == np.int32 else \
        np.asarray(words, dtype=np.uint32)
    bits = (w[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    nx, ny, nw = w.shape
    return bits.reshape(nx, ny, nw * 32)[:, :, :nz].astype(bool)
