"""FP64 CPU oracle for the Gaussian source-finder hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only users.
The CUDA library never imports or links this package, and this package never
imports the CUDA library.

The arithmetic lives in ``sf_oracle.c`` (plain FP64 loops, one function per
definition of the paper):

* taps: sampled Gaussian, truncated at ``R = ceil(truncation * sigma)``,
  normalised to sum 1 (Sec. 2.1 and Sec. 3.4; the paper gives no sigma or
  truncation, the filter bank is a parameter);
* filter: Eq. 2, zero outside the cube, 3D filter = outer product of the 1D
  taps (separable evaluation, plus the literal triple sum for spot checks);
* window statistics: population mean and standard deviation over
  non-overlapping windows from the origin (Sec. 3.3, statistics over a range of
  voxels around each voxel, read as the window holding it);
* threshold: ``c > mean + k * std`` (Sec. 3.3 z-score selection), OR over the
  bank, packed 32 consecutive z per uint32 word.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsforacle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile sf_oracle.c into oracle/_build/libsforacle.so (gcc, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.or_radius.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.or_radius.restype = ctypes.c_int
        lib.or_taps.argtypes = [ctypes.c_double, ctypes.c_int, _dp]
        lib.or_taps.restype = None
        lib.or_filter_box.argtypes = [_fp, _i64, _i64, _i64, _dp, ctypes.c_int, _dp,
                                      ctypes.c_int, _dp, ctypes.c_int, _i64, _i64, _i64,
                                      _i64, _i64, _i64, ctypes.c_int, _dp]
        lib.or_filter_box.restype = ctypes.c_int
        lib.or_filter_direct_voxel.argtypes = [_fp, _i64, _i64, _i64, _dp, ctypes.c_int,
                                               _dp, ctypes.c_int, _dp, ctypes.c_int,
                                               _i64, _i64, _i64]
        lib.or_filter_direct_voxel.restype = ctypes.c_double
        lib.or_moments.argtypes = [_dp, _i64, ctypes.c_int, _dp, _dp]
        lib.or_moments.restype = None
        lib.or_window_stats.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, _dp, _dp]
        lib.or_window_stats.restype = ctypes.c_int
        lib.or_threshold.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _dp, _dp, ctypes.c_double,
                                     ctypes.c_double, _u32p, _u32p]
        lib.or_threshold.restype = None
        lib.or_detect_window.argtypes = [_fp, _i64, _i64, _i64, ctypes.c_int, _ip, _dp, _ip,
                                         _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, _i64, _i64, _i64,
                                         _dp, _dp, _u8p, _u8p, _dp, _dp]
        lib.or_detect_window.restype = ctypes.c_int
        lib.or_detect.argtypes = [_fp, _i64, _i64, _i64, ctypes.c_int, _ip, _dp, _ip, _dp,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, _u32p, _u32p, _dp, _dp, ctypes.c_int]
        lib.or_detect.restype = ctypes.c_int
        lib.or_detect_windows.argtypes = [_fp, _i64, _i64, _i64, ctypes.c_int, _ip, _dp, _ip, _dp,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double,
                                          ctypes.c_double, _i64,
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
        lib.or_detect_windows.restype = ctypes.c_int
        lib.or_local_stats.argtypes = [_dp, _i64, _i64, _i64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), _i64, _dp,
                                       _dp, ctypes.c_int]
        lib.or_local_stats.restype = ctypes.c_int
        lib.or_weighted_filter_box.argtypes = [_fp, _fp, _i64, _i64, _i64, _dp, ctypes.c_int, _dp,
                                               ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _i64,
                                               _i64, _i64, _i64, _i64, _i64, _dp]
        lib.or_weighted_filter_box.restype = ctypes.c_int
        lib.or_weighted_direct_voxel.argtypes = [_fp, _fp, _i64, _i64, _i64, _dp, ctypes.c_int, _dp,
                                                 ctypes.c_int, _dp, ctypes.c_int, ctypes.c_int, _i64,
                                                 _i64, _i64]
        lib.or_weighted_direct_voxel.restype = ctypes.c_double
        _lib = lib
        return lib


def _ptr(a: np.ndarray, typ):
    return a.ctypes.data_as(typ)


def _cube(d) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(d), dtype=np.float32)
    if d.ndim != 3:
        raise ValueError("cube must be 3D [x][y][z]")
    return d


# ---------------------------------------------------------------- taps -------
def radius(sigma: float, truncation: float) -> int:
    """R = ceil(truncation * sigma); 0 when sigma <= 0."""
    return int(_load().or_radius(float(sigma), float(truncation)))


def taps(sigma: float, truncation: float) -> np.ndarray:
    """Normalised truncated Gaussian taps, length 2R+1, offset o at index o+R."""
    r = radius(sigma, truncation)
    g = np.empty(2 * r + 1, dtype=np.float64)
    _load().or_taps(float(sigma), r, _ptr(g, _dp))
    return g


# -------------------------------------------------------------- filter -------
def filter_box(d, sigma_xy: float, sigma_z: float, truncation: float,
               box=None, take_abs: bool = False) -> np.ndarray:
    """Eq. 2 filtered values (float64) on box ((x0,x1),(y0,y1),(z0,z1))."""
    d = _cube(d)
    nx, ny, nz = d.shape
    if box is None:
        box = ((0, nx), (0, ny), (0, nz))
    (x0, x1), (y0, y1), (z0, z1) = box
    gxy = taps(sigma_xy, truncation)
    gz = taps(sigma_z, truncation)
    rxy, rz = (len(gxy) - 1) // 2, (len(gz) - 1) // 2
    out = np.empty((x1 - x0, y1 - y0, z1 - z0), dtype=np.float64)
    rc = _load().or_filter_box(_ptr(d, _fp), nx, ny, nz, _ptr(gxy, _dp), rxy,
                               _ptr(gxy, _dp), rxy, _ptr(gz, _dp), rz,
                               x0, x1, y0, y1, z0, z1, int(take_abs), _ptr(out, _dp))
    if rc != 0:
        raise MemoryError("oracle filter_box: out of memory")
    return out


def filter_direct_voxel(d, sigma_xy: float, sigma_z: float, truncation: float,
                        x: int, y: int, z: int) -> float:
    """Eq. 2 as the literal triple sum at one voxel."""
    d = _cube(d)
    nx, ny, nz = d.shape
    gxy = taps(sigma_xy, truncation)
    gz = taps(sigma_z, truncation)
    rxy, rz = (len(gxy) - 1) // 2, (len(gz) - 1) // 2
    return float(_load().or_filter_direct_voxel(_ptr(d, _fp), nx, ny, nz, _ptr(gxy, _dp),
                                                rxy, _ptr(gxy, _dp), rxy, _ptr(gz, _dp),
                                                rz, x, y, z))


# --------------------------------------------------------------- stats -------
def moments(values, ddof: int = 0) -> tuple[float, float]:
    """Mean and std (squared deviations over n - ddof: 0 population, 1 sample)."""
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64).ravel())
    m = ctypes.c_double()
    s = ctypes.c_double()
    _load().or_moments(_ptr(v, _dp), v.size, int(ddof), ctypes.byref(m), ctypes.byref(s))
    return m.value, s.value


def window_grid(shape, window) -> tuple[int, int, int]:
    return tuple(-(-int(n) // int(w)) for n, w in zip(shape, window))


def window_stats(c, window, ddof: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Mean and std per window of a filtered cube, [nwx][nwy][nwz] (ddof 0:
    population std, 1: sample std)."""
    c = np.ascontiguousarray(np.asarray(c), dtype=np.float64)
    nx, ny, nz = c.shape
    wx, wy, wz = window
    grid = window_grid(c.shape, window)
    mean = np.empty(grid, dtype=np.float64)
    std = np.empty(grid, dtype=np.float64)
    if _load().or_window_stats(_ptr(c, _dp), nx, ny, nz, wx, wy, wz, int(ddof),
                               _ptr(mean, _dp), _ptr(std, _dp)) != 0:
        raise MemoryError("oracle window_stats: out of memory")
    return mean, std


def mask_words_shape(shape) -> tuple[int, int, int]:
    nx, ny, nz = shape
    return (nx, ny, -(-nz // 32))


def threshold(c, window, mean, std, k: float, band_rel: float = 1e-4):
    """Packed masks (fire, ambiguous) of c > mean + k*std per window."""
    c = np.ascontiguousarray(np.asarray(c), dtype=np.float64)
    nx, ny, nz = c.shape
    wx, wy, wz = window
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    std = np.ascontiguousarray(std, dtype=np.float64)
    mask = np.zeros(mask_words_shape(c.shape), dtype=np.uint32)
    amb = np.zeros_like(mask)
    _load().or_threshold(_ptr(c, _dp), nx, ny, nz, wx, wy, wz, _ptr(mean, _dp),
                         _ptr(std, _dp), float(k), float(band_rel), _ptr(mask, _u32p),
                         _ptr(amb, _u32p))
    return mask, amb


# -------------------------------------------------------------- detect -------
def _bank_arrays(bank, truncation):
    rxy, rz, gxy, gz = [], [], [], []
    for sxy, sz in bank:
        a = taps(sxy, truncation)
        b = taps(sz, truncation)
        rxy.append((len(a) - 1) // 2)
        rz.append((len(b) - 1) // 2)
        gxy.append(a)
        gz.append(b)
    return (np.array(rxy, dtype=np.int32), np.concatenate(gxy),
            np.array(rz, dtype=np.int32), np.concatenate(gz))


def detect_window(d, bank, truncation, window, k, widx, band_rel: float = 1e-4, ddof: int = 0):
    """Whole method on one window (a, b, e); returns a dict of float64/uint8 arrays.

    Keys: mean[f], std[f], thr[f], fire/sure [window voxels as x,y,z box], c[f][box].
    """
    d = _cube(d)
    nx, ny, nz = d.shape
    wx, wy, wz = window
    a, b, e = widx
    ex = min(wx, nx - a * wx)
    ey = min(wy, ny - b * wy)
    ez = min(wz, nz - e * wz)
    if ex <= 0 or ey <= 0 or ez <= 0:
        raise ValueError("window index outside the cube")
    nf = len(bank)
    rxy, gxy, rz, gz = _bank_arrays(bank, truncation)
    n = ex * ey * ez
    mean = np.empty(nf)
    std = np.empty(nf)
    thr = np.empty(nf)
    fire = np.empty(n, dtype=np.uint8)
    sure = np.empty(n, dtype=np.uint8)
    cv = np.empty((nf, n))
    rc = _load().or_detect_window(_ptr(d, _fp), nx, ny, nz, nf, _ptr(rxy, _ip), _ptr(gxy, _dp),
                                  _ptr(rz, _ip), _ptr(gz, _dp), wx, wy, wz, int(ddof), float(k),
                                  float(band_rel), a, b, e, _ptr(mean, _dp), _ptr(std, _dp),
                                  _ptr(fire, _u8p), _ptr(sure, _u8p), _ptr(cv, _dp),
                                  _ptr(thr, _dp))
    if rc != 0:
        raise MemoryError("oracle detect_window: out of memory")
    box = (ex, ey, ez)
    return {"mean": mean, "std": std, "thr": thr, "fire": fire.reshape(box),
            "sure": sure.reshape(box), "c": cv.reshape((nf,) + box),
            "origin": (a * wx, b * wy, e * wz)}


def detect(d, bank, truncation, window, k, band_rel: float = 1e-4, nthreads: int = 0,
           ddof: int = 0):
    """Whole method on the whole cube.

    Returns dict: mask, sure (packed uint32 [nx][ny][ceil(nz/32)]), mean, std
    ([nf][nwx][nwy][nwz]) and threads (OpenMP threads used).
    """
    d = _cube(d)
    nx, ny, nz = d.shape
    wx, wy, wz = window
    nf = len(bank)
    rxy, gxy, rz, gz = _bank_arrays(bank, truncation)
    grid = window_grid(d.shape, window)
    mask = np.zeros(mask_words_shape(d.shape), dtype=np.uint32)
    sure = np.zeros_like(mask)
    mean = np.empty((nf,) + grid)
    std = np.empty((nf,) + grid)
    used = _load().or_detect(_ptr(d, _fp), nx, ny, nz, nf, _ptr(rxy, _ip), _ptr(gxy, _dp),
                             _ptr(rz, _ip), _ptr(gz, _dp), wx, wy, wz, int(ddof), float(k),
                             float(band_rel), _ptr(mask, _u32p), _ptr(sure, _u32p),
                             _ptr(mean, _dp), _ptr(std, _dp), int(nthreads))
    if used < 0:
        raise MemoryError("oracle detect: out of memory")
    return {"mask": mask, "sure": sure, "mean": mean, "std": std, "threads": used}


def detect_windows(d, bank, truncation, window, k, widx, band_rel: float = 1e-4,
                   nthreads: int = 0, ddof: int = 0):
    """Whole method on a list of windows (n x 3 indices), in parallel.

    Returns (fired voxels per window, OpenMP threads used).
    """
    d = _cube(d)
    nx, ny, nz = d.shape
    wx, wy, wz = window
    rxy, gxy, rz, gz = _bank_arrays(bank, truncation)
    idx = np.ascontiguousarray(np.asarray(widx, dtype=np.int64).reshape(-1, 3))
    fired = np.zeros(idx.shape[0], dtype=np.int64)
    used = _load().or_detect_windows(_ptr(d, _fp), nx, ny, nz, len(bank), _ptr(rxy, _ip),
                                     _ptr(gxy, _dp), _ptr(rz, _ip), _ptr(gz, _dp), wx, wy, wz,
                                     int(ddof), float(k), float(band_rel), idx.shape[0],
                                     _ptr(idx, ctypes.POINTER(ctypes.c_int64)),
                                     _ptr(fired, ctypes.POINTER(ctypes.c_int64)), int(nthreads))
    if used < 0:
        raise MemoryError("oracle detect_windows: out of memory")
    return fired, used


def pack_bits(bits) -> np.ndarray:
    """Pack a boolean [nx][ny][nz] array into the mask word layout (bit z%32)."""
    bits = np.asarray(bits, dtype=bool)
    nx, ny, nz = bits.shape
    nw = -(-nz // 32)
    padded = np.zeros((nx, ny, nw * 32), dtype=np.uint64)
    padded[:, :, :nz] = bits
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    words = (padded.reshape(nx, ny, nw, 32) * weights).sum(axis=-1)
    return words.astype(np.uint32)


def unpack_bits(words, nz: int) -> np.ndarray:
    """Inverse of pack_bits: packed words -> boolean [nx][ny][nz]."""
    words = np.asarray(words, dtype=np.uint32)
    bits = (words[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    nx, ny, nw = words.shape
    return bits.reshape(nx, ny, nw * 32)[:, :, :nz].astype(bool)


# ------------------------------------------------- per-voxel local statistics
def local_stats(c, half, idx=None, nthreads: int = 0, ddof: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Mean and population std of the filtered cube c over the box of
    half-widths half = (sx, sy, sz) around each voxel, clipped to the cube
    (Sec. 3.3).  idx: flat voxel indices to evaluate (default: all voxels,
    returned with c's shape)."""
    c = np.ascontiguousarray(np.asarray(c), dtype=np.float64)
    nx, ny, nz = c.shape
    sx, sy, sz = (int(v) for v in half)
    if min(sx, sy, sz) < 0:
        raise ValueError("half-widths must be >= 0")
    if idx is None:
        mean = np.empty(c.shape, dtype=np.float64)
        std = np.empty(c.shape, dtype=np.float64)
        _load().or_local_stats(_ptr(c, _dp), nx, ny, nz, sx, sy, sz, int(ddof), None, 0,
                               _ptr(mean, _dp), _ptr(std, _dp), int(nthreads))
        return mean, std
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).ravel())
    mean = np.empty(idx.shape, dtype=np.float64)
    std = np.empty(idx.shape, dtype=np.float64)
    _load().or_local_stats(_ptr(c, _dp), nx, ny, nz, sx, sy, sz, int(ddof),
                           _ptr(idx, ctypes.POINTER(ctypes.c_int64)), idx.size,
                           _ptr(mean, _dp), _ptr(std, _dp), int(nthreads))
    return mean, std


def local_zscore(c, half, idx=None, ddof: int = 0) -> np.ndarray:
    """Per-voxel z-score (c - mean) / std over the clipped box of half-widths
    half (Sec. 3.3, the statistics the voxel selection tests against), 0
    where std = 0.  idx: flat voxel indices (default: every voxel)."""
    c = np.ascontiguousarray(np.asarray(c), dtype=np.float64)
    mean, std = local_stats(c, half, idx, ddof=ddof)
    cv = c if idx is None else c.ravel()[np.asarray(idx, dtype=np.int64).ravel()]
    z = np.zeros_like(mean)
    ok = std > 0
    z[ok] = (cv[ok] - mean[ok]) / std[ok]
    return z


def local_detect(d, bank, truncation, half, k, band_rel: float = 1e-4, voxels=None, ddof: int = 0):
    """The sliding-statistics form of the method (Sec. 3.3 read per voxel):
    every filter of the bank (Eq. 2), the local mean/std of each filtered cube
    over the box `half` around the voxel, c_f > mean_f + k std_f, OR over the
    bank.  voxels: (x, y, z) triples to evaluate (default: the whole cube).

    Returns (fire, sure, c, mean, std): fire / sure as uint8 per evaluated
    voxel (sure = the OR cannot flip with rounding: no filter within
    band_rel * std of its threshold unless another fires by more), and the
    per-filter filtered values and statistics [nf][n]."""
    d = _cube(d)
    nx, ny, nz = d.shape
    sx, sy, sz = (int(v) for v in half)
    if voxels is None:
        xs, ys, zs = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        voxels = np.stack([xs.ravel(), ys.ravel(), zs.ravel()], axis=1)
    voxels = np.asarray(voxels, dtype=np.int64).reshape(-1, 3)
    nv = voxels.shape[0]
    nf = len(bank)
    cv = np.empty((nf, nv))
    mv = np.empty((nf, nv))
    sv = np.empty((nf, nv))
    for f, (sxy, szz) in enumerate(bank):
        if nv > 64:
            c = filter_box(d, sxy, szz, truncation)
            flat = (voxels[:, 0] * ny + voxels[:, 1]) * nz + voxels[:, 2]
            mv[f], sv[f] = local_stats(c, (sx, sy, sz), flat, ddof=ddof)
            cv[f] = c.ravel()[flat]
        else:
            for i, (x, y, z) in enumerate(voxels):
                box = ((max(0, x - sx), min(nx, x + sx + 1)), (max(0, y - sy), min(ny, y + sy + 1)),
                       (max(0, z - sz), min(nz, z + sz + 1)))
                c = filter_box(d, sxy, szz, truncation, box)
                lx, ly, lz = x - box[0][0], y - box[1][0], z - box[2][0]
                m, s_ = local_stats(c, (sx, sy, sz), [(lx * c.shape[1] + ly) * c.shape[2] + lz],
                                    ddof=ddof)
                mv[f, i], sv[f, i] = m[0], s_[0]
                cv[f, i] = c[lx, ly, lz]
    thr = mv + k * sv
    fire_f = cv > thr
    near = np.abs(cv - thr) < band_rel * sv
    fire = fire_f.any(axis=0)
    clear = (fire_f & ~near).any(axis=0)
    sure = clear | ~near.any(axis=0)
    return fire.astype(np.uint8), sure.astype(np.uint8), cv, mv, sv


# ------------------------------------------------- weighted convolution (Eq. 1)
DEN_MODES = {"fw": 0, "w": 1}


def weighted_filter_box(d, w, sigma_xy: float, sigma_z: float, truncation: float, den: str = "fw",
                        box=None) -> np.ndarray:
    """Eq. 1 on box ((x0,x1),(y0,y1),(z0,z1)) (float64): sum d f w / D with
    D = sum f w (den="fw", normalised convolution) or D = sum w (den="w", as
    printed); 0 where D = 0."""
    d = _cube(d)
    w = _cube(w)
    if d.shape != w.shape:
        raise ValueError("cube and weights must have the same shape")
    nx, ny, nz = d.shape
    if box is None:
        box = ((0, nx), (0, ny), (0, nz))
    (x0, x1), (y0, y1), (z0, z1) = box
    gxy = taps(sigma_xy, truncation)
    gz = taps(sigma_z, truncation)
    rxy, rz = (len(gxy) - 1) // 2, (len(gz) - 1) // 2
    out = np.empty((x1 - x0, y1 - y0, z1 - z0), dtype=np.float64)
    rc = _load().or_weighted_filter_box(_ptr(d, _fp), _ptr(w, _fp), nx, ny, nz, _ptr(gxy, _dp), rxy,
                                        _ptr(gxy, _dp), rxy, _ptr(gz, _dp), rz, DEN_MODES[den],
                                        x0, x1, y0, y1, z0, z1, _ptr(out, _dp))
    if rc != 0:
        raise MemoryError("oracle weighted_filter_box: out of memory")
    return out


def weighted_direct_voxel(d, w, sigma_xy: float, sigma_z: float, truncation: float, x: int, y: int,
                          z: int, den: str = "fw") -> float:
    """Eq. 1 as the literal triple sums at one voxel."""
    d = _cube(d)
    w = _cube(w)
    nx, ny, nz = d.shape
    gxy = taps(sigma_xy, truncation)
    gz = taps(sigma_z, truncation)
    rxy, rz = (len(gxy) - 1) // 2, (len(gz) - 1) // 2
    return float(_load().or_weighted_direct_voxel(_ptr(d, _fp), _ptr(w, _fp), nx, ny, nz,
                                                  _ptr(gxy, _dp), rxy, _ptr(gxy, _dp), rxy,
                                                  _ptr(gz, _dp), rz, DEN_MODES[den], x, y, z))


def weighted_detect(d, w, bank, truncation, window, k, den: str = "fw", band_rel: float = 1e-4,
                    ddof: int = 0):
    """The method with Eq. 1 filtering: every filter of the bank weighted by w,
    window statistics (Sec. 3.3), c > mean + k std, OR over the bank.
    Returns dict(mask, sure (packed words), mean, std [nf][nwx][nwy][nwz])."""
    d = _cube(d)
    nf = len(bank)
    grid = window_grid(d.shape, window)
    mask = np.zeros(mask_words_shape(d.shape), dtype=np.uint32)
    means = np.empty((nf,) + grid)
    stds = np.empty((nf,) + grid)
    fire = np.zeros(d.shape, dtype=bool)
    clear = np.zeros(d.shape, dtype=bool)
    near_any = np.zeros(d.shape, dtype=bool)
    for f, (sxy, sz) in enumerate(bank):
        c = weighted_filter_box(d, w, sxy, sz, truncation, den)
        m, s = window_stats(c, window, ddof=ddof)
        means[f], stds[f] = m, s
        wi = [np.arange(n) // wn for n, wn in zip(d.shape, window)]
        mb = m[np.ix_(*wi)]
        sb = s[np.ix_(*wi)]
        thr = mb + k * sb
        ff = c > thr
        near = np.abs(c - thr) < band_rel * sb
        fire |= ff
        clear |= ff & ~near
        near_any |= near
    sure = clear | ~near_any
    return {"mask": pack_bits(fire), "sure": pack_bits(sure), "mean": means, "std": stds}
