"""Seeded synthetic inputs for the D8 up-slope-area tests and benchmark.

This module makes INPUTS only (elevations, direction patterns, weights,
cotangents, batch shapes).  It contains none of the method's arithmetic:
flow directions and up-slope areas are computed by the CUDA library under
test and, independently, by the CPU oracle.  Both sides receive what this
module produces.

Recipes (the paper names no dataset; these stand in for real DEMs):

* ``fractal``: diamond-square (roughness H=0.8) on a lattice of power-of-two
  squares, cropped, rescaled to 0..1000 m, then Priority-Flood+epsilon with
  eps=1e-3 m so every interior cell has a strictly lower neighbour and every
  descent path reaches the grid edge (the paper assumes pits and flats have
  been removed, "The Algorithm", first paragraph).
* ``plane``: z = 0.05*(H-1-i) + 0.02*(W-1-j) + 0.01 + U(-0.01, 0.01) m, then the
  same fill.
* ``serpentine_dirs``: a boustrophedon direction field, one path of H*W cells.
* ``serpentine_dem``: a realisable serpentine (channels on odd rows, ridges on
  even rows), one path of roughly H*W/2 cells.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "demgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdemgen.so")
_lib = None

EPS_FILL = 1e-3
ROUGHNESS = 0.8
RELIEF = 1000.0
SEED_BASE = 1605


def build(force: bool = False) -> str:
    """Compile the generator with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u64, vp, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double
        lib.demgen_fractal.argtypes = [vp, i64, i64, u64, dbl, dbl]
        lib.demgen_plane.argtypes = [vp, i64, i64, u64, dbl, dbl, dbl]
        lib.demgen_eps_fill.argtypes = [vp, i64, i64, ctypes.c_float]
        lib.demgen_count_undrained.argtypes = [vp, i64, i64]
        lib.demgen_count_undrained.restype = i64
        lib.demgen_serpentine_dirs.argtypes = [vp, i64, i64]
        lib.demgen_serpentine_dem.argtypes = [vp, i64, i64]
        lib.demgen_splitmix64_at.argtypes = [u64, u64]
        lib.demgen_splitmix64_at.restype = u64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def splitmix64_at(seed: int, n: int) -> int:
    return int(_load().demgen_splitmix64_at(seed, n))


def fractal_raw(H: int, W: int, seed: int) -> np.ndarray:
    """Diamond-square elevations rescaled to [0, RELIEF], before pit filling."""
    z = np.empty((H, W), dtype=np.float32)
    rc = _load().demgen_fractal(_ptr(z), H, W, seed, ROUGHNESS, RELIEF)
    if rc:
        raise RuntimeError(f"demgen_fractal failed ({rc})")
    return z


def eps_fill(z: np.ndarray, eps: float = EPS_FILL) -> np.ndarray:
    """Priority-Flood+epsilon in place on a C-contiguous float32 array."""
    assert z.dtype == np.float32 and z.flags.c_contiguous
    rc = _load().demgen_eps_fill(_ptr(z), z.shape[0], z.shape[1], eps)
    if rc:
        raise RuntimeError(f"demgen_eps_fill failed ({rc})")
    return z


def count_undrained(z: np.ndarray) -> int:
    z = np.ascontiguousarray(z, dtype=np.float32)
    return int(_load().demgen_count_undrained(_ptr(z), z.shape[0], z.shape[1]))


def _cache_dir() -> str:
    d = os.environ.get("D8_DEM_CACHE", os.path.join(tempfile.gettempdir(), "d8_dem_cache"))
    os.makedirs(d, exist_ok=True)
    return d


def _cached(key: str, make):
    """Cache large generated arrays as .npy files (keyed by recipe + source hash)."""
    with open(_SRC, "rb") as f:
        h = hashlib.sha1(f.read()).hexdigest()[:10]
    path = os.path.join(_cache_dir(), f"{key}_{h}.npy")
    if os.path.exists(path):
        try:
            return np.load(path, mmap_mode=None)
        except Exception:
            pass
    a = make()
    if a.size >= (1 << 22):
        tmp = path + f".tmp{os.getpid()}.npy"
        np.save(tmp, a)
        os.replace(tmp, path)
    return a


def fractal(H: int, W: int, seed: int = SEED_BASE, cache: bool = True) -> np.ndarray:
    """Pit-free fractal DEM (diamond-square + Priority-Flood+eps)."""

    def make():
        z = fractal_raw(H, W, seed)
        eps_fill(z)
        if H >= 3 and W >= 3:
            bad = count_undrained(z)
            if bad:
                raise RuntimeError(f"fractal {H}x{W} seed {seed}: {bad} undrained cells")
        return z

    return _cached(f"fractal_{H}x{W}_s{seed}", make) if cache else make()


def plane(H: int, W: int, seed: int = SEED_BASE + 1, cache: bool = True) -> np.ndarray:
    """Tilted plane draining S/E with +-0.01 m noise, then Priority-Flood+eps."""

    def make():
        z = np.empty((H, W), dtype=np.float32)
        rc = _load().demgen_plane(_ptr(z), H, W, seed, 0.05, 0.02, 0.01)
        if rc:
            raise RuntimeError("demgen_plane failed")
        eps_fill(z)
        return z

    return _cached(f"plane_{H}x{W}_s{seed}", make) if cache else make()


def plane_raw(H: int, W: int, seed: int = SEED_BASE + 1) -> np.ndarray:
    """The tilted plane with its +-0.01 m noise, before the fill (it has pits)."""
    z = np.empty((H, W), dtype=np.float32)
    rc = _load().demgen_plane(_ptr(z), H, W, seed, 0.05, 0.02, 0.01)
    if rc:
        raise RuntimeError("demgen_plane failed")
    return z


def plane_exact(H: int, W: int, sy: float = 1.0, sx: float = 0.0) -> np.ndarray:
    """Noise-free plane z = sy*(H-1-i) + sx*(W-1-j) (no fill)."""
    z = np.empty((H, W), dtype=np.float32)
    rc = _load().demgen_plane(_ptr(z), H, W, 0, sy, sx, 0.0)
    if rc:
        raise RuntimeError("demgen_plane failed")
    return z


def serpentine_dirs(H: int, W: int) -> np.ndarray:
    d = np.empty((H, W), dtype=np.uint8)
    if _load().demgen_serpentine_dirs(_ptr(d), H, W):
        raise RuntimeError("demgen_serpentine_dirs failed")
    return d


def serpentine_dem(H: int, W: int) -> np.ndarray:
    z = np.empty((H, W), dtype=np.float32)
    if _load().demgen_serpentine_dem(_ptr(z), H, W):
        raise RuntimeError("demgen_serpentine_dem failed")
    return z


def lognormal_weights(H: int, W: int, seed: int) -> np.ndarray:
    """Rainfall-like cell weights, lognormal(mu=0, sigma=1), float32."""
    return np.random.default_rng(seed).lognormal(0.0, 1.0, size=(H, W)).astype(np.float32)


def normal_cotangent(H: int, W: int, seed: int) -> np.ndarray:
    """Loss coefficients c ~ N(0, 1), float32 (L = sum c*A)."""
    return np.random.default_rng(seed).standard_normal(size=(H, W)).astype(np.float32)


def random_dirs(H: int, W: int, seed: int, codes: int = 10) -> np.ndarray:
    """Uniform random direction codes in [0, codes) (may contain cycles)."""
    return np.random.default_rng(seed).integers(0, codes, size=(H, W), dtype=np.uint8)


def batch_shapes(n: int = 512, seed: int = SEED_BASE + 3, lo: int = 128, hi: int = 4096,
                 max_aspect: float = 4.0):
    """Shapes of a batch of DEMs: long side log-uniform in [lo, hi], aspect
    log-uniform in [1, max_aspect], short side max(lo, round(L/r)), random
    orientation."""
    rng = np.random.default_rng(seed)
    L = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
    r = np.exp(rng.uniform(0.0, np.log(max_aspect), size=n))
    flip = rng.integers(0, 2, size=n)
    shapes = []
    for k in range(n):
        a = int(round(L[k]))
        b = max(lo, int(round(L[k] / r[k])))
        shapes.append((a, b) if flip[k] else (b, a))
    return shapes
