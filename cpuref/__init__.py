"""Multi-core CPU reference (OpenMP direction pass + the paper's shared-memory
queue method with one queue per thread): the CPU baseline beside the GPU.

MEASUREMENT INFRASTRUCTURE ONLY: the benchmark's CPU-baseline leg and the
tests (which check it against the oracle) are its only callers.  The code is
in ``d8_cpuref.c``; this module compiles it with gcc and marshals arrays."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d8_cpuref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libd8cpuref.so")
_lib = None
RULES = {"steepest": 0, "lowest": 1}


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, vp, i32 = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
        lib.cpuref_flowdir.argtypes = [vp, i64, i64, i32, i32, vp]
        lib.cpuref_accumulate.argtypes = [vp, i64, i64, i32, vp]
        _lib = lib
    return _lib


def cores() -> int:
    """Threads the reference uses by default: the cores this process may run on."""
    return len(os.sched_getaffinity(0))


def flowdir(z: np.ndarray, rule: str = "steepest", threads: int | None = None) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float32)
    H, W = z.shape
    d = np.empty((H, W), dtype=np.uint8)
    rc = _load().cpuref_flowdir(z.ctypes.data, H, W, RULES[rule], threads or cores(), d.ctypes.data)
    if rc not in (0, 3):
        raise RuntimeError(f"cpuref_flowdir: error {rc}")
    return d


def accumulate(dir: np.ndarray, threads: int | None = None) -> np.ndarray:
    d = np.ascontiguousarray(dir, dtype=np.uint8)
    H, W = d.shape
    A = np.empty((H, W), dtype=np.uint32)
    rc = _load().cpuref_accumulate(d.ctypes.data, H, W, threads or cores(), A.ctypes.data)
    if rc:
        raise RuntimeError(f"cpuref_accumulate: error {rc}")
    return A
