"""CPU oracle for D8 flow directions and up-slope area.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg are the only callers.  The product
(the CUDA library ``libd8`` and its binding) never imports this package.

The arithmetic lives in ``d8_oracle.c`` (plain sequential C, fp32 directions
without FMA contraction, exact uint64 counts, fp64 weighted sums); this module
only compiles it with gcc and marshals numpy arrays.  See the C file's header
for the passages of the paper each function follows and the readings used
where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "d8_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libd8oracle.so")
_lib = None

OK, ERR_ARG, ERR_NONFINITE, ERR_CYCLE, ERR_NOMEM, ERR_OVERFLOW = 0, 1, 3, 4, 5, 8
RULES = {"steepest": 0, "lowest": 1, "steepest_nodata": 2, "lowest_nodata": 3}
OUTLET, SINK = 8, 9


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    i64, vp = ctypes.c_int64, ctypes.c_void_p
    lib.oracle_flowdir.argtypes = [vp, i64, i64, ctypes.c_int, vp]
    lib.oracle_accumulate_f64.argtypes = [vp, i64, i64, vp, vp, vp]
    lib.oracle_accumulate_u64.argtypes = [vp, i64, i64, vp]
    lib.oracle_transposed_f64.argtypes = [vp, i64, i64, vp, vp]
    lib.oracle_fill_eps.argtypes = [vp, i64, i64, ctypes.c_float, vp]
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


class use_library:
    """Context manager that points this module at another build of the oracle
    source (used by the tests that plant a mistake in a copy of the oracle and
    check that the pins catch it)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _load()
        _lib = None
        lib = ctypes.CDLL(self.path)
        _lib = _configure(lib)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def flowdir(z: np.ndarray, rule: str = "steepest", allow_nonfinite: bool = False) -> np.ndarray:
    """D8 code per cell (0..7 = N,NE,E,SE,S,SW,W,NW; 8 OUTLET; 9 SINK)."""
    z = _c(z, np.float32)
    H, W = z.shape
    d = np.empty((H, W), dtype=np.uint8)
    rc = _load().oracle_flowdir(z.ctypes.data, H, W, RULES[rule], d.ctypes.data)
    if rc == ERR_NONFINITE and allow_nonfinite:
        return d
    if rc:
        raise OracleError(rc, "flowdir")
    return d


def accumulate(dir: np.ndarray) -> np.ndarray:
    """Unit-weight up-slope counts (Eq. 1, w = 1) as uint32 (exact)."""
    d = _c(dir, np.uint8)
    H, W = d.shape
    A = np.empty((H, W), dtype=np.uint64)
    rc = _load().oracle_accumulate_u64(d.ctypes.data, H, W, A.ctypes.data)
    if rc:
        raise OracleError(rc, "accumulate")
    return A.astype(np.uint32)


def accumulate_u64(dir: np.ndarray) -> np.ndarray:
    d = _c(dir, np.uint8)
    H, W = d.shape
    A = np.empty((H, W), dtype=np.uint64)
    rc = _load().oracle_accumulate_u64(d.ctypes.data, H, W, A.ctypes.data)
    if rc and rc != ERR_OVERFLOW:
        raise OracleError(rc, "accumulate")
    return A


def accumulate_weighted(dir: np.ndarray, w: np.ndarray | None) -> np.ndarray:
    """Weighted up-slope area A = w + sum of upstream A, in fp64."""
    d = _c(dir, np.uint8)
    H, W = d.shape
    A = np.empty((H, W), dtype=np.float64)
    wp = None
    if w is not None:
        w64 = _c(w, np.float64)
        assert w64.shape == (H, W)
        wp = w64.ctypes.data
    rc = _load().oracle_accumulate_f64(d.ctypes.data, H, W, wp, A.ctypes.data, None)
    if rc:
        raise OracleError(rc, "accumulate_weighted")
    return A


def finishing_order(dir: np.ndarray) -> np.ndarray:
    """Order in which the one-worker queue method finishes the cells."""
    d = _c(dir, np.uint8)
    H, W = d.shape
    A = np.empty((H, W), dtype=np.float64)
    order = np.empty(H * W, dtype=np.int64)
    rc = _load().oracle_accumulate_f64(d.ctypes.data, H, W, None, A.ctypes.data, order.ctypes.data)
    if rc:
        raise OracleError(rc, "finishing_order")
    return order


def transposed(dir: np.ndarray, c: np.ndarray) -> np.ndarray:
    """dL/dw for L = sum c*A: G(q) = c(q) + G(down-slope neighbour of q), fp64."""
    d = _c(dir, np.uint8)
    H, W = d.shape
    c64 = _c(c, np.float64)
    G = np.empty((H, W), dtype=np.float64)
    rc = _load().oracle_transposed_f64(d.ctypes.data, H, W, c64.ctypes.data, G.ctypes.data)
    if rc:
        raise OracleError(rc, "transposed")
    return G


def fill_eps(z: np.ndarray, eps: float = 1e-3) -> np.ndarray:
    """Pit and flat removal by epsilon filling (priority flood from the edge):
    the unique surface with F = z on the edge and, inside, F(c) = z(c) where z
    is above the lowest neighbouring F, else that F raised by eps (at least
    one fp32 step).  float32 in and out."""
    z = _c(z, np.float32)
    H, W = z.shape
    F = np.empty((H, W), dtype=np.float32)
    rc = _load().oracle_fill_eps(z.ctypes.data, H, W, np.float32(eps), F.ctypes.data)
    if rc:
        raise OracleError(rc, "fill_eps")
    return F
