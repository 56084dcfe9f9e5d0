"""GB300-native D8 flow directions and up-slope area.

Barnes, Lehman, Mulla, "Distributed Parallel D8 Up-Slope Area Calculation in
Digital Elevation Models" (PDPTA 2011).

This package is a thin binding over the C ABI of ``libd8.so`` (declared in
``include/d8.h``).  It allocates output tensors with PyTorch, checks dtypes and
layouts, and passes raw device pointers, leading dimensions and the current
CUDA stream to the library.  All computation happens in the library's CUDA
kernels; there is no CPU path and no fallback: if the library is missing the
calls raise.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import torch

from . import build as _build

__all__ = [
    "load", "fill", "flowdir", "flowdir_strip", "accumulate", "accumulate_inflow", "set_strategy", "STRATEGIES", "flowdir_accumulate", "accumulate_weighted", "accumulate_backward",
    "weighted_upslope", "WeightedUpslope", "BatchPlan", "autotune_batch", "shape_class", "get_status", "set_tile", "set_profiling",
    "stage_times", "combine_stats", "D8Error", "OUTLET", "SINK", "RULES",
]

OUTLET, SINK = 8, 9
# direction rules; the "_nodata" forms treat non-finite elevations as cells
# outside the study area (OUTLET, as are the cells next to them)
RULES = {"steepest": 0, "lowest": 1, "steepest_nodata": 2, "lowest_nodata": 3}
# in-tile frontier strategies of the unit-count tile passes (identical results)
STRATEGIES = {"ring": 0, "lane_mask": 1, "jump": 2}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_SHAPE", 3: "ERR_NONFINITE", 4: "ERR_CYCLE", 5: "ERR_NOMEM",
          6: "ERR_CUDA", 7: "ERR_TIMEOUT", 8: "ERR_CAPACITY"}

_lib = None
_lock = threading.Lock()
_ctx: dict[int, ctypes.c_void_p] = {}
_tile: int = 64
_strategy: int = 0
_profiling: bool = False


class D8Error(RuntimeError):
    def __init__(self, code: int, what: str):
        name = STATUS.get(code, str(code))
        text = _lib.d8_status_string(code).decode() if _lib is not None else name
        super().__init__(f"{what}: {name} ({text})")
        self.code = code
        self.name = name


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libd8.so from the package's build folder (build it first with
    ``python -m paper_1605_05773_gb300.build`` or ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libd8 is not built ({path} missing); run python -m paper_1605_05773_gb300.build")
        L = ctypes.CDLL(path)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sigs = {
            "d8_create": [ctypes.POINTER(vp), i32],
            "d8_destroy": [vp],
            "d8_set_tile": [vp, i32],
            "d8_set_strategy": [vp, i32],
            "d8_flowdir": [vp, vp, i64, i64, i64, vp, i64, i32, vp],
            "d8_accumulate": [vp, vp, i64, i64, i64, vp, i64, vp],
            "d8_flowdir_accumulate": [vp, vp, i64, i64, i64, i32, vp, i64, vp, i64, vp],
            "d8_flowdir_strip": [vp, vp, i64, i64, i64, i32, i32, vp, i64, vp],
            "d8_accumulate_inflow": [vp, vp, i64, i64, i64, vp, vp, vp, i64, vp],
            "d8_accumulate_weighted": [vp, vp, i64, i64, i64, vp, i64, vp, i64, vp],
            "d8_accumulate_backward": [vp, vp, i64, i64, i64, vp, i64, vp, i64, vp],
            "d8_batch_plan": [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(vp)],
            "d8_batch_flowdir_accumulate": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i32, vp],
            "d8_batch_destroy": [vp],
            "d8_batch_autotune": [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(vp),
                                  ctypes.POINTER(vp), ctypes.POINTER(vp), i32, vp, ctypes.POINTER(i32),
                                  ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float)],
            "d8_get_status": [vp, vp],
            "d8_fill": [vp, vp, i64, i64, i64, ctypes.c_float, vp, i64, ctypes.POINTER(i64), vp],
            "d8_combine_stats": [vp, vp, ctypes.POINTER(i64), i32],
            "d8_set_profiling": [vp, i32],
            "d8_stage_times": [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i64), i32, ctypes.POINTER(i32)],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = i32
        L.d8_status_string.argtypes = [i32]
        L.d8_status_string.restype = ctypes.c_char_p
        L.d8_stage_name.argtypes = [i32]
        L.d8_stage_name.restype = ctypes.c_char_p
        L.d8_version.argtypes = []
        L.d8_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise D8Error(rc, what)


def context(device=None) -> ctypes.c_void_p:
    """The library context of a CUDA device (created on first use)."""
    L = load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    if idx not in _ctx:
        h = ctypes.c_void_p()
        _check(L.d8_create(ctypes.byref(h), idx), "d8_create")
        _check(L.d8_set_tile(h, _tile), "d8_set_tile")
        _check(L.d8_set_strategy(h, _strategy), "d8_set_strategy")
        L.d8_set_profiling(h, 1 if _profiling else 0)
        _ctx[idx] = h
    return _ctx[idx]


def set_tile(tile: int, device=None):
    """Tile side (32, 64 or 128) used by later calls."""
    global _tile
    _tile = int(tile)
    _check(load().d8_set_tile(context(device), _tile), "d8_set_tile")


def set_strategy(strategy, device=None):
    """Frontier strategy for later calls: "ring" (0, the default: chain walks
    fed from a per-warp ring in the tiles, queue walk at the combine's top
    level), "lane_mask" (1: the tiles' walks fed from per-thread source
    masks) or "jump" (2: ring walks in the tiles, pointer jumping at the top
    level, for DEMs whose channels cross tile borders very many times).
    Counts are identical; weighted sums may differ in the last bits."""
    global _strategy
    _strategy = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
    _check(load().d8_set_strategy(context(device), _strategy), "d8_set_strategy")


def set_profiling(on: bool, device=None):
    global _profiling
    _profiling = bool(on)
    _check(load().d8_set_profiling(context(device), 1 if on else 0), "d8_set_profiling")


def stage_times(device=None) -> dict:
    """{stage: (milliseconds, kernel launches)} since the last call (resets)."""
    L = load()
    ms = (ctypes.c_float * 16)()
    nl = (ctypes.c_int64 * 16)()
    n = ctypes.c_int()
    _check(L.d8_stage_times(context(device), ms, nl, 16, ctypes.byref(n)), "d8_stage_times")
    return {L.d8_stage_name(s).decode(): (float(ms[s]), int(nl[s])) for s in range(n.value)}


def _stream(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _grid(t: torch.Tensor, dtype: torch.dtype, name: str) -> tuple[int, int, int]:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != 2 or t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        raise ValueError(f"{name} must be a 2-D row-major tensor with unit column stride")
    return t.shape[0], t.shape[1], t.stride(0)


def _same_shape(a, b, names):
    if tuple(a.shape) != tuple(b.shape):
        raise ValueError(f"{names}: shapes differ {tuple(a.shape)} vs {tuple(b.shape)}")


def flowdir(z: torch.Tensor, rule: str = "steepest", out: torch.Tensor | None = None) -> torch.Tensor:
    """D8 direction codes (uint8) of an fp32 DEM."""
    H, W, ldz = _grid(z, torch.float32, "z")
    d = torch.empty((H, W), dtype=torch.uint8, device=z.device) if out is None else out
    _, _, ldd = _grid(d, torch.uint8, "out")
    _check(load().d8_flowdir(context(z.device), z.data_ptr(), H, W, ldz, d.data_ptr(), ldd, RULES[rule], _stream(z)),
           "d8_flowdir")
    return d


def fill(z: torch.Tensor, eps: float = 1e-3, out: torch.Tensor | None = None, return_rounds: bool = False):
    """Pit and flat removal by epsilon filling (d8_fill): every interior cell
    of the result has a strictly lower neighbour.  Synchronises the stream."""
    H, W, ldz = _grid(z, torch.float32, "z")
    F = torch.empty((H, W), dtype=torch.float32, device=z.device) if out is None else out
    _, _, ldf = _grid(F, torch.float32, "out")
    _same_shape(z, F, "z/out")
    r = ctypes.c_int64()
    _check(load().d8_fill(context(z.device), z.data_ptr(), H, W, ldz, float(eps), F.data_ptr(), ldf,
                          ctypes.byref(r), _stream(z)), "d8_fill")
    return (F, r.value) if return_rounds else F


def accumulate(dir: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """Unit up-slope counts (uint32) of a direction field."""
    H, W, ldd = _grid(dir, torch.uint8, "dir")
    A = torch.empty((H, W), dtype=torch.uint32, device=dir.device) if out is None else out
    _, _, lda = _grid(A, torch.uint32, "out")
    _same_shape(dir, A, "dir/out")
    _check(load().d8_accumulate(context(dir.device), dir.data_ptr(), H, W, ldd, A.data_ptr(), lda, _stream(dir)),
           "d8_accumulate")
    return A


def flowdir_strip(z: torch.Tensor, halo: int, rule: str = "steepest", out: torch.Tensor | None = None) -> torch.Tensor:
    """Directions of a horizontal strip of a taller grid (d8_flowdir_strip).
    z: a view of the strip's rows inside a larger row-major tensor; halo bit 0
    means the row above the view belongs to the grid (and is readable), bit 1
    the row below."""
    H, W, ldz = _grid(z, torch.float32, "z")
    d = torch.empty((H, W), dtype=torch.uint8, device=z.device) if out is None else out
    _, _, ldd = _grid(d, torch.uint8, "out")
    _same_shape(z, d, "z/out")
    _check(load().d8_flowdir_strip(context(z.device), z.data_ptr(), H, W, ldz, int(halo), RULES[rule], d.data_ptr(),
                                   ldd, _stream(z)), "d8_flowdir_strip")
    return d


def accumulate_inflow(dir: torch.Tensor, top_in: torch.Tensor | None, bottom_in: torch.Tensor | None,
                      out: torch.Tensor | None = None) -> torch.Tensor:
    """Unit counts with flow entering across the first and last rows
    (d8_accumulate_inflow): top_in[j] enters cell (0, j), bottom_in[j] cell
    (H-1, j); uint32 CUDA vectors of length W, or None."""
    H, W, ldd = _grid(dir, torch.uint8, "dir")
    A = torch.empty((H, W), dtype=torch.uint32, device=dir.device) if out is None else out
    _, _, lda = _grid(A, torch.uint32, "out")
    _same_shape(dir, A, "dir/out")
    ptrs = []
    for t, nm in ((top_in, "top_in"), (bottom_in, "bottom_in")):
        if t is None:
            ptrs.append(None)
            continue
        if not t.is_cuda or t.dtype != torch.uint32 or t.dim() != 1 or t.shape[0] != W or not t.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous CUDA uint32 vector of length {W}")
        ptrs.append(t.data_ptr())
    _check(load().d8_accumulate_inflow(context(dir.device), dir.data_ptr(), H, W, ldd, ptrs[0], ptrs[1],
                                       A.data_ptr(), lda, _stream(dir)), "d8_accumulate_inflow")
    return A


def flowdir_accumulate(z: torch.Tensor, rule: str = "steepest", dir: torch.Tensor | None = None,
                       A: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """Directions and unit counts in one fused pipeline."""
    H, W, ldz = _grid(z, torch.float32, "z")
    d = torch.empty((H, W), dtype=torch.uint8, device=z.device) if dir is None else dir
    A = torch.empty((H, W), dtype=torch.uint32, device=z.device) if A is None else A
    _, _, ldd = _grid(d, torch.uint8, "dir")
    _, _, lda = _grid(A, torch.uint32, "A")
    _same_shape(z, d, "z/dir")
    _same_shape(z, A, "z/A")
    _check(load().d8_flowdir_accumulate(context(z.device), z.data_ptr(), H, W, ldz, RULES[rule], d.data_ptr(), ldd,
                                        A.data_ptr(), lda, _stream(z)), "d8_flowdir_accumulate")
    return d, A


def accumulate_weighted(dir: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """Weighted up-slope area (fp32, compensated accumulation)."""
    H, W, ldd = _grid(dir, torch.uint8, "dir")
    _, _, ldw = _grid(w, torch.float32, "w")
    _same_shape(dir, w, "dir/w")
    A = torch.empty((H, W), dtype=torch.float32, device=dir.device) if out is None else out
    _, _, lda = _grid(A, torch.float32, "out")
    _check(load().d8_accumulate_weighted(context(dir.device), dir.data_ptr(), H, W, ldd, w.data_ptr(), ldw,
                                         A.data_ptr(), lda, _stream(dir)), "d8_accumulate_weighted")
    return A


def accumulate_backward(dir: torch.Tensor, dA: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """dL/dw from dL/dA: the sum of dA along each cell's flow path."""
    H, W, ldd = _grid(dir, torch.uint8, "dir")
    _, _, lda = _grid(dA, torch.float32, "dA")
    _same_shape(dir, dA, "dir/dA")
    dw = torch.empty((H, W), dtype=torch.float32, device=dir.device) if out is None else out
    _, _, ldw = _grid(dw, torch.float32, "out")
    _check(load().d8_accumulate_backward(context(dir.device), dir.data_ptr(), H, W, ldd, dA.data_ptr(), lda,
                                         dw.data_ptr(), ldw, _stream(dir)), "d8_accumulate_backward")
    return dw


class WeightedUpslope(torch.autograd.Function):
    """A = upslope(dir, w); the direction field gets no gradient."""

    @staticmethod
    def forward(ctx, dir, w):
        ctx.save_for_backward(dir)
        return accumulate_weighted(dir, w.contiguous())

    @staticmethod
    def backward(ctx, grad_A):
        (dir,) = ctx.saved_tensors
        return None, accumulate_backward(dir, grad_A.contiguous())


def weighted_upslope(dir: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    return WeightedUpslope.apply(dir, w)


def get_status(device=None, stream=None) -> str:
    """Synchronise, read and clear the device status word; 'OK' or the error name."""
    L = load()
    dev = device if device is not None else torch.cuda.current_device()
    s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
    rc = L.d8_get_status(context(dev), ctypes.c_void_p(s))
    return STATUS.get(rc, str(rc))


def combine_stats(device=None) -> dict:
    """Link-graph statistics of the last forward call's combine: group levels,
    top-level units, top-level exits and (strategy "jump") the pointer-jumping
    rounds that found work, which bound the graph's depth by 2^rounds."""
    L = load()
    dev = device if device is not None else torch.cuda.current_device()
    out = (ctypes.c_int64 * 4)()
    _check(L.d8_combine_stats(context(dev), ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream), out, 4),
           "d8_combine_stats")
    return {"group_levels": int(out[0]), "top_units": int(out[1]), "top_exits": int(out[2]),
            "top_jump_rounds": int(out[3]) if out[3] >= 0 else None}


def check_status(what: str = "device", device=None):
    st = get_status(device)
    if st != "OK":
        raise D8Error([k for k, v in STATUS.items() if v == st][0], what)


def _batch_buffers(shapes, zs, dirs, As, device):
    n = len(shapes)
    if len(zs) != n:
        raise ValueError("one elevation grid per planned DEM")
    dirs = dirs or [torch.empty(s, dtype=torch.uint8, device=device) for s in shapes]
    As = As or [torch.empty(s, dtype=torch.uint32, device=device) for s in shapes]
    for k, (z, d, a) in enumerate(zip(zs, dirs, As)):
        for t, dt, nm in ((z, torch.float32, "z"), (d, torch.uint8, "dir"), (a, torch.uint32, "A")):
            if tuple(t.shape) != shapes[k] or not t.is_contiguous() or t.dtype != dt or not t.is_cuda:
                raise ValueError(f"{nm}[{k}] must be a contiguous CUDA {dt} tensor of shape {shapes[k]}")
    vp = ctypes.c_void_p
    ptrs = tuple((vp * n)(*[t.data_ptr() for t in ts]) for ts in (zs, dirs, As))
    return dirs, As, ptrs


def shape_class(shapes) -> str:
    """Coarse class of a batch for the autotuner cache: the number of DEMs and
    the total and largest sizes, each rounded to a power of two."""
    cells = sum(h * w for h, w in shapes)
    side = max(max(h, w) for h, w in shapes)
    return f"n{len(shapes)}_cells2^{max(cells, 1).bit_length() - 1}_side2^{max(side, 1).bit_length() - 1}"


def _cache_key(device, shapes, rule) -> str:
    return f"{torch.cuda.get_device_name(device)}|{shape_class(shapes)}|{rule}"


def _read_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune_batch(zs, dirs=None, As=None, rule: str = "steepest", device=None, cache: str | None = None):
    """Pick the tile side and frontier strategy for a batch by timing the
    batched pipeline at every (tile, strategy) point (d8_batch_autotune).
    Sets them for later calls on this device and returns
    (tile, strategy name, {(tile, strategy name): median ms}).

    cache: optional path of a JSON file keyed by GPU name, the batch's shape
    class (shape_class) and the rule.  A hit sets the stored choice without
    timing anything (its timings dict is the stored one); a miss times and
    stores."""
    global _tile, _strategy
    L = load()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    shapes = [tuple(int(x) for x in z.shape) for z in zs]
    names = {v: k for k, v in STRATEGIES.items()}
    key = _cache_key(dev, shapes, rule)
    if cache is not None:
        hit = _read_cache(cache).get(key)
        if hit is not None:
            set_tile(int(hit["tile"]), dev)
            set_strategy(hit["strategy"], dev)
            timings = {(int(t), st): float(m) for t, st, m in hit.get("ms", [])}
            return int(hit["tile"]), hit["strategy"], timings
    n = len(shapes)
    dirs, As, (zp, dp, ap) = _batch_buffers(shapes, zs, dirs, As, dev)
    Hs = (ctypes.c_int64 * n)(*[h for h, _ in shapes])
    Ws = (ctypes.c_int64 * n)(*[w for _, w in shapes])
    best, best_s = ctypes.c_int(), ctypes.c_int()
    ms = (ctypes.c_float * 9)()
    _check(L.d8_batch_autotune(context(dev), n, Hs, Ws, zp, dp, ap, RULES[rule],
                               ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream), ctypes.byref(best),
                               ctypes.byref(best_s), ms),
           "d8_batch_autotune")
    _tile, _strategy = best.value, best_s.value
    timings = {(t, names[s]): float(ms[3 * k + s]) for k, t in enumerate((32, 64, 128)) for s in range(3)}
    if cache is not None:
        entries = _read_cache(cache)
        entries[key] = {"tile": best.value, "strategy": names[best_s.value],
                        "ms": [[t, st, m] for (t, st), m in timings.items()]}
        tmp = f"{cache}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(entries, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return best.value, names[best_s.value], timings


class BatchPlan:
    """Many DEMs in one pipeline: persistent launches over all tiles of all
    DEMs with a device tile work queue, replayed from a CUDA graph."""

    def __init__(self, shapes, device=None):
        L = load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.shapes = [(int(h), int(w)) for h, w in shapes]
        n = len(self.shapes)
        Hs = (ctypes.c_int64 * n)(*[h for h, _ in self.shapes])
        Ws = (ctypes.c_int64 * n)(*[w for _, w in self.shapes])
        self._h = ctypes.c_void_p()
        _check(L.d8_batch_plan(context(self.device), n, Hs, Ws, ctypes.byref(self._h)), "d8_batch_plan")

    def run(self, zs, dirs=None, As=None, rule: str = "steepest"):
        dirs, As, (zp, dp, ap) = _batch_buffers(self.shapes, zs, dirs, As, self.device)
        vp = ctypes.c_void_p
        _check(load().d8_batch_flowdir_accumulate(self._h, zp, dp, ap, RULES[rule],
                                                  vp(torch.cuda.current_stream(self.device).cuda_stream)),
               "d8_batch_flowdir_accumulate")
        return dirs, As

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().d8_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
