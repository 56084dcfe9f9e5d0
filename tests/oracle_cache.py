"""Oracle results for the largest parity cases, cached beside the cached DEMs.

The oracle needs one to two minutes per rule at 32768^2, so its directions
and counts are kept as .npy files in the DEM cache folder (``$D8_DEM_CACHE``,
default ``<tmp>/d8_dem_cache``), keyed by the DEM's name, the rule and hashes
of the oracle and generator sources.  Every value in them is computed by
``oracle/`` from a DEM made by ``demgen/``; nothing comes from the CUDA path."""
from __future__ import annotations

import hashlib
import os

import numpy as np

import demgen
import oracle


def _key(name: str, rule: str) -> str:
    h = hashlib.sha1()
    for src in (oracle._SRC, demgen._SRC):
        with open(src, "rb") as f:
            h.update(f.read())
    return f"oracle_{name}_{rule}_{h.hexdigest()[:10]}"


def flowdir_accumulate(z: np.ndarray, name: str, rule: str):
    """(directions, uint32 counts) of the oracle for DEM `name`, from the cache
    when present, else computed and stored."""
    base = os.path.join(demgen._cache_dir(), _key(name, rule))
    pd, pa = base + "_dir.npy", base + "_A.npy"
    if os.path.exists(pd) and os.path.exists(pa):
        try:
            return np.load(pd), np.load(pa)
        except Exception:
            pass
    d = oracle.flowdir(z, rule)
    A = oracle.accumulate(d)
    try:
        for path, a in ((pd, d), (pa, A)):
            tmp = path + f".tmp{os.getpid()}.npy"
            np.save(tmp, a)
            os.replace(tmp, path)
    except OSError:
        pass
    return d, A
