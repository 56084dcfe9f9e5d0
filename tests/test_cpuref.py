"""The multi-core CPU reference (the benchmark's CPU baseline) gives the
oracle's directions and counts at any thread count."""
import numpy as np
import pytest

import cpuref
import demgen
import oracle
from tests.gpu_util import spiral_dirs


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_cpuref_matches_oracle(threads):
    cases = [demgen.fractal(300, 257, seed=41, cache=False), demgen.plane(200, 333, seed=42, cache=False),
             demgen.serpentine_dem(150, 130)]
    for z in cases:
        for rule in ("steepest", "lowest"):
            d = cpuref.flowdir(z, rule, threads)
            d_ref = oracle.flowdir(z, rule)
            np.testing.assert_array_equal(d, d_ref)
            np.testing.assert_array_equal(cpuref.accumulate(d, threads), oracle.accumulate(d_ref))
    rng = np.random.default_rng(threads)
    for f in (demgen.serpentine_dirs(120, 97), spiral_dirs(90, 110),
              rng.choice(np.array([2, 3, 4, 5, 8, 9], dtype=np.uint8), size=(130, 140))):
        np.testing.assert_array_equal(cpuref.accumulate(f, threads), oracle.accumulate(f))


def test_cpuref_reports_cycles_and_bad_codes():
    cyc = np.full((20, 30), 8, dtype=np.uint8)
    cyc[5, 5], cyc[5, 6] = 2, 6
    with pytest.raises(RuntimeError, match="error 4"):
        cpuref.accumulate(cyc, 4)
    bad = np.full((10, 10), 8, dtype=np.uint8)
    bad[3, 3] = 11
    with pytest.raises(RuntimeError, match="error 1"):
        cpuref.accumulate(bad, 2)
