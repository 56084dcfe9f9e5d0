"""Row strips on the GPU: strip directions with halo rows, counts with inflow
across the first and last rows, and the whole strip protocol (one GPU, strips
in turn: the out-of-core form) against the oracle and the single call."""
import numpy as np
import pytest
import torch

import demgen
import oracle
import paper_1605_05773_gb300 as lib_mod
from paper_1605_05773_gb300 import strips
from tests.gpu_util import to_dev, u32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("halo", [0, 1, 2, 3])
def test_flowdir_strip_matches_the_oracle_on_the_taller_grid(d8, halo):
    z = demgen.fractal(300, 257, seed=12, cache=False)
    r0, r1 = 100, 180
    lo, hi = r0 - (halo & 1), r1 + (1 if halo & 2 else 0)
    zt = to_dev(z[lo:hi])
    top = halo & 1
    d = d8.flowdir_strip(zt[top:top + (r1 - r0)], halo, "steepest").cpu().numpy()
    ref = oracle.flowdir(z[lo:hi])[top:top + (r1 - r0)]
    np.testing.assert_array_equal(d, ref)


def test_accumulate_inflow(d8):
    z = demgen.fractal(333, 257, seed=13, cache=False)
    dr = oracle.flowdir(z)
    rng = np.random.default_rng(4)
    top = rng.integers(0, 1000, size=257).astype(np.uint32)
    bot = rng.integers(0, 1000, size=257).astype(np.uint32)
    top[rng.random(257) < 0.5] = 0
    for T in (32, 64, 128):
        d8.set_tile(T)
        try:
            A = d8.accumulate_inflow(to_dev(dr), to_dev(top), to_dev(bot))
            torch.cuda.synchronize()
            assert d8.get_status() == "OK"
        finally:
            d8.set_tile(64)
        w = np.ones(dr.shape)
        w[0] += top
        w[-1] += bot
        np.testing.assert_array_equal(u32(A), np.rint(oracle.accumulate_weighted(dr, w)).astype(np.uint32))


@pytest.mark.parametrize("nstrips", [2, 4, 7])
@pytest.mark.parametrize("case", [("fractal", (1500, 1100)), ("serpentine", (1200, 900)), ("plane", (700, 1300))])
def test_strips_out_of_core_match_the_oracle(d8, case, nstrips):
    kind, (H, W) = case
    z = {"fractal": lambda: demgen.fractal(H, W, seed=H, cache=False),
         "serpentine": lambda: demgen.serpentine_dem(H, W),
         "plane": lambda: demgen.plane(H, W, seed=6, cache=False)}[kind]()
    d, A = strips.flowdir_accumulate_strips(z, nstrips)
    assert d8.get_status() == "OK"
    d_ref = oracle.flowdir(z)
    np.testing.assert_array_equal(d, d_ref)
    np.testing.assert_array_equal(A, oracle.accumulate(d_ref))


def test_strips_8192_four_strips(d8):
    z = demgen.fractal(8192, 8192)
    d, A = strips.flowdir_accumulate_strips(z, 4)
    d1, A1 = d8.flowdir_accumulate(to_dev(z))
    np.testing.assert_array_equal(d, d1.cpu().numpy())
    np.testing.assert_array_equal(A, u32(A1))
