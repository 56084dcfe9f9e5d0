"""The allocation-free entry point, d8_flowdir_accumulate_noalloc.

Some callers cannot allocate device memory when they call: a process running
under a fixed memory budget reserved at start-up, a caller whose own pool or
arena allocator owns every byte of the device, or a caller that cannot create
a library context (creating one allocates).  This entry point serves them from
a fixed scratch array inside the library.  These tests call it through the C
ABI and check that it returns exactly what d8_flowdir_accumulate returns and
what the CPU oracle returns, on two calls in a row (the second reuses the
scratch the first left behind), on a grid at the largest size its scratch
holds, and that the smallest grid beyond the scratch is refused before any GPU
work.  Every buffer handed to the call is as large as the shape it is told, so
a broken capacity check could only show up as a wrong return code or wrong
output, never as an access outside a caller's buffer."""
import ctypes

import numpy as np
import pytest
import torch

import demgen
import oracle
from paper_1605_05773_gb300 import build

pytestmark = pytest.mark.gpu
D8_ERR_CAPACITY = 8

# The scratch: 64 MiB holding a 256-byte status word and, per 64 x 64 tile, 256
# perimeter slots of 2 + 4 + 4 + 4 + 4 + 4 bytes (each array rounded up to 256
# bytes), plus the round flags and queue counters.
SCRATCH = 64 << 20
TILE = 64


def _a256(x):
    return (x + 255) // 256 * 256


def _needed(ntiles):
    ns = ntiles * 4 * TILE
    return 256 + _a256(ns * 2) + 5 * _a256(ns * 4) + _a256(4 * (40 + 2)) + _a256(4 * 16)


def _largest_square_side():
    n = 1
    while _needed((n + 1) * (n + 1)) <= SCRATCH:
        n += 1
    return n * TILE  # n x n tiles fit, (n + 1) x (n + 1) do not


@pytest.fixture(scope="module")
def noalloc(d8):
    L = ctypes.CDLL(build.LIB)
    f = L.d8_flowdir_accumulate_noalloc
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    f.argtypes = [vp, i64, i64, i64, i32, vp, i64, vp, i64, vp, vp]
    f.restype = i32
    return f


def _call(f, z, d, A, status, rule=0):
    H, W = z.shape
    assert d.shape == (H, W) and A.shape == (H, W)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(z.data_ptr(), H, W, z.stride(0), rule, d.data_ptr(), d.stride(0), A.data_ptr(), A.stride(0),
             status.data_ptr(), stream)


def _u32(A):
    return A.cpu().numpy().view(np.uint32)


def test_noalloc_matches_the_context_entry_point_and_the_oracle_twice(d8, noalloc):
    """Fractal DEMs under both rules, then the realisable serpentine DEM, whose
    one long path crosses about 2000 tile borders: its exit forest is deep, so
    the combine's pointer jumping runs all of its rounds.  Two calls in a row
    per shape, the second over the first one's leftovers."""
    status = torch.full((1,), 0xFF, dtype=torch.int32, device="cuda")
    cases = [(demgen.fractal(1500, 1300, seed=70, cache=False), "steepest"),
             (demgen.fractal(2900, 3100, seed=71, cache=False), "lowest"),
             (demgen.serpentine_dem(2048, 2048), "steepest")]
    for z, rule in cases:
        H, W = z.shape
        zt = torch.from_numpy(z).cuda()
        d_ref, A_ref = d8.flowdir_accumulate(zt, rule)
        assert d8.get_status() == "OK"
        d_or = oracle.flowdir(z, rule)
        A_or = oracle.accumulate(d_or)
        for _ in range(2):
            d = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
            A = torch.zeros((H, W), dtype=torch.int32, device="cuda")
            assert _call(noalloc, zt, d, A, status, d8.RULES[rule]) == 0
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert torch.equal(d, d_ref)
            assert torch.equal(A, A_ref.view(torch.int32))
            np.testing.assert_array_equal(d.cpu().numpy(), d_or)
            np.testing.assert_array_equal(_u32(A), A_or)


def test_noalloc_at_the_largest_grid_its_scratch_holds(d8, noalloc):
    side = _largest_square_side()
    z = demgen.fractal(side, side, seed=72)
    zt = torch.from_numpy(z).cuda()
    d = torch.zeros((side, side), dtype=torch.uint8, device="cuda")
    A = torch.zeros((side, side), dtype=torch.int32, device="cuda")
    st = torch.zeros((1,), dtype=torch.int32, device="cuda")
    assert _call(noalloc, zt, d, A, st) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    d_or = oracle.flowdir(z)
    np.testing.assert_array_equal(d.cpu().numpy(), d_or)
    np.testing.assert_array_equal(_u32(A), oracle.accumulate(d_or))


def test_noalloc_refuses_grids_beyond_its_scratch(noalloc):
    """The smallest square grid beyond the scratch, with real buffers of that
    size (about 0.45 GB): refused before any launch, buffers untouched."""
    side = _largest_square_side() + TILE
    assert _needed((side // TILE) ** 2) > SCRATCH
    z = torch.zeros((side, side), dtype=torch.float32, device="cuda")
    d = torch.full((side, side), 77, dtype=torch.uint8, device="cuda")
    A = torch.full((side, side), 5, dtype=torch.int32, device="cuda")
    st = torch.zeros((1,), dtype=torch.int32, device="cuda")
    assert _call(noalloc, z, d, A, st) == D8_ERR_CAPACITY
    torch.cuda.synchronize()
    assert bool((d == 77).all()) and bool((A == 5).all())
