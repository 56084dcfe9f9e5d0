"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Directions and unit counts must match bit for bit; every case runs at the
three tile sizes where it is cheap, over shapes that span several tiles and
leave ragged tails."""
import numpy as np
import pytest
import torch

import demgen
import oracle
from tests import brute, oracle_cache
from tests.gpu_util import recursion_residual_gpu, spiral_dirs, terminal_sum_gpu, to_dev, u32

pytestmark = pytest.mark.gpu
TILES = (32, 64, 128)
RULES = ("steepest", "lowest")


@pytest.fixture(params=TILES)
def tile(request, d8):
    d8.set_tile(request.param)
    yield request.param
    d8.set_tile(64)


def _fused(d8, z, rule):
    d, A = d8.flowdir_accumulate(to_dev(z), rule)
    torch.cuda.synchronize()
    assert d8.get_status() == "OK"
    return d.cpu().numpy(), u32(A)


@pytest.mark.parametrize("rule", RULES)
def test_512_fractal_fused(d8, tile, rule):
    """512x512 pit-free fractal, unit weights: dirs + counts bit-exact."""
    z = demgen.fractal(512, 512)
    d, A = _fused(d8, z, rule)
    d_ref = oracle.flowdir(z, rule)
    np.testing.assert_array_equal(d, d_ref)
    np.testing.assert_array_equal(A, oracle.accumulate(d_ref))


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 3), (5, 130), (130, 5), (33, 31),
                                   (65, 65), (129, 257), (333, 517)])
def test_ragged_and_degenerate_shapes(d8, tile, shape):
    H, W = shape
    z = demgen.fractal(H, W, seed=H * 1000 + W, cache=False)
    for rule in RULES:
        d, A = _fused(d8, z, rule)
        d_ref = oracle.flowdir(z, rule)
        np.testing.assert_array_equal(d, d_ref)
        np.testing.assert_array_equal(A, oracle.accumulate(d_ref))
        sd = d8.flowdir(to_dev(z), rule).cpu().numpy()
        np.testing.assert_array_equal(sd, d_ref)


def test_strided_inputs(d8):
    """Leading dimensions larger than the width (views into wider buffers)."""
    z = demgen.fractal(200, 300, seed=5, cache=False)
    big = torch.zeros((200, 333), dtype=torch.float32, device="cuda")
    big[:, :300] = to_dev(z)
    zv = big[:, :300]
    dbuf = torch.zeros((200, 320), dtype=torch.uint8, device="cuda")
    Abuf = torch.zeros((200, 301), dtype=torch.uint32, device="cuda")
    d8.flowdir_accumulate(zv, "steepest", dir=dbuf[:, :300], A=Abuf[:, :300])
    d_ref = oracle.flowdir(z)
    np.testing.assert_array_equal(dbuf[:, :300].cpu().numpy(), d_ref)
    np.testing.assert_array_equal(u32(Abuf)[:, :300], oracle.accumulate(d_ref))
    assert (dbuf[:, 300:] == 0).all() and (u32(Abuf)[:, 300:] == 0).all()


@pytest.mark.parametrize("shape", [(64, 64), (97, 131), (200, 45)])
def test_accumulate_fields(d8, tile, shape):
    """Direction fields given directly: serpentine, spiral, planes, random
    acyclic fields with terminals and off-grid targets."""
    H, W = shape
    fields = [demgen.serpentine_dirs(H, W), spiral_dirs(H, W)]
    rng = np.random.default_rng(H + W)
    for _ in range(3):
        fields.append(rng.choice(np.array([2, 3, 4, 5, 8, 9], dtype=np.uint8), size=(H, W),
                                 p=[.2, .2, .3, .2, .05, .05]))
    fields.append(oracle.flowdir(demgen.plane(H, W, seed=3, cache=False)))
    for f in fields:
        A = d8.accumulate(to_dev(f))
        torch.cuda.synchronize()
        assert d8.get_status() == "OK"
        np.testing.assert_array_equal(u32(A), oracle.accumulate(f))


def test_figure1_paths_small_tiles(d8):
    """Hand-checked tile-border cases with 32x32 tiles: a path that stays in
    its tile (A), enters from a neighbour and ends (B), loops back across the
    same border (C), and passes through from one neighbour to another (D)."""
    d8.set_tile(32)
    try:
        H, W = 96, 96
        d = np.full((H, W), 9, dtype=np.uint8)
        # A: inside tile (0,0): row 5, cols 3..10 east, ends at a sink
        d[5, 3:10] = 2
        # B: starts in tile (0,1) at row 10 col 40, goes west into tile (0,0) and ends
        d[10, 25:41] = 6
        # C: starts in tile (1,0) row 40 col 20, east across the border into tile (1,1)
        #    to col 35, south one row, back west into tile (1,0) to col 25
        d[40, 20:35] = 2
        d[40, 35] = 4
        d[41, 26:36] = 6
        # D: from tile (2,0) east through tile (2,1) into tile (2,2)
        d[70, 10:80] = 2
        A = d8.accumulate(to_dev(d))
        got = u32(A)
        np.testing.assert_array_equal(got, oracle.accumulate(d))
        np.testing.assert_array_equal(got, brute.counts(d).astype(np.uint32))
        assert got[5, 10] == 8 and got[10, 24] == 17 and got[41, 25] == 27 and got[70, 80] == 71
    finally:
        d8.set_tile(64)


@pytest.mark.parametrize("strategy", ["ring", "lane_mask", "jump"])
def test_strategies_bit_exact(d8, strategy):
    """Every frontier strategy gives the oracle's counts: fractal DEMs under
    both rules (ragged shapes, and one large enough for a top level above the
    512-cell groups), serpentine and spiral fields (one chain through many
    tiles), and random acyclic fields with terminals, at every tile side."""
    d8.set_strategy(strategy)
    try:
        for T in TILES:
            d8.set_tile(T)
            for H, W, seed in ((512, 512, 1605), (333, 517, 7), (130, 65, 8)):
                z = demgen.fractal(H, W, seed=seed, cache=False)
                for rule in RULES:
                    d, A = _fused(d8, z, rule)
                    d_ref = oracle.flowdir(z, rule)
                    np.testing.assert_array_equal(d, d_ref)
                    np.testing.assert_array_equal(A, oracle.accumulate(d_ref))
            z = demgen.fractal(1500, 1100, seed=9, cache=False)  # big enough for a top level above 512
            d, A = _fused(d8, z, "steepest")
            d_ref = oracle.flowdir(z)
            np.testing.assert_array_equal(d, d_ref)
            np.testing.assert_array_equal(A, oracle.accumulate(d_ref))
            rng = np.random.default_rng(T)
            fields = [demgen.serpentine_dirs(200, 190), spiral_dirs(150, 170),
                      rng.choice(np.array([2, 3, 4, 5, 8, 9], dtype=np.uint8), size=(257, 129),
                                 p=[.2, .2, .3, .2, .05, .05]),
                      demgen.serpentine_dirs(1300, 1100), spiral_dirs(1200, 1000)]
            for f in fields:
                A = d8.accumulate(to_dev(f))
                torch.cuda.synchronize()
                assert d8.get_status() == "OK"
                np.testing.assert_array_equal(u32(A), oracle.accumulate(f))
    finally:
        d8.set_tile(64)
        d8.set_strategy("ring")


def test_tile_size_invariance(d8):
    z = demgen.fractal(700, 555, seed=77, cache=False)
    outs = []
    for T in TILES:
        d8.set_tile(T)
        outs.append(_fused(d8, z, "steepest"))
    d8.set_tile(64)
    for d, A in outs[1:]:
        np.testing.assert_array_equal(d, outs[0][0])
        np.testing.assert_array_equal(A, outs[0][1])


def test_device_errors(d8):
    z = demgen.fractal(100, 90, seed=9, cache=False)
    z[50, 40] = np.nan
    d, A = d8.flowdir_accumulate(to_dev(z))
    assert d8.get_status() == "ERR_NONFINITE"
    assert d.cpu().numpy()[50, 40] == d8.SINK
    assert d8.get_status() == "OK"  # reading clears it
    cyc = np.full((40, 50), 8, dtype=np.uint8)
    cyc[10, 10], cyc[10, 11] = 2, 6
    d8.accumulate(to_dev(cyc))
    assert d8.get_status() == "ERR_CYCLE"
    # a cycle that spans several tiles (only the combine can see it)
    d8.set_tile(32)
    try:
        big = np.full((96, 96), 8, dtype=np.uint8)
        big[10, 10:60] = 2
        big[10, 60] = 4
        big[11, 11:61] = 6
        big[11, 10] = 0
        d8.accumulate(to_dev(big))
        assert d8.get_status() == "ERR_CYCLE"
    finally:
        d8.set_tile(64)
    bad = np.full((20, 20), 8, dtype=np.uint8)
    bad[5, 5] = 12
    d8.accumulate(to_dev(bad))
    assert d8.get_status() == "ERR_ARG"


def test_host_errors(d8):
    z = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        d8.flowdir(z.t())  # not row-major
    with pytest.raises(TypeError):
        d8.flowdir(z.double())
    with pytest.raises(KeyError):
        d8.flowdir(z, "nearest")


# ------------------------------------------------------------- full sizes
@pytest.fixture(scope="module")
def dem8192():
    return demgen.fractal(8192, 8192)


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("kind", ["fractal", "plane", "serpentine_dem"])
def test_8192_fused_full_oracle(d8, kind, rule, dem8192):
    """The three 8192^2 structures under both direction rules: directions and
    counts against the oracle at every cell."""
    z = {"fractal": lambda: dem8192, "plane": lambda: demgen.plane(8192, 8192),
         "serpentine_dem": lambda: demgen.serpentine_dem(8192, 8192)}[kind]()
    d, A = _fused(d8, z, rule)
    d_ref = oracle.flowdir(z, rule)
    np.testing.assert_array_equal(d, d_ref)
    np.testing.assert_array_equal(A, oracle.accumulate(d_ref))
    if kind == "serpentine_dem":
        assert A.max() > 8192 * 8192 // 2 - 8192 * 8  # one path of about H*W/2 cells


@pytest.mark.parametrize("strategy", ["ring", "jump"])
def test_8192_serpentine_dir_field(d8, strategy):
    """One boustrophedon path of 8192^2 cells (about 10^6 tile crossings), with
    the walks and with pointer jumping (every tile holds one 4096-cell chain)."""
    f = demgen.serpentine_dirs(8192, 8192)
    d8.set_strategy(strategy)
    try:
        A = u32(d8.accumulate(to_dev(f)))
    finally:
        d8.set_strategy("ring")
    assert d8.get_status() == "OK"
    np.testing.assert_array_equal(A, oracle.accumulate(f))
    assert A[8191, 0] == 8192 * 8192  # the last cell of the path (odd row ends at col 0)


@pytest.mark.parametrize("rule", RULES)
def test_32768_fused_full_oracle(d8, rule):
    """The headline 32768^2 fractal under both rules: directions and counts
    against the oracle at every one of its 1.07 G cells (the oracle's result
    is cached beside the DEM), plus the Eq. 1 recursion and conservation on
    the GPU result."""
    H = W = 32768
    z = demgen.fractal(H, W)
    d_ref, A_ref = oracle_cache.flowdir_accumulate(z, f"fractal_{H}x{W}_s{demgen.SEED_BASE}", rule)
    zt = to_dev(z)
    d, A = d8.flowdir_accumulate(zt, rule)
    torch.cuda.synchronize()
    assert d8.get_status() == "OK"
    del zt
    assert recursion_residual_gpu(d, A) == 0
    assert terminal_sum_gpu(d, A) == H * W
    np.testing.assert_array_equal(d.cpu().numpy(), d_ref)
    del d
    np.testing.assert_array_equal(u32(A), A_ref)


@pytest.mark.parametrize("rule", RULES)
def test_65536x16384_properties(d8, rule):
    """The anisotropic 16384 x 65536 fractal: directions against the oracle at
    every cell, counts by the Eq. 1 recursion at every cell plus conservation
    (together these fix the counts uniquely)."""
    H, W = 16384, 65536
    z = demgen.fractal(H, W)
    zt = to_dev(z)
    d, A = d8.flowdir_accumulate(zt, rule)
    torch.cuda.synchronize()
    assert d8.get_status() == "OK"
    del zt
    np.testing.assert_array_equal(d.cpu().numpy(), oracle.flowdir(z, rule))
    assert recursion_residual_gpu(d, A) == 0
    assert terminal_sum_gpu(d, A) == H * W


@pytest.mark.parametrize("rule", ["steepest_nodata", "lowest_nodata"])
@pytest.mark.parametrize("shape", [(97, 131), (512, 512), (1500, 1100)])
def test_nodata_masks(d8, tile, rule, shape):
    """NODATA masks: non-finite elevations (scattered holes, a lake, a band of
    NaN and +-inf along a ragged side) are cells outside the study area;
    directions and counts against the oracle, and no error raised."""
    H, W = shape
    z = demgen.fractal(H, W, seed=H + 3 * W, cache=False)
    rng = np.random.default_rng(H * W)
    z[rng.random(z.shape) < 0.02] = np.nan
    z[H // 3:H // 2, W // 4:W // 3] = np.nan
    z[:, W - 5:W - 2] = np.inf
    z[H - 7, :W // 2] = -np.inf
    d, A = _fused(d8, z, rule)
    d_ref = oracle.flowdir(z, rule)
    np.testing.assert_array_equal(d, d_ref)
    np.testing.assert_array_equal(A, oracle.accumulate(d_ref))
