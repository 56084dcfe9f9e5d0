"""Batched pipeline: many DEMs of uneven sizes through one persistent launch
per stage (tile work queue), replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

import demgen
import oracle
from tests.gpu_util import recursion_residual_gpu, terminal_sum_gpu, to_dev, u32

pytestmark = pytest.mark.gpu


def test_small_batch_bit_exact_and_replay(d8):
    shapes = [(1, 1), (3, 7), (64, 64), (65, 129), (300, 257), (128, 512), (700, 130), (31, 33), (256, 256)]
    zs = [demgen.fractal(h, w, seed=100 + k, cache=False) for k, (h, w) in enumerate(shapes)]
    plan = d8.BatchPlan(shapes)
    zt = [to_dev(z) for z in zs]
    for rule in ("steepest", "lowest", "steepest"):
        dirs, As = plan.run(zt, rule=rule)
        torch.cuda.synchronize()
        assert d8.get_status() == "OK"
        for z, d, A in zip(zs, dirs, As):
            d_ref = oracle.flowdir(z, rule)
            np.testing.assert_array_equal(d.cpu().numpy(), d_ref)
            np.testing.assert_array_equal(u32(A), oracle.accumulate(d_ref))
    # replay into fresh output buffers (new pointers, same graph)
    dirs2 = [torch.empty(s, dtype=torch.uint8, device="cuda") for s in shapes]
    As2 = [torch.empty(s, dtype=torch.uint32, device="cuda") for s in shapes]
    plan.run(zt, dirs2, As2)
    for A, A2 in zip(As, As2):
        assert torch.equal(A.view(torch.int32), A2.view(torch.int32))
    plan.close()


def test_batch_512_dems(d8):
    """The 512-DEM configuration: sides log-uniform in [128, 4096], aspect up to
    1:4.  Every DEM is checked by the Eq. 1 recursion and conservation; every
    16th also against the oracle cell by cell."""
    shapes = demgen.batch_shapes(512)
    zs = [demgen.fractal(h, w, seed=2000 + k) for k, (h, w) in enumerate(shapes)]
    plan = d8.BatchPlan(shapes)
    zt = [to_dev(z) for z in zs]
    dirs, As = plan.run(zt)
    torch.cuda.synchronize()
    assert d8.get_status() == "OK"
    for k, (z, d, A) in enumerate(zip(zs, dirs, As)):
        assert recursion_residual_gpu(d, A) == 0, k
        assert terminal_sum_gpu(d, A) == z.size, k
        if k % 16 == 0:
            d_ref = oracle.flowdir(z)
            np.testing.assert_array_equal(d.cpu().numpy(), d_ref)
            np.testing.assert_array_equal(u32(A), oracle.accumulate(d_ref))
    plan.close()


def test_autotune_picks_a_tile_and_strategy_and_keeps_results_exact(d8, tmp_path):
    """The autotuner times the batch at every (tile side, strategy) point,
    leaves the fastest set, stores it in its cache (a second call reads the
    cache and times nothing), and the chosen pair produces the oracle's
    results.  The batch holds a serpentine field's DEM version too, so the
    chain-heavy case is among the inputs."""
    shapes = [(200, 300), (513, 129), (64, 64), (1000, 257), (129, 700)]
    zs = [demgen.fractal(h, w, seed=300 + k, cache=False) for k, (h, w) in enumerate(shapes)]
    zs.append(demgen.serpentine_dem(1200, 700))
    shapes.append((1200, 700))
    zt = [to_dev(z) for z in zs]
    cache = str(tmp_path / "autotune.json")
    try:
        tile, strat, ms = d8.autotune_batch(zt, cache=cache)
        assert tile in (32, 64, 128) and strat in d8.STRATEGIES
        assert set(ms) == {(t, s) for t in (32, 64, 128) for s in d8.STRATEGIES}
        assert all(v > 0 for v in ms.values())
        assert ms[(tile, strat)] == min(ms.values())
        tile2, strat2, ms2 = d8.autotune_batch(zt, cache=cache)  # a cache hit
        assert (tile2, strat2) == (tile, strat) and ms2 == ms
        plan = d8.BatchPlan(shapes)
        dirs, As = plan.run(zt)
        torch.cuda.synchronize()
        assert d8.get_status() == "OK"
        for z, d, A in zip(zs, dirs, As):
            d_ref = oracle.flowdir(z)
            np.testing.assert_array_equal(d.cpu().numpy(), d_ref)
            np.testing.assert_array_equal(u32(A), oracle.accumulate(d_ref))
        plan.close()
    finally:
        d8.set_tile(64)
        d8.set_strategy("ring")
