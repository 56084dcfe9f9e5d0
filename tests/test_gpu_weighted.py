"""Weighted up-slope area (compensated fp32) and its hand-written adjoint,
against the fp64 oracle, the transposed solve and central differences."""
import numpy as np
import pytest
import torch

import demgen
import oracle
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5  # max relative error against fp64


def grad_error(g32, d_ref, c):
    """|G32 - G64| / max(|G64|, sum over the path of |c|) (the scale-aware
    reading of the relative error for a signed gradient)."""
    G64 = oracle.transposed(d_ref, c.astype(np.float64))
    scale = np.maximum(np.abs(G64), oracle.transposed(d_ref, np.abs(c).astype(np.float64)))
    return (np.abs(g32.astype(np.float64) - G64) / scale).max(), G64


@pytest.mark.parametrize("T", [32, 64, 128])
@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (97, 131), (300, 257), (520, 130), (131, 300), (64, 1024)])
def test_weighted_and_backward_small(d8, T, shape):
    d8.set_tile(T)
    try:
        H, W = shape
        z = demgen.fractal(H, W, seed=H + 7 * W, cache=False)
        d_ref = oracle.flowdir(z)
        w = demgen.lognormal_weights(H, W, seed=1)
        c = demgen.normal_cotangent(H, W, seed=2)
        dt = to_dev(d_ref)
        A = d8.accumulate_weighted(dt, to_dev(w)).cpu().numpy()
        A64 = oracle.accumulate_weighted(d_ref, w.astype(np.float64))
        assert (np.abs(A - A64) / np.abs(A64)).max() <= TOL
        g = d8.accumulate_backward(dt, to_dev(c)).cpu().numpy()
        err, _ = grad_error(g, d_ref, c)
        assert err <= TOL
        assert d8.get_status() == "OK"
    finally:
        d8.set_tile(64)


def test_unit_weights_reproduce_counts(d8):
    z = demgen.fractal(400, 333, seed=3, cache=False)
    d_ref = oracle.flowdir(z)
    dt = to_dev(d_ref)
    A = d8.accumulate_weighted(dt, torch.ones((400, 333), device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(A, oracle.accumulate(d_ref).astype(np.float32))
    # c = 1: path lengths, exactly
    g = d8.accumulate_backward(dt, torch.ones((400, 333), device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(g, oracle.transposed(d_ref, np.ones((400, 333))).astype(np.float32))


def test_spiral_and_serpentine_weighted(d8):
    from tests.gpu_util import spiral_dirs

    for f in (spiral_dirs(150, 170), demgen.serpentine_dirs(130, 200)):
        H, W = f.shape
        w = demgen.lognormal_weights(H, W, seed=5)
        c = demgen.normal_cotangent(H, W, seed=6)
        A = d8.accumulate_weighted(to_dev(f), to_dev(w)).cpu().numpy()
        A64 = oracle.accumulate_weighted(f, w.astype(np.float64))
        assert (np.abs(A - A64) / np.abs(A64)).max() <= TOL
        g = d8.accumulate_backward(to_dev(f), to_dev(c)).cpu().numpy()
        assert grad_error(g, f, c)[0] <= TOL


def test_autograd_function_and_central_differences(d8):
    H, W = 256, 192
    z = demgen.fractal(H, W, seed=21, cache=False)
    d_ref = oracle.flowdir(z)
    w = demgen.lognormal_weights(H, W, seed=7)
    c = demgen.normal_cotangent(H, W, seed=8)
    wt = to_dev(w).requires_grad_(True)
    A = d8.weighted_upslope(to_dev(d_ref), wt)
    (A * to_dev(c)).sum().backward()
    g = wt.grad.cpu().numpy()
    err, G64 = grad_error(g, d_ref, c)
    assert err <= TOL
    # fp64 central differences of L(w) = sum c * A(w) (linear, so h = 1 is exact)
    rng = np.random.default_rng(9)
    w64, c64 = w.astype(np.float64), c.astype(np.float64)
    for q in rng.choice(H * W, size=64, replace=False):
        e = np.zeros(H * W)
        e[q] = 1.0
        e = e.reshape(H, W)
        fd = ((c64 * oracle.accumulate_weighted(d_ref, w64 + e)).sum() -
              (c64 * oracle.accumulate_weighted(d_ref, w64 - e)).sum()) / 2.0
        scale = max(abs(fd), oracle.transposed(d_ref, np.abs(c64)).ravel()[q])
        assert abs(g.ravel()[q] - fd) <= TOL * scale


def test_8192_weighted_forward_backward(d8):
    """8192^2 fractal, w ~ lognormal(0,1), L = sum c*A with c ~ N(0,1)."""
    H = W = 8192
    z = demgen.fractal(H, W)
    d_ref = oracle.flowdir(z)
    w = demgen.lognormal_weights(H, W, seed=11)
    c = demgen.normal_cotangent(H, W, seed=12)
    dt = to_dev(d_ref)
    A = d8.accumulate_weighted(dt, to_dev(w)).cpu().numpy()
    A64 = oracle.accumulate_weighted(d_ref, w.astype(np.float64))
    assert (np.abs(A - A64) / np.abs(A64)).max() <= TOL
    del A64
    g = d8.accumulate_backward(dt, to_dev(c)).cpu().numpy()
    err, G64 = grad_error(g, d_ref, c)
    assert err <= TOL
    # adjoint identity in fp64 on the GPU outputs: c.A(w) == G.w
    lhs = float((c.astype(np.float64) * A.astype(np.float64)).sum())
    rhs = float((g.astype(np.float64) * w.astype(np.float64)).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))
    assert d8.get_status() == "OK"


@pytest.mark.parametrize("strategy", ["ring", "jump"])
def test_weighted_top_level_strategies(d8, strategy):
    """Weighted areas through a top level above the 512-cell groups, solved by
    the queue walk and by pointer jumping (float-float sums added in another
    order): both within the bar against fp64, on a fractal DEM and on a
    serpentine field whose one chain crosses the top level's units."""
    d8.set_strategy(strategy)
    try:
        for f in (oracle.flowdir(demgen.fractal(1500, 1300, seed=31, cache=False)),
                  demgen.serpentine_dirs(1400, 1200)):
            H, W = f.shape
            w = demgen.lognormal_weights(H, W, seed=9)
            A = d8.accumulate_weighted(to_dev(f), to_dev(w)).cpu().numpy()
            assert d8.get_status() == "OK"
            A64 = oracle.accumulate_weighted(f, w.astype(np.float64))
            assert (np.abs(A - A64) / np.abs(A64)).max() <= TOL
    finally:
        d8.set_strategy("ring")


@pytest.mark.parametrize("T", [32, 64])
def test_backward_long_exit_chains(d8, T):
    """A serpentine field: one path through every cell, so the exit forest of
    the adjoint's combine is a single chain crossing tile borders tens of
    thousands of times (many pointer-jumping rounds).  With c = 1 the gradient
    is the path length, exact in fp32; with c ~ N(0, 1) within the bar."""
    d8.set_tile(T)
    try:
        f = demgen.serpentine_dirs(1536, 1024)
        H, W = f.shape
        g = d8.accumulate_backward(to_dev(f), torch.ones((H, W), device="cuda")).cpu().numpy()
        np.testing.assert_array_equal(g, oracle.transposed(f, np.ones((H, W))).astype(np.float32))
        c = demgen.normal_cotangent(H, W, seed=14)
        g = d8.accumulate_backward(to_dev(f), to_dev(c)).cpu().numpy()
        assert grad_error(g, f, c)[0] <= TOL
        assert d8.get_status() == "OK"
    finally:
        d8.set_tile(64)


@pytest.mark.parametrize("T", [32, 64])
def test_backward_reports_cycles(d8, T):
    """A 2-cycle inside a tile and a loop through two tiles (seen only by the
    combine) both end with ERR_CYCLE; a valid field afterwards is clean."""
    d8.set_tile(T)
    try:
        cyc = np.full((40, 50), 8, dtype=np.uint8)
        cyc[10, 10], cyc[10, 11] = 2, 6
        d8.accumulate_backward(to_dev(cyc), torch.ones((40, 50), device="cuda"))
        assert d8.get_status() == "ERR_CYCLE"
        big = np.full((96, 150), 8, dtype=np.uint8)
        big[10, 10:100] = 2
        big[10, 100] = 4
        big[11, 11:101] = 6
        big[11, 10] = 0
        d8.accumulate_backward(to_dev(big), torch.ones((96, 150), device="cuda"))
        assert d8.get_status() == "ERR_CYCLE"
        ok = np.full((96, 150), 8, dtype=np.uint8)
        ok[10, 10:100] = 2
        g = d8.accumulate_backward(to_dev(ok), torch.ones((96, 150), device="cuda")).cpu().numpy()
        assert d8.get_status() == "OK"
        np.testing.assert_array_equal(g, oracle.transposed(ok, np.ones((96, 150))).astype(np.float32))
    finally:
        d8.set_tile(64)


def test_weighted_wide_dynamic_range(d8):
    """Weights spanning eleven orders of magnitude: a band of huge weights
    upstream sends rivers of ~1e9 through tiles whose other receivers carry
    inflows near 1e-2.  The per-tile fixed-point finalise must keep those
    small inflows within the bar (its scale follows the tile's summed
    inflow, not only the largest)."""
    H, W = 1200, 1100
    z = demgen.fractal(H, W, seed=41, cache=False)
    d_ref = oracle.flowdir(z)
    w = demgen.lognormal_weights(H, W, seed=13) * np.float32(1e-2)
    hi = z > np.quantile(z, 0.9)  # the highest tenth of the DEM
    w[hi] *= np.float32(1e9)
    A = d8.accumulate_weighted(to_dev(d_ref), to_dev(w)).cpu().numpy()
    A64 = oracle.accumulate_weighted(d_ref, w.astype(np.float64))
    assert A64.max() / A64.min() > 1e10
    assert (np.abs(A - A64) / np.abs(A64)).max() <= TOL
    assert d8.get_status() == "OK"


@pytest.mark.parametrize("T", [32, 64])
def test_weighted_signed_weights(d8, T):
    """Weights of both signs (N(0, 1)), so inflows cancel along the paths and
    the finalise's fixed point carries negative values and borrows.  Error
    is measured against the scale of the terms, |A32 - A64| / (sum of |w|
    over the up-slope set), the reading used for signed gradients."""
    d8.set_tile(T)
    try:
        H, W = 1100, 1300
        d_ref = oracle.flowdir(demgen.fractal(H, W, seed=43, cache=False))
        w = demgen.normal_cotangent(H, W, seed=15)
        A = d8.accumulate_weighted(to_dev(d_ref), to_dev(w)).cpu().numpy()
        A64 = oracle.accumulate_weighted(d_ref, w.astype(np.float64))
        scale = oracle.accumulate_weighted(d_ref, np.abs(w).astype(np.float64))
        assert (np.abs(A.astype(np.float64) - A64) / scale).max() <= TOL
        assert d8.get_status() == "OK"
    finally:
        d8.set_tile(64)
