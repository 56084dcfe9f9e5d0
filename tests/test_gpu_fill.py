"""Pit and flat removal on the GPU (d8_fill) against the oracle's priority
flood, bit for bit: raw fractal DEMs (before the generator's own fill), the
noisy tilted plane, random noise fields full of pits and flats, ragged and
degenerate shapes, strided buffers, the hand-worked cases, and the filled
surface fed to the direction and accumulation pipeline."""
import numpy as np
import pytest
import torch

import demgen
import oracle
from tests.golden_io import grid, named
from tests.gpu_util import to_dev, u32

pytestmark = pytest.mark.gpu
EPS = 1e-3


def _fill(d8, z, eps=EPS):
    F, rounds = d8.fill(to_dev(z), eps, return_rounds=True)
    torch.cuda.synchronize()
    assert d8.get_status() == "OK"
    return F.cpu().numpy(), rounds


@pytest.mark.parametrize("shape", [(1, 1), (2, 7), (3, 3), (5, 130), (65, 65), (130, 257), (333, 517), (512, 512)])
def test_fill_fractal_and_noise(d8, shape):
    H, W = shape
    for z in (demgen.fractal_raw(H, W, seed=H + W), (np.random.default_rng(H * W).random((H, W)) * 7).astype(np.float32),
              np.random.default_rng(W).integers(0, 4, size=(H, W)).astype(np.float32)):
        F, _ = _fill(d8, z)
        np.testing.assert_array_equal(F, oracle.fill_eps(z, EPS))


def test_fill_golden_cases(d8):
    g = named("fill_cases.txt")
    for name in ("bowl", "plateau", "spill", "keep", "step"):
        rows = g[name]
        F, _ = _fill(d8, grid(rows[1:], np.float32), float(rows[0][0]))
        np.testing.assert_array_equal(F, grid(g[name + "_F"], np.float32), err_msg=name)


def test_fill_pit_free_input_is_unchanged(d8):
    z = demgen.fractal(1000, 700, seed=3, cache=False)  # already drains everywhere
    F, _ = _fill(d8, z)
    np.testing.assert_array_equal(F, z)


def test_fill_strided_and_errors(d8):
    z = demgen.fractal_raw(200, 300, seed=11)
    big = torch.zeros((200, 320), dtype=torch.float32, device="cuda")
    big[:, :300] = to_dev(z)
    out = torch.full((200, 333), -1.0, dtype=torch.float32, device="cuda")
    d8.fill(big[:, :300], EPS, out=out[:, :300])
    np.testing.assert_array_equal(out[:, :300].cpu().numpy(), oracle.fill_eps(z, EPS))
    assert bool((out[:, 300:] == -1.0).all())
    with pytest.raises(d8.D8Error):
        d8.fill(big, EPS, out=big)  # output overlapping the input
    bad = z.copy()
    bad[50, 60] = np.nan
    d8.fill(to_dev(bad), EPS)
    assert d8.get_status() == "ERR_NONFINITE"


def test_fill_8192_then_pipeline(d8):
    """The 8192^2 raw fractal and the noisy plane: the fill bit-exact against
    the oracle, then directions and counts on the filled surface (no SINK,
    counts against the oracle)."""
    for z in (demgen.fractal_raw(8192, 8192, demgen.SEED_BASE), demgen.plane_raw(8192, 8192)):
        F, rounds = _fill(d8, z)
        F_ref = oracle.fill_eps(z, EPS)
        np.testing.assert_array_equal(F, F_ref)
        assert rounds >= 1
        d, A = d8.flowdir_accumulate(to_dev(F))
        torch.cuda.synchronize()
        assert d8.get_status() == "OK"
        d = d.cpu().numpy()
        assert not (d == 9).any()
        np.testing.assert_array_equal(u32(A), oracle.accumulate(oracle.flowdir(F_ref)))
