"""The row-strip partition (the paper's workers, two messages each) on the
host: partition, border summaries, the link solve and both exchanges, with
each strip computed by the oracle; single process with 1-6 strips and gloo
ranks (world sizes 2 and 3), checked bit for bit against the oracle on the
whole grid."""
import os
import socket
import sys

import numpy as np
import pytest
import torch

import demgen
import oracle
from paper_1605_05773_gb300 import strips
from tests.strip_oracle_backend import OracleStrips

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition():
    assert strips.partition(10, 3) == [(0, 3), (3, 6), (6, 10)]  # the last strip takes the rest
    assert strips.partition(5, 5) == [(k, k + 1) for k in range(5)]
    with pytest.raises(ValueError):
        strips.partition(3, 4)


def test_summary_record_round_trip():
    s = strips.Summary(6, np.array([0, 1]), np.array([2, 5]), np.array([3, 4]), np.array([7, 9], dtype=np.uint64),
                       np.arange(6), np.arange(6)[::-1].copy())
    t = strips.Summary.unpack(s.pack(), 6)
    for a, b in zip((s.exit_side, s.exit_col, s.exit_target, s.exit_value, s.top_exit, s.bottom_exit),
                    (t.exit_side, t.exit_col, t.exit_target, t.exit_value, t.top_exit, t.bottom_exit)):
        np.testing.assert_array_equal(a, b)


CASES = [("fractal", (130, 97)), ("fractal", (61, 200)), ("serpentine", (90, 70)), ("plane", (80, 66))]


def _dem(kind, shape):
    H, W = shape
    if kind == "fractal":
        return demgen.fractal(H, W, seed=H + W, cache=False)
    if kind == "plane":
        return demgen.plane(H, W, seed=5, cache=False)
    return demgen.serpentine_dem(H, W)


@pytest.mark.parametrize("rule", ["steepest", "lowest"])
@pytest.mark.parametrize("nstrips", [1, 2, 3, 6])
@pytest.mark.parametrize("case", CASES)
def test_strips_one_process_match_the_oracle(case, nstrips, rule):
    z = _dem(*case)
    d, A = strips.flowdir_accumulate_strips(z, nstrips, rule, backend=OracleStrips(rule), device="cpu")
    d_ref = oracle.flowdir(z, rule)
    np.testing.assert_array_equal(d, d_ref)
    np.testing.assert_array_equal(A, oracle.accumulate(d_ref))


def test_one_row_strips():
    z = demgen.fractal(7, 40, seed=3, cache=False)
    d, A = strips.flowdir_accumulate_strips(z, 7, backend=OracleStrips(), device="cpu")
    d_ref = oracle.flowdir(z)
    np.testing.assert_array_equal(d, d_ref)
    np.testing.assert_array_equal(A, oracle.accumulate(d_ref))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, kind, shape, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z = _dem(kind, shape)  # every rank makes the same grid and keeps its own rows
        r0, r1 = strips.partition(z.shape[0], world)[rank]
        d, A = strips.distributed_flowdir_accumulate(torch.from_numpy(z[r0:r1].copy()), z.shape[0], rank, world,
                                                     backend=OracleStrips())
        out.put((rank, d.numpy(), A.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", [("serpentine", (90, 70)), ("fractal", (130, 97))])
def test_strips_gloo_ranks_match_the_oracle(world, case):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, case[0], case[1], q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(world):
        rank, d, A = q.get(timeout=180)
        got[rank] = (d, A)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    z = _dem(*case)
    d_ref = oracle.flowdir(z)
    A_ref = oracle.accumulate(d_ref)
    for rank, (r0, r1) in enumerate(strips.partition(z.shape[0], world)):
        np.testing.assert_array_equal(got[rank][0], d_ref[r0:r1])
        np.testing.assert_array_equal(got[rank][1], A_ref[r0:r1])
