"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
max-over-ranks timing reduction, the barrier, and the reference arm under
torchrun (rank 0 alone prints one JSON line; the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        m = bench.max_over_ranks(1.5 + rank, world)  # each rank's "elapsed ms"
        out.put((rank, m))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]  # both ranks see the slowest rank's time


def test_reference_arm_under_torchrun_prints_one_line():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "fractal_512", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["e2e"]["h2d_bytes_per_step"] == 0



def test_measured_traffic_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    """bench.py quotes ncu traffic only while the kernel's source still has the
    hash recorded with the capture."""
    import hashlib

    sys.path.insert(0, ROOT)
    import bench

    src_dir = tmp_path / "paper_1605_05773_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src_dir / "d8_unit.cu").write_text("// kernel v1\n")
    (src_dir / "d8_flowdir.cu").write_text("// stencil v1\n")
    sha = hashlib.sha1(b"// kernel v1\n").hexdigest()[:12]
    (tmp_path / bench.TRAFFIC_FILE).write_text(json.dumps({
        "kernel_source": {"tile_up": "d8_unit.cu", "flowdir": "d8_flowdir.cu"},
        "kernel_source_sha1": {"d8_unit.cu": sha, "d8_flowdir.cu": "000000000000"},
        "dram_bytes_per_cell": {"tile_up": 4.48, "flowdir": 4.79}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("tile_up") == 4.48
    assert bench.measured_traffic("flowdir") is None  # hash differs: stale capture
    (src_dir / "d8_unit.cu").write_text("// kernel v2\n")
    assert bench.measured_traffic("tile_up") is None


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))


def test_unknown_extras_are_refused():
    """bench.py --extras names the extra lines to add; a misspelt name is an
    argument error (before any GPU work), not a silently skipped line."""
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--extras", "fwd_bwd,fil"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2
    assert "unknown extras" in r.stderr and "fil" in r.stderr
