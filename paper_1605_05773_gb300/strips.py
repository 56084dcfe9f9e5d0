"""Row strips of a grid: the paper's partition across processes, and the same
partition on one GPU for grids larger than its memory.

Barnes, Lehman, Mulla ("The Algorithm"): the grid is cut into strips of
consecutive rows, one per worker, the last taking the rows left over; each
worker finds the internal up-slope area of its strip with the inflow from
its neighbours unknown (Algorithms 1-4), sends one message to the master with
its border summary, the master resolves the links between strips
(Algorithms 5-6) and replies with the inflow entering each border cell, and
each worker finishes its strip (Algorithms 7-8): two messages per worker.

Here a worker is a GPU (one strip per rank, the summaries exchanged with one
all-gather so that every rank solves the links itself and the reply needs no
message) or a turn of one GPU (`flowdir_accumulate_strips`: strips in turn,
the grid on the host, one strip on the device at a time).  Per strip:

  1. directions with the rows above and below as halo (d8_flowdir_strip) and
     local counts (d8_accumulate on the strip alone: a path leaving the strip
     ends there; its last cell is one of the strip's exits);
  2. the border summary: the exits (cells of the first or last row whose
     direction leaves the strip; their column, target column and local
     count) and, for every cell of the first and last row, the exit its path
     in the strip reaches: the adjoint (d8_accumulate_backward) with each
     exit's number as its cotangent gives every cell the number of the exit on
     its path (a sum with one non-zero term, exact in fp32), or 0;
  3. the link solve (`solve_links`, on the host: the links are two rows per
     strip): an exit's parent is the exit reached, in the neighbouring strip,
     by the cell it drains into; F(x) = local count + sum of F over children;
     the inflow into a border cell is the sum of F over the exits draining into
     it;
  4. the final counts (d8_accumulate_inflow with those inflows).

Every per-strip step runs in the library's kernels; the compute backend is a
parameter only so that a host test can drive the partition, the exchange and
the link solve with strips computed another way.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import accumulate, accumulate_backward, accumulate_inflow, flowdir_strip

# codes 0..7: N, NE, E, SE, S, SW, W, NW; those leaving a strip upwards / downwards
_DJ = np.array([0, 1, 1, 1, 0, -1, -1, -1])
_UP = (0, 1, 7)
_DOWN = (3, 4, 5)


def partition(H: int, n: int) -> list[tuple[int, int]]:
    """Row ranges of n strips: H // n rows each, the last taking the rest."""
    if n < 1 or n > H:
        raise ValueError(f"cannot cut {H} rows into {n} strips")
    base = H // n
    return [(k * base, (k + 1) * base if k < n - 1 else H) for k in range(n)]


class GpuStrips:
    """Per-strip compute in the library's kernels (CUDA tensors)."""

    def __init__(self, rule: str = "steepest"):
        self.rule = rule

    def directions(self, z_ext: torch.Tensor, halo: int) -> torch.Tensor:
        top = halo & 1
        h = z_ext.shape[0] - top - ((halo >> 1) & 1)
        return flowdir_strip(z_ext[top:top + h], halo, self.rule)

    def local_counts(self, dir: torch.Tensor) -> torch.Tensor:
        return accumulate(dir)

    def exit_numbers(self, dir: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
        return accumulate_backward(dir, c)

    def final_counts(self, dir: torch.Tensor, top_in, bottom_in) -> torch.Tensor:
        return accumulate_inflow(dir, top_in, bottom_in)


@dataclass
class Summary:
    """The border summary of one strip (message 1)."""
    W: int
    exit_side: np.ndarray    # 0: leaves through the top, 1: through the bottom
    exit_col: np.ndarray     # column of the exit cell
    exit_target: np.ndarray  # column of the cell it drains into, in the neighbouring strip
    exit_value: np.ndarray   # local count at the exit (uint64)
    top_exit: np.ndarray     # per column of the first row: number of the exit its path reaches, 0 = none
    bottom_exit: np.ndarray  # the same for the last row

    def pack(self) -> np.ndarray:
        """Fixed-size int64 record for an all-gather: [n, 4 x 2W exit fields, W, W]."""
        W = self.W
        out = np.zeros(1 + 8 * W + 2 * W, dtype=np.int64)
        n = len(self.exit_col)
        out[0] = n
        for k, a in enumerate((self.exit_side, self.exit_col, self.exit_target, self.exit_value)):
            out[1 + 2 * W * k:1 + 2 * W * k + n] = a
        out[1 + 8 * W:1 + 9 * W] = self.top_exit
        out[1 + 9 * W:] = self.bottom_exit
        return out

    @staticmethod
    def unpack(rec: np.ndarray, W: int) -> "Summary":
        n = int(rec[0])
        f = [rec[1 + 2 * W * k:1 + 2 * W * k + n].copy() for k in range(4)]
        return Summary(W, f[0], f[1], f[2], f[3].astype(np.uint64), rec[1 + 8 * W:1 + 9 * W].copy(),
                       rec[1 + 9 * W:].copy())


def summarise(backend, dir: torch.Tensor, A_loc: torch.Tensor, halo: int) -> Summary:
    """Step 2: the strip's exits and the exit reached from each border cell."""
    h, W = dir.shape
    first = dir[0].cpu().numpy().astype(np.int64)
    last = dir[h - 1].cpu().numpy().astype(np.int64)
    cols = np.arange(W)
    sides, ecols, targets = [], [], []
    for side, row, codes, open_ in ((0, first, _UP, halo & 1), (1, last, _DOWN, halo & 2)):
        if not open_:
            continue
        k = np.where(np.isin(row, codes))[0]
        t = k + _DJ[row[k]]
        ok = (t >= 0) & (t < W)  # a target beside the grid ends the path inside the strip
        k, t = k[ok], t[ok]
        sides.append(np.full(len(k), side))
        ecols.append(k)
        targets.append(t)
    side = np.concatenate(sides) if sides else np.zeros(0, np.int64)
    col = np.concatenate(ecols) if ecols else np.zeros(0, np.int64)
    tgt = np.concatenate(targets) if targets else np.zeros(0, np.int64)
    row_of = np.where(side == 0, 0, h - 1)
    A_first = A_loc[0].view(torch.int32).cpu().numpy().view(np.uint32).astype(np.uint64)
    A_last = A_loc[h - 1].view(torch.int32).cpu().numpy().view(np.uint32).astype(np.uint64)
    value = np.where(side == 0, A_first[col] if len(col) else 0, A_last[col] if len(col) else 0).astype(np.uint64)
    # exit numbers as cotangents: every cell's path sum is the number of its exit
    c = torch.zeros((h, W), dtype=torch.float32, device=dir.device)
    if len(col):
        c[torch.as_tensor(row_of, device=dir.device), torch.as_tensor(col, device=dir.device)] = \
            torch.arange(1, len(col) + 1, dtype=torch.float32, device=dir.device)
    G = backend.exit_numbers(dir, c)
    top_exit = G[0].cpu().numpy().astype(np.int64)
    bottom_exit = G[h - 1].cpu().numpy().astype(np.int64)
    return Summary(W, side, col, tgt, value, top_exit, bottom_exit)


def solve_links(summaries: list[Summary]) -> list[tuple[np.ndarray, np.ndarray]]:
    """Step 3 (Algorithms 5-6 over the strips' links): from every strip's
    summary, the inflow entering each strip's first and last row, as uint32
    (top_in, bottom_in) per strip."""
    n = len(summaries)
    W = summaries[0].W
    base = np.zeros(n + 1, dtype=np.int64)
    for k, s in enumerate(summaries):
        base[k + 1] = base[k] + len(s.exit_col)
    N = int(base[-1])
    parent = np.full(N, -1, dtype=np.int64)
    value = np.zeros(N, dtype=np.uint64)
    for k, s in enumerate(summaries):
        m = len(s.exit_col)
        if not m:
            continue
        value[base[k]:base[k + 1]] = s.exit_value
        for side, nb, key in ((0, k - 1, "bottom_exit"), (1, k + 1, "top_exit")):
            sel = np.where(s.exit_side == side)[0]
            if not len(sel):
                continue
            if nb < 0 or nb >= n:
                raise ValueError(f"strip {k} has exits towards a strip that does not exist")
            num = getattr(summaries[nb], key)[s.exit_target[sel]]
            parent[base[k] + sel] = np.where(num > 0, base[nb] + num - 1, -1)
    # subtree sums, children before parents (Kahn on the forest)
    left = np.bincount(parent[parent >= 0], minlength=N).astype(np.int64) if N else np.zeros(0, np.int64)
    F = value.copy()
    queue = list(np.where(left == 0)[0])
    done = 0
    while queue:
        x = queue.pop()
        done += 1
        p = parent[x]
        if p >= 0:
            F[p] += F[x]
            left[p] -= 1
            if left[p] == 0:
                queue.append(p)
    if done != N:
        raise ValueError("the strips' links contain a cycle")
    out = []
    for k in range(n):
        top = np.zeros(W, dtype=np.uint64)
        bottom = np.zeros(W, dtype=np.uint64)
        if k > 0:  # the strip above drains down into this strip's first row
            s = summaries[k - 1]
            sel = np.where(s.exit_side == 1)[0]
            np.add.at(top, s.exit_target[sel], F[base[k - 1] + sel])
        if k < n - 1:  # the strip below drains up into this strip's last row
            s = summaries[k + 1]
            sel = np.where(s.exit_side == 0)[0]
            np.add.at(bottom, s.exit_target[sel], F[base[k + 1] + sel])
        if top.max(initial=0) > 0xFFFFFFFF or bottom.max(initial=0) > 0xFFFFFFFF:
            raise OverflowError("counts above 2^32 - 1")
        out.append((top.astype(np.uint32), bottom.astype(np.uint32)))
    return out


def _halo(r0: int, r1: int, H: int) -> int:
    return (1 if r0 > 0 else 0) | (2 if r1 < H else 0)


def _as_dev(a: np.ndarray, device):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def flowdir_accumulate_strips(z: np.ndarray, nstrips: int, rule: str = "steepest", backend=None,
                              device="cuda") -> tuple[np.ndarray, np.ndarray]:
    """Directions and unit counts of a host-resident grid, strip by strip on one
    device (for grids larger than its memory): one strip (with its halo rows) on
    the device at a time; directions kept on the host between the two passes.
    Returns host arrays (uint8 directions, uint32 counts)."""
    backend = backend or GpuStrips(rule)
    H, W = z.shape
    rows = partition(H, nstrips)
    dirs = np.empty((H, W), dtype=np.uint8)
    summaries = []
    for r0, r1 in rows:
        halo = _halo(r0, r1, H)
        z_ext = _as_dev(z[r0 - (halo & 1):r1 + (1 if halo & 2 else 0)], device)
        d = backend.directions(z_ext, halo)
        del z_ext
        A_loc = backend.local_counts(d)
        summaries.append(summarise(backend, d, A_loc, halo))
        dirs[r0:r1] = d.cpu().numpy()
        del d, A_loc
    inflows = solve_links(summaries)
    A = np.empty((H, W), dtype=np.uint32)
    for (r0, r1), (top, bottom) in zip(rows, inflows):
        d = _as_dev(dirs[r0:r1], device)
        A[r0:r1] = backend.final_counts(d, _as_dev(top, device) if r0 > 0 else None,
                                        _as_dev(bottom, device) if r1 < H else None).view(
            torch.int32).cpu().numpy().view(np.uint32)
    return dirs, A


def distributed_flowdir_accumulate(z_strip: torch.Tensor, H: int, rank: int, world: int, group=None,
                                   rule: str = "steepest", backend=None):
    """Directions and unit counts of this rank's strip of an H-row grid (rows
    partition(H, world)[rank]), with torch.distributed initialised: one
    all-gather of the strips' boundary rows (the halo), one all-gather of the
    border summaries (message 1; every rank then solves the links, so the
    reply is local).  z_strip: this rank's rows on its device.  Returns the
    strip's (directions, counts) as tensors on that device."""
    import torch.distributed as dist

    backend = backend or GpuStrips(rule)
    r0, r1 = partition(H, world)[rank]
    h, W = z_strip.shape
    if h != r1 - r0:
        raise ValueError(f"rank {rank} holds {h} rows, its strip has {r1 - r0}")
    dev = z_strip.device
    edges = torch.stack([z_strip[0], z_strip[h - 1]]).contiguous()
    gathered = [torch.empty_like(edges) for _ in range(world)]
    dist.all_gather(gathered, edges, group=group)
    halo = _halo(r0, r1, H)
    parts = ([gathered[rank - 1][1:2]] if halo & 1 else []) + [z_strip] + ([gathered[rank + 1][0:1]] if halo & 2 else [])
    z_ext = torch.cat(parts).contiguous()
    d = backend.directions(z_ext, halo)
    del z_ext
    A_loc = backend.local_counts(d)
    rec = torch.from_numpy(summarise(backend, d, A_loc, halo).pack())
    rec = rec.to(dev) if dev.type == "cuda" else rec
    recs = [torch.empty_like(rec) for _ in range(world)]
    dist.all_gather(recs, rec, group=group)
    summaries = [Summary.unpack(r.cpu().numpy(), W) for r in recs]
    top, bottom = solve_links(summaries)[rank]
    A = backend.final_counts(d, _as_dev(top, dev) if halo & 1 else None, _as_dev(bottom, dev) if halo & 2 else None)
    return d, A
