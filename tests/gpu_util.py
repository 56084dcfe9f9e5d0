"""Helpers for the GPU parity tests (plain torch / numpy; test code only)."""
import numpy as np
import torch

DI = (-1, -1, 0, 1, 1, 1, 0, -1)
DJ = (0, 1, 1, 1, 0, -1, -1, -1)


def u32(t: torch.Tensor) -> np.ndarray:
    return t.view(torch.int32).cpu().numpy().view(np.uint32)


def to_dev(a: np.ndarray, dev="cuda") -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@torch.no_grad()
def recursion_residual_gpu(dir: torch.Tensor, A: torch.Tensor, w: torch.Tensor | None = None) -> int:
    """max |A(p) - w(p) - sum_{n drains into p} A(n)| with plain torch ops in
    int64 (unit) -- the Eq. 1 check at any size, independent of libd8."""
    H, W = dir.shape
    dpad = torch.full((H + 2, W + 2), 255, dtype=torch.uint8, device=dir.device)
    dpad[1:-1, 1:-1] = dir
    Apad = torch.zeros((H + 2, W + 2), dtype=torch.int64, device=dir.device)
    Apad[1:-1, 1:-1] = A.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    inflow = torch.zeros((H, W), dtype=torch.int64, device=dir.device)
    for k in range(8):
        di, dj = DI[k], DJ[k]
        nd = dpad[1 + di:1 + di + H, 1 + dj:1 + dj + W]
        na = Apad[1 + di:1 + di + H, 1 + dj:1 + dj + W]
        inflow += torch.where(nd == ((k + 4) % 8), na, 0)
        del nd, na
    base = 1 if w is None else w
    res = (Apad[1:-1, 1:-1] - base - inflow).abs().max().item()
    return int(res)


@torch.no_grad()
def terminal_sum_gpu(dir: torch.Tensor, A: torch.Tensor) -> int:
    """Sum of A over cells whose path ends there (codes 8/9 or off-grid target)."""
    H, W = dir.shape
    i = torch.arange(H, device=dir.device).view(H, 1)
    j = torch.arange(W, device=dir.device).view(1, W)
    term = dir >= 8
    for k in range(8):
        off = ((i + DI[k] < 0) | (i + DI[k] >= H)) | ((j + DJ[k] < 0) | (j + DJ[k] >= W))
        term |= (dir == k) & off
    return int((A.view(torch.int32).to(torch.int64) & 0xFFFFFFFF)[term].sum().item())


def spiral_dirs(H: int, W: int) -> np.ndarray:
    """Inward rectangular spiral: one path that crosses every tile border many
    times in both directions (the paper's Fig. 1 cases B, C and D at once);
    the centre cell is a SINK."""
    d = np.full((H, W), 9, dtype=np.uint8)
    top, bot, left, right = 0, H - 1, 0, W - 1
    path = []
    while top <= bot and left <= right:
        for j in range(left, right + 1):
            path.append((top, j))
        for i in range(top + 1, bot + 1):
            path.append((i, right))
        if top < bot:
            for j in range(right - 1, left - 1, -1):
                path.append((bot, j))
        if left < right:
            for i in range(bot - 1, top, -1):
                path.append((i, left))
        top, bot, left, right = top + 1, bot - 1, left + 1, right - 1
    for (a, b), (c, e) in zip(path[:-1], path[1:]):
        k = [(DI[m], DJ[m]) for m in range(8)].index((c - a, e - b))
        d[a, b] = k
    return d
