"""Brute-force references used to pin the oracle (test code only).

They restate the problem in the most direct way possible -- follow every
cell's flow path cell by cell -- and share no code with the oracle or the
CUDA library.
"""
import numpy as np

# neighbour offsets for codes 0..7 = N, NE, E, SE, S, SW, W, NW (row grows south)
_DI = (-1, -1, 0, 1, 1, 1, 0, -1)
_DJ = (0, 1, 1, 1, 0, -1, -1, -1)


def successors(dir):
    """Flat index of each cell's down-slope neighbour, -1 where the path ends."""
    H, W = dir.shape
    d = np.asarray(dir).astype(np.int64)
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    di = np.array(_DI + (0,) * 248)[np.minimum(d, 255)]
    dj = np.array(_DJ + (0,) * 248)[np.minimum(d, 255)]
    ti, tj = ii + di, jj + dj
    ok = (d < 8) & (ti >= 0) & (ti < H) & (tj >= 0) & (tj < W)
    return np.where(ok, ti * W + tj, -1).ravel()


def paths(dir):
    """Each cell's full flow path (list of flat indices, starting at the cell);
    None if the path revisits a cell (a cycle)."""
    nxt = successors(dir)
    n = nxt.size
    out = []
    for c in range(n):
        p, seen = [c], {c}
        x = c
        while nxt[x] >= 0:
            x = int(nxt[x])
            if x in seen:
                return None
            seen.add(x)
            p.append(x)
        out.append(p)
    return out


def counts(dir, w=None):
    """A(p) = total weight of the cells whose path passes through p."""
    H, W = dir.shape
    ps = paths(dir)
    if ps is None:
        return None
    A = np.zeros(H * W, dtype=np.float64 if w is not None else np.int64)
    wf = None if w is None else np.asarray(w, dtype=np.float64).ravel()
    for c, p in enumerate(ps):
        for x in p:
            A[x] += 1 if wf is None else wf[c]
    return A.reshape(H, W)


def path_sums(dir, c):
    """G(q) = sum of c over q's path (q included)."""
    H, W = dir.shape
    ps = paths(dir)
    cf = np.asarray(c, dtype=np.float64).ravel()
    return np.array([cf[p].sum() for p in ps]).reshape(H, W)


def recursion_residual(dir, A, w=None):
    """max |A(p) - w(p) - sum_{n: succ(n)=p} A(n)| (vectorised, Eq. 1)."""
    H, W = dir.shape
    nxt = successors(dir)
    A = np.asarray(A, dtype=np.float64).ravel()
    wf = np.ones(H * W) if w is None else np.asarray(w, dtype=np.float64).ravel()
    inflow = np.zeros(H * W)
    m = nxt >= 0
    np.add.at(inflow, nxt[m], A[m])
    return np.abs(A - wf - inflow).max()


def terminal_mask(dir):
    return (successors(dir) < 0).reshape(dir.shape)
