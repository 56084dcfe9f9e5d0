"""Reader for the hand-worked text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def sections(name):
    """Return a list of (header, rows) pairs; header is the text inside [...]
    (plus anything after it on that line), rows the numeric lines below."""
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                head = line[1:line.index("]")]
                rest = line[line.index("]") + 1:].split()
                out.append([head, [] if not rest else [rest]])
            else:
                out[-1][1].append(line.split())
    return [(h, rows) for h, rows in out]


def grid(rows, dtype):
    return np.array([[float(x) for x in r] for r in rows]).astype(dtype)


def named(name):
    return {h: rows for h, rows in sections(name)}
