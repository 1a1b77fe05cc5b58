"""Reader for the hand-worked fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    """Parse `name`: '#' comments, 'key value' lines, and matrices written as
    'NAME rows cols' followed by `rows` lines of numbers."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        parts = lines[i].split()
        if len(parts) == 3 and parts[1].isdigit() and parts[2].isdigit():
            key, r, c = parts[0], int(parts[1]), int(parts[2])
            rows = [lines[i + 1 + t].split() for t in range(r)]
            out[key] = [[float(v) if ("." in v or "e" in v or "inf" in v) else int(v)
                         for v in row] for row in rows]
            assert all(len(row) == c for row in rows)
            i += 1 + r
        else:
            out[parts[0]] = parts[1] if len(parts) > 1 else None
            i += 1
    return out


def as_i32(m):
    return np.array(m, dtype=np.int64).astype(np.int32)


def as_f32(m):
    return np.array(m, dtype=np.float64).astype(np.float32)
