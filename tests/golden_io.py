"""Reader for the hand-worked fixtures under tests/golden (key: value lines and
whitespace-separated grids; '#' starts a comment)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out, key, rows = {}, None, []
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            if ":" in line:
                if key is not None:
                    out[key] = rows
                k, v = line.split(":", 1)
                key, rows = k.strip(), []
                v = v.strip()
                if v:
                    out[key] = v
                    key = None
            else:
                rows.append(line.split())
        if key is not None:
            out[key] = rows
    return out


def grid(rows, dtype):
    return np.array([[dtype(x) for x in r] for r in rows])


def ints(s: str):
    return [int(x, 0) for x in s.split()]
