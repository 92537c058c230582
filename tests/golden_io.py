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


def field(g: dict) -> np.ndarray:
    """A fixture's input field as float32: 2D from 'field', 3D from the planes
    'field_z0', 'field_z1', ..."""
    if "field" in g:
        return grid(g["field"], np.float32).astype(np.float32)
    nz = sum(1 for k in g if k.startswith("field_z"))
    return np.stack([grid(g[f"field_z{z}"], np.float32) for z in range(nz)]).astype(np.float32)
