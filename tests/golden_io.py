"""Reader for the hand-worked fixtures under tests/golden/."""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out, block, rows = {}, None, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.endswith(":") and line[:-1].isidentifier():
                if block is not None:
                    out[block] = np.array(rows, dtype=np.uint32)
                block, rows = line[:-1], []
            elif ":" in line and block is None:
                k, v = line.split(":", 1)
                out[k.strip()] = int(v)
            else:
                rows.append([int(t) for t in line.split()])
    if block is not None:
        out[block] = np.array(rows, dtype=np.uint32)
    return out


def all_fixtures():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
