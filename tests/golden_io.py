"""Readers for the text fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def constants():
    out = {}
    with open(os.path.join(GOLDEN, "constants.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            vals = [float(v) for v in vals]
            out[key] = vals[0] if len(vals) == 1 else vals
    return out


def multi_indices():
    rows = []
    with open(os.path.join(GOLDEN, "multi_indices.txt")) as f:
        lines = [l.split() for l in f if l.strip() and not l.startswith("#")]
    M, p = int(lines[0][0]), int(lines[0][1])
    for l in lines[1:]:
        rows.append([int(v) for v in l])
    return M, p, rows
