"""Reader for the hand-worked fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_bodies(name):
    """Returns (pos [n][3], mass [n], acc [n][3], pot [n], eps)."""
    rows, eps = [], None
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [l.strip() for l in f if l.strip() and not l.lstrip().startswith("#")]
    eps = float(lines[-1])
    for l in lines[:-1]:
        rows.append([float(v) for v in l.split()])
    a = np.array(rows)
    return a[:, 0:3], a[:, 3], a[:, 4:7], a[:, 7], eps
