"""Operator element format (paper Sec. 5.2, ``elements`` of a Hamiltonian term).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

One line per non-zero element: the states of the source and target sites
before the operator acts, then after, then the real and imaginary parts.
The matrix is O[after, before] on the combined index (source * d1 + target).
"""
from __future__ import annotations

import numpy as np


def op_from_elements(d0: int, d1: int, lines) -> np.ndarray:
    n = d0 * d1
    op = np.zeros((n, n))
    for (i0, j0, i1, j1, re, im) in lines:
        if im != 0.0:
            raise ValueError("real operators only")
        op[i1 * d1 + j1, i0 * d1 + j0] += re
    return op


def parse_elements(text: str):
    out = []
    for line in text.strip().splitlines():
        f = line.split()
        if not f:
            continue
        out.append((int(f[0]), int(f[1]), int(f[2]), int(f[3]), float(f[4]), float(f[5])))
    return out
