"""Independent tensor-network builder for pinning the oracle's contractions.

The networks here are generated from grid geometry -- which tensor sits
next to which -- rather than from hand-written contraction strings, and are
contracted by a generic pairwise contractor.  A wrong leg or a swapped
operand in the oracle's hand-written contractions shows up as a mismatch.

Conventions (same as the library): A[s,l,u,r,d], y up; environment of a
site clockwise C1[c_T4,c_T1] T1[c_C1,k,k',c_C2] C2[c_T1,c_T2]
T2[c_C2,k,k',c_C3] C3[c_T2,c_T3] T3[c_C3,k,k',c_C4] C4[c_T3,c_T4]
T4[c_C4,k,k',c_C1].
"""
from __future__ import annotations

import itertools
import string

import numpy as np


def contract(tensors, open_order):
    """tensors: list of (array, [label, ...]); every label appears once (open)
    or twice (bond).  Greedy pairwise contraction; open legs in open_order."""
    ts = [(np.asarray(a), list(l)) for a, l in tensors]
    while len(ts) > 1:
        best = None
        for i, j in itertools.combinations(range(len(ts)), 2):
            shared = set(ts[i][1]) & set(ts[j][1])
            if not shared:
                continue
            out = [l for l in ts[i][1] if l not in shared] + [l for l in ts[j][1] if l not in shared]
            dims = {l: n for l, n in zip(ts[i][1], ts[i][0].shape)}
            dims.update({l: n for l, n in zip(ts[j][1], ts[j][0].shape)})
            size = int(np.prod([dims[l] for l in out])) if out else 1
            if best is None or size < best[0]:
                best = (size, i, j, out)
        if best is None:
            i, j, out = 0, 1, ts[0][1] + ts[1][1]
        else:
            _, i, j, out = best
        (a, la), (b, lb) = ts[i], ts[j]
        sym = {}
        for l in la + lb:
            sym.setdefault(l, string.ascii_letters[len(sym)])
        spec = ("".join(sym[l] for l in la) + "," + "".join(sym[l] for l in lb) + "->"
                + "".join(sym[l] for l in out))
        c = np.einsum(spec, a, b)
        ts = [t for k, t in enumerate(ts) if k not in (i, j)] + [(c, out)]
    a, labels = ts[0]
    assert sorted(map(repr, labels)) == sorted(map(repr, open_order)), (labels, open_order)
    return np.transpose(a, [labels.index(l) for l in open_order])


def _site(x, y, Lx, Ly):
    return (x % Lx) + Lx * (y % Ly)


def block_network(envs, As, x0, y0, nx, ny, open_sites=(), Lx=2, Ly=2):
    """The sites x0..x0+nx-1 by y0..y0+ny-1 (ket and bra layers) with their
    environment: T1 above every top site, T3 below every bottom site, T2
    right of every right site, T4 left of every left site, and the corner
    of each corner site.  Open legs: ('ket', i) / ('bra', i) for open sites."""
    xs = range(x0, x0 + nx)
    ys = range(y0, y0 + ny)
    xl, xr, yb, yt = x0, x0 + nx - 1, y0, y0 + ny - 1
    st = lambda x, y: _site(x, y, Lx, Ly)
    T = []
    for x in xs:
        for y in ys:
            i = st(x, y)
            for layer in ("k", "b"):
                phys = ("phys", x, y)
                if i in open_sites:
                    phys = ("ket" if layer == "k" else "bra", i)
                # horizontal bond (x,y)-(x+1,y) = (layer,'h',x,y); vertical (x,y)-(x,y+1) = (layer,'v',x,y)
                T.append((As[i], [phys, (layer, "h", x - 1, y), (layer, "v", x, y),
                                  (layer, "h", x, y), (layer, "v", x, y - 1)]))
    for x in xs:   # top and bottom edges
        T.append((envs[st(x, yt)]["T1"], [("top", x - 1), ("k", "v", x, yt), ("b", "v", x, yt), ("top", x)]))
        T.append((envs[st(x, yb)]["T3"], [("bot", x), ("k", "v", x, yb - 1), ("b", "v", x, yb - 1), ("bot", x - 1)]))
    for y in ys:   # right and left edges
        T.append((envs[st(xr, y)]["T2"], [("right", y), ("k", "h", xr, y), ("b", "h", xr, y), ("right", y - 1)]))
        T.append((envs[st(xl, y)]["T4"], [("left", y - 1), ("k", "h", xl - 1, y), ("b", "h", xl - 1, y), ("left", y)]))
    T.append((envs[st(xl, yt)]["C1"], [("left", yt), ("top", xl - 1)]))
    T.append((envs[st(xr, yt)]["C2"], [("top", xr), ("right", yt)]))
    T.append((envs[st(xr, yb)]["C3"], [("right", yb - 1), ("bot", xr)]))
    T.append((envs[st(xl, yb)]["C4"], [("bot", xl - 1), ("left", yb - 1)]))
    return T


def row_strip(envs, x0, nx, yb, yt, Lx=2, Ly=2):
    """No sites: the top edges of row yt and the bottom edges of row yb over
    columns x0.., joined ket-to-ket and bra-to-bra, closed by the corners."""
    st = lambda x, y: _site(x, y, Lx, Ly)
    xl, xr = x0, x0 + nx - 1
    T = []
    for x in range(x0, x0 + nx):
        T.append((envs[st(x, yt)]["T1"], [("top", x - 1), ("gk", x), ("gb", x), ("top", x)]))
        T.append((envs[st(x, yb)]["T3"], [("bot", x), ("gk", x), ("gb", x), ("bot", x - 1)]))
    T.append((envs[st(xl, yt)]["C1"], [("L",), ("top", xl - 1)]))
    T.append((envs[st(xr, yt)]["C2"], [("top", xr), ("R",)]))
    T.append((envs[st(xr, yb)]["C3"], [("R",), ("bot", xr)]))
    T.append((envs[st(xl, yb)]["C4"], [("bot", xl - 1), ("L",)]))
    return T


def column_strip(envs, xl, xr, y0, ny, Lx=2, Ly=2):
    """No sites: right edges of column xr and left edges of column xl over
    rows y0.., joined through their ket/bra legs, closed by the corners."""
    st = lambda x, y: _site(x, y, Lx, Ly)
    yb, yt = y0, y0 + ny - 1
    T = []
    for y in range(y0, y0 + ny):
        T.append((envs[st(xr, y)]["T2"], [("right", y), ("gk", y), ("gb", y), ("right", y - 1)]))
        T.append((envs[st(xl, y)]["T4"], [("left", y - 1), ("gk", y), ("gb", y), ("left", y)]))
    T.append((envs[st(xl, yt)]["C1"], [("left", yt), ("T",)]))
    T.append((envs[st(xr, yt)]["C2"], [("T",), ("right", yt)]))
    T.append((envs[st(xr, yb)]["C3"], [("right", yb - 1), ("B",)]))
    T.append((envs[st(xl, yb)]["C4"], [("B",), ("left", yb - 1)]))
    return T


def corners_only(envs, xl, xr, yb, yt, Lx=2, Ly=2):
    st = lambda x, y: _site(x, y, Lx, Ly)
    return [(envs[st(xl, yt)]["C1"], [("L",), ("T",)]),
            (envs[st(xr, yt)]["C2"], [("T",), ("R",)]),
            (envs[st(xr, yb)]["C3"], [("R",), ("B",)]),
            (envs[st(xl, yb)]["C4"], [("B",), ("L",)])]
