"""Correlation functions and the transfer-matrix spectrum of a converged
CTMRG environment (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

What it computes (paper Sec. 5.3, ``correlation`` and
``correlation_length`` sections):
  * C(r, r0) = <A(r0) B(r0 + r)> for r = (i, 0) and (0, i), 0 <= i <= r_max,
    with every site of the unit cell taken as r0 (Eq. for C(r, r0));
  * the effective correlation length xi^-1 = e_1 = -log(lambda_1 / lambda_0)
    and the further e_2, e_3, ... from the eigenvalues lambda_i of the
    transfer matrix, |lambda_0| >= |lambda_1| >= ..., which enter the
    finite-chi extrapolation 1/xi(inf) = 1/xi(chi) + k (e_2 - e_1).

Readings where the paper is silent:
  * the expectation value is the strip network (the row of sites through
    r0 and r0 + r between the row's edge tensors, closed by the corner and
    edge tensors at both ends) with A on the ket of r0 and B on the ket of
    r0 + r, divided by the same strip with no operators;
  * r = 0 is the one-site expectation of the operator product A B (B acts
    first);
  * the transfer matrix is that of one period of the cell along the
    direction (the Lx columns of a row for x, the Ly rows of a column for
    y): edge tensor above, the double-layer sites, edge tensor below;
    e_i = -ln|lambda_i / lambda_0| / period, so xi is in lattice spacings;
    the moduli are used because the lambda_i of a non-symmetric transfer
    matrix may be complex.

Leg conventions are those of ``oracle.ctmrg_ref``: C1[T4-side, T1-side],
T1[C1-side, u, u', C2-side], C2[T1-side, T2-side], T2[C2-side, r, r',
C3-side], C3[T2-side, T3-side], T3[C3-side, d, d', C4-side], C4[T3-side,
T4-side], T4[C4-side, l, l', C1-side]; A[s, l, u, r, d]; operators
O[after, before].
"""
from __future__ import annotations

import numpy as np

from .ctmrg_ref import PAIRWISE, _site


def ket_with_op(A, op):
    """A_O[t, l, u, r, d] = sum_s O[t, s] A[s, l, u, r, d]."""
    return np.einsum("ts,slurd->tlurd", op, A, optimize=PAIRWISE)


# --------------------------------------------------------------------------
# strips along +x (a row of the lattice)
# left vector L[b, l, l', t]: b the open chi index below (to the next T3),
# (l, l') the open ket/bra legs toward the next site, t the open chi index
# above (to the next T1)
# --------------------------------------------------------------------------
def left_edge_x(e):
    """C4 T4 C1 of the first site: L[b, l, l', t]."""
    return np.einsum("mn,nlLa,at->mlLt", e["C4"], e["T4"], e["C1"], optimize=PAIRWISE)


def right_edge_x(e):
    """C2 T2 C3 of the last site: R[t, r, r', b]."""
    return np.einsum("ce,erRf,fk->crRk", e["C2"], e["T2"], e["C3"], optimize=PAIRWISE)


def absorb_column(L, e, Aket, Abra):
    """L'[b', r, r', t'] = L[b, l, l', t] T1[t, u, u', t'] Aket[s, l, u, r, d]
    Abra[s, l', u', r', d'] T3[b', d, d', b]."""
    return np.einsum("mlLb,buUc,slurd,sLURD,kdDm->krRc", L, e["T1"], Aket, Abra, e["T3"], optimize=PAIRWISE)


def close_x(L, R):
    return float(np.einsum("mlLb,blLm->", L, R, optimize=PAIRWISE))


# --------------------------------------------------------------------------
# strips along +y (a column of the lattice)
# bottom vector B[w, u, u', e]: w the open chi index on the left (to the
# next T4), (u, u') the open legs toward the next site, e the open chi
# index on the right (to the next T2)
# --------------------------------------------------------------------------
def bottom_edge_y(e):
    """C4 T3 C3 of the first site: B[w, d, d', e]."""
    return np.einsum("mn,gdDm,fg->ndDf", e["C4"], e["T3"], e["C3"], optimize=PAIRWISE)


def top_edge_y(e):
    """C1 T1 C2 of the last site: T[w, u, u', e]."""
    return np.einsum("ab,buUc,ce->auUe", e["C1"], e["T1"], e["C2"], optimize=PAIRWISE)


def absorb_row(B, e, Aket, Abra):
    """B'[w', u, u', e'] = B[w, d, d', e] T4[w, l, l', w'] Aket[s, l, u, r, d]
    Abra[s, l', u', r', d'] T2[e', r, r', e]."""
    return np.einsum("ndDf,nlLa,slurd,sLURD,erRf->auUe", B, e["T4"], Aket, Abra, e["T2"], optimize=PAIRWISE)


def close_y(B, T):
    return float(np.einsum("auUe,auUe->", B, T, optimize=PAIRWISE))


def strip_value(envs, As, ops, direction, x0, y0, Lx=2, Ly=2):
    """Unnormalised strip of len(ops) sites from (x0, y0) along +x
    (direction 0) or +y (direction 1); ops[j] (or None) acts on the ket of
    the j-th site."""
    step = (1, 0) if direction == 0 else (0, 1)
    sites = [_site(x0 + j * step[0], y0 + j * step[1], Lx, Ly) for j in range(len(ops))]
    if direction == 0:
        v = left_edge_x(envs[sites[0]])
    else:
        v = bottom_edge_y(envs[sites[0]])
    for s, op in zip(sites, ops):
        Aket = As[s] if op is None else ket_with_op(As[s], op)
        v = absorb_column(v, envs[s], Aket, As[s]) if direction == 0 else absorb_row(v, envs[s], Aket, As[s])
    last = envs[sites[-1]]
    return close_x(v, right_edge_x(last)) if direction == 0 else close_y(v, top_edge_y(last))


def correlation(envs, As, opA, opB, rmax, direction, Lx=2, Ly=2):
    """C[i, r] = <A(r_i) B(r_i + r e)>, e = x (direction 0) or y (1), for
    every site i = x + Lx y of the cell and 0 <= r <= rmax."""
    out = np.zeros((Lx * Ly, rmax + 1))
    for i in range(Lx * Ly):
        x0, y0 = i % Lx, i // Lx
        for r in range(rmax + 1):
            if r == 0:
                ops, ones = [opA @ opB], [None]
            else:
                ops = [opA] + [None] * (r - 1) + [opB]
                ones = [None] * (r + 1)
            out[i, r] = (strip_value(envs, As, ops, direction, x0, y0, Lx, Ly)
                         / strip_value(envs, As, ones, direction, x0, y0, Lx, Ly))
    return out


# --------------------------------------------------------------------------
# transfer matrix of one period and its spectrum
# --------------------------------------------------------------------------
def _dense(apply, shape):
    """Matrix of the linear map `apply` on arrays of `shape` (column j =
    apply(e_j)), built in blocks of basis vectors."""
    n = int(np.prod(shape))
    Tm = np.zeros((n, n))
    for j0 in range(0, n, 256):
        j1 = min(n, j0 + 256)
        basis = np.zeros((j1 - j0, n))
        basis[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
        out = apply(basis.reshape((j1 - j0,) + tuple(shape)))
        Tm[:, j0:j1] = out.reshape(j1 - j0, n).T
    return Tm


def transfer_matrix(envs, As, direction, index, Lx=2, Ly=2):
    """Dense transfer matrix of one period: row y = index (direction 0;
    columns x = 0 .. Lx-1 in order) or column x = index (direction 1; rows
    y = 0 .. Ly-1), acting on left vectors L[b, l, l', t] (bottom vectors
    B[w, u, u', e])."""
    if direction == 0:
        sites = [_site(x, index, Lx, Ly) for x in range(Lx)]
    else:
        sites = [_site(index, y, Lx, Ly) for y in range(Ly)]
    chi = envs[sites[0]]["C1"].shape[0]
    D = As[sites[0]].shape[1]

    def apply(V):
        for s in sites:
            e, A = envs[s], As[s]
            if direction == 0:
                V = np.einsum("nmlLb,buUc,slurd,sLURD,kdDm->nkrRc", V, e["T1"], A, A, e["T3"], optimize=PAIRWISE)
            else:
                V = np.einsum("nwdDf,wlLa,slurd,sLURD,erRf->nauUe", V, e["T4"], A, A, e["T2"], optimize=PAIRWISE)
        return V

    return _dense(apply, (chi, D, D, chi))


def transfer_spectrum(envs, As, direction, index, nev=4, Lx=2, Ly=2):
    """(lambda_i / lambda_0 for i < nev, complex; e_i = -ln|lambda_i/lambda_0|
    / period for 0 < i < nev; xi = 1 / e_1)."""
    lam = np.linalg.eigvals(transfer_matrix(envs, As, direction, index, Lx, Ly))
    lam = lam[np.argsort(-np.abs(lam), kind="stable")][:nev]
    ratio = lam / lam[0]
    period = Lx if direction == 0 else Ly
    with np.errstate(divide="ignore"):
        e = -np.log(np.abs(ratio[1:])) / period
    xi = 1.0 / e[0] if len(e) and e[0] > 0 else np.inf
    return ratio, e, xi
