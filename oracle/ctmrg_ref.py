"""Plain FP64 directional CTMRG for an iTPS unit cell (oracle).

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

What it computes (paper Sec. 2.2, "Contraction of iTPS"):
  the bra and ket layers are merged site by site into a single-layer
  network of bond dimension D^2; the environment of every site is a set of
  four corner matrices (chi x chi) and four edge tensors (chi x D x D x chi);
  they are found iteratively by the directional CTMRG of Corboz et al. for
  arbitrary unit cells, modified so that the projectors are built without
  the QR step.  Expectation values of one- and two-site operators follow
  from the reduced density matrices of the converged network (Sec. 5.3,
  ``observable`` section).

The projector of a cut is the plain definition: the two half systems H_u,
H_d are formed as dense matrices, M = H_u^T H_d, a full SVD M = U S V^T is
taken and truncated to chi, and
    P_up = H_d V S^{-1/2},   P_dn = S^{-1/2} U^T H_u^T,
so that P_dn P_up = 1 (kept part) and H_u^T P_up P_dn H_d = U_chi S_chi V_chi^T.
(The randomized / Arnoldi partial SVD the paper mentions is a faster way to
reach the same truncated triplets and is not used here.)

Readings where the paper is silent:
  * one sweep = left, top, right, bottom moves; each move visits the columns
    in order and, per column, computes the projectors of every row cut
    before updating any tensor (Corboz-style simultaneous row update);
  * top/right/bottom moves are left moves of the lattice rotated by 90
    degrees counter-clockwise (site (x,y) -> (-y, x), A legs relabelled,
    C/T relabelled cyclically);
  * singular values below ``cutoff * s_0`` (default 1e-12) get
    S^{-1/2} := 0; closer to the FP64 noise floor of M the noise
    directions, amplified by S^{-1/2}, destabilise the iteration;
  * every new C and T is divided by its largest absolute element;
  * convergence: the normalised (sum = 1) singular values of all corners,
    max-abs change between consecutive sweeps.

Layout conventions are those of ``paper_2112_13184_gb300.inputs``.
"""
from __future__ import annotations

import numpy as np

ENV_NAMES = ("C1", "T1", "C2", "T2", "C3", "T3", "C4", "T4")

# Einsums are evaluated as chains of pairwise (BLAS) contractions with no
# cap on the size of the intermediates.  (numpy's default cap makes it fold
# the last three operands of an enlarged corner into one unblocked loop,
# which takes minutes at D = 8.)  The two 8-operand strips of ln kappa keep
# numpy's capped search, which there avoids a D^6 chi^2-sized intermediate.
# This fixes only the order in which each einsum's sum is evaluated, not
# what it sums.
PAIRWISE = ("greedy", 1 << 40)


def _site(x, y, Lx, Ly):
    return (x % Lx) + Lx * (y % Ly)


# --------------------------------------------------------------------------
# double layer (Sec. 2.2, Fig. 2(b))
# --------------------------------------------------------------------------
def double_layer(A):
    """a[(l l'), (u u'), (r r'), (d d')] = sum_s A[s,l,u,r,d] A[s,l',u',r',d']."""
    d, D1, D2, D3, D4 = A.shape
    a = np.einsum("slurd,sLURD->lLuUrRdD", A, A, optimize=PAIRWISE)
    return a.reshape(D1 * D1, D2 * D2, D3 * D3, D4 * D4)


# --------------------------------------------------------------------------
# enlarged corners around a horizontal cut (left move)
# Each returns an N x N matrix, N = chi D^2; grouped legs are
# (chi index, ket leg, bra leg) in that order.
# --------------------------------------------------------------------------
def enlarged_ul(C1, T1, T4, A):
    """Upper-left: rows = down leg (T4.c_C4, A.d, A*.d), cols = right leg (T1.c_C2, A.r, A*.r)."""
    Q = np.einsum("gh,huUb,alLg,slurd,sLURD->adDbrR", C1, T1, T4, A, A, optimize=PAIRWISE)
    s = Q.shape
    return Q.reshape(s[0] * s[1] * s[2], s[3] * s[4] * s[5])


def enlarged_ur(T1, C2, T2, A):
    """Upper-right: rows = left leg (T1.c_C1, A.l, A*.l), cols = down leg (T2.c_C3, A.d, A*.d)."""
    Q = np.einsum("buUg,gh,hrRe,slurd,sLURD->blLedD", T1, C2, T2, A, A, optimize=PAIRWISE)
    s = Q.shape
    return Q.reshape(s[0] * s[1] * s[2], s[3] * s[4] * s[5])


def enlarged_br(T2, C3, T3, A):
    """Lower-right: rows = left leg (T3.c_C4, A.l, A*.l), cols = up leg (T2.c_C2, A.u, A*.u)."""
    Q = np.einsum("erRg,gh,hdDz,slurd,sLURD->zlLeuU", T2, C3, T3, A, A, optimize=PAIRWISE)
    s = Q.shape
    return Q.reshape(s[0] * s[1] * s[2], s[3] * s[4] * s[5])


def enlarged_bl(T4, C4, T3, A):
    """Lower-left: rows = up leg (T4.c_C1, A.u, A*.u), cols = right leg (T3.c_C3, A.r, A*.r)."""
    Q = np.einsum("glLa,hg,zdDh,slurd,sLURD->auUzrR", T4, C4, T3, A, A, optimize=PAIRWISE)
    s = Q.shape
    return Q.reshape(s[0] * s[1] * s[2], s[3] * s[4] * s[5])


def cut_corners(envs, As, x, y, Lx, Ly):
    """The four enlarged corners around the cut between rows y and y+1 at
    columns x, x+1: TL=(x,y+1), TR=(x+1,y+1), BR=(x+1,y), BL=(x,y)."""
    tl = _site(x, y + 1, Lx, Ly)
    tr = _site(x + 1, y + 1, Lx, Ly)
    br = _site(x + 1, y, Lx, Ly)
    bl = _site(x, y, Lx, Ly)
    Qul = enlarged_ul(envs[tl]["C1"], envs[tl]["T1"], envs[tl]["T4"], As[tl])
    Qur = enlarged_ur(envs[tr]["T1"], envs[tr]["C2"], envs[tr]["T2"], As[tr])
    Qbr = enlarged_br(envs[br]["T2"], envs[br]["C3"], envs[br]["T3"], As[br])
    Qbl = enlarged_bl(envs[bl]["T4"], envs[bl]["C4"], envs[bl]["T3"], As[bl])
    return Qul, Qur, Qbr, Qbl


# --------------------------------------------------------------------------
# projectors without QR (Sec. 2.2)
# --------------------------------------------------------------------------
def half_systems(Qul, Qur, Qbr, Qbl):
    """H_u[a, b] = Q_ul Q_ur ; H_d[a, b] = Q_bl Q_br (a = left cut bond, b = right).

    Each corner maps the bond it shares with its predecessor to the next one
    around the cut: a -> e -> b above (e the vertical bond between TL, TR),
    a -> f -> b below (f between BL, BR)."""
    return Qul @ Qur, Qbl @ Qbr


def projectors(Qul, Qur, Qbr, Qbl, chi, cutoff=1e-12):
    """Return (P_up [N x chi], P_dn [chi x N], s [chi]) for one cut.

    M = H_u^T H_d ; full SVD ; truncation to chi ; S^{-1/2} of singular
    values below cutoff * s_0 set to zero.
    """
    Hu, Hd = half_systems(Qul, Qur, Qbr, Qbl)
    M = Hu.T @ Hd
    U, S, Vt = np.linalg.svd(M)
    k = min(chi, S.shape[0])
    s = S[:k]
    inv = np.zeros(k)
    keep = s > cutoff * S[0]
    inv[keep] = 1.0 / np.sqrt(s[keep])
    P_up = (Hd @ Vt[:k].T) * inv[None, :]
    P_dn = inv[:, None] * (U[:, :k].T @ Hu.T)
    if k < chi:  # pad to fixed shape (only when N < chi)
        P_up = np.pad(P_up, ((0, 0), (0, chi - k)))
        P_dn = np.pad(P_dn, ((0, chi - k), (0, 0)))
        s = np.pad(s, (0, chi - k))
    return P_up, P_dn, s


# --------------------------------------------------------------------------
# absorption + renormalisation (left move)
# --------------------------------------------------------------------------
def absorb_C1(C1, T1, P_up):
    """C1'[c, b] = sum_a P_up[a, c] (C1 T1)[a=(C1.c_T4, T1.k, T1.k'), b=T1.c_C2]."""
    CT = np.einsum("gh,huUb->guUb", C1, T1, optimize=PAIRWISE)
    s = CT.shape
    return P_up.T @ CT.reshape(s[0] * s[1] * s[2], s[3])


def absorb_C4(C4, T3, P_dn):
    """C4'[z, c] = sum_a (C4 T3)[a=(C4.c_T4, T3.k, T3.k'), z=T3.c_C3] P_dn[c, a]."""
    CT = np.einsum("hg,zdDh->gdDz", C4, T3, optimize=PAIRWISE)
    s = CT.shape
    return CT.reshape(s[0] * s[1] * s[2], s[3]).T @ P_dn.T


def absorb_T4(T4, A, P_up_below, P_dn_above):
    """T4'[c1, r, r', c2] = P_up(cut below)[a_b, c1] (T4 A A*)[a_b, (r r'), a_t] P_dn(cut above)[c2, a_t].

    a_b = (T4.c_C4, A.d, A*.d), a_t = (T4.c_C1, A.u, A*.u)."""
    X = np.einsum("alLg,slurd,sLURD->adDrRguU", T4, A, A, optimize=PAIRWISE)
    s = X.shape
    X = X.reshape(s[0] * s[1] * s[2], s[3], s[4], s[5] * s[6] * s[7])
    return np.einsum("ac,arRb,eb->crRe", P_up_below, X, P_dn_above, optimize=PAIRWISE)


def normalise(t):
    m = np.max(np.abs(t))
    return t / m if m > 0 else t


def left_move_column(envs, As, x, Lx, Ly, chi, cutoff=1e-12):
    """Absorb column x into the left boundary: new C1, T4, C4 of column x+1."""
    Pup, Pdn = {}, {}
    for y in range(Ly):
        Pup[y], Pdn[y], _ = projectors(*cut_corners(envs, As, x, y, Lx, Ly), chi, cutoff)
    new = {}
    for y in range(Ly):
        i = _site(x, y, Lx, Ly)
        e = envs[i]
        ym = (y - 1) % Ly
        new[y] = (normalise(absorb_C1(e["C1"], e["T1"], Pup[y])),
                  normalise(absorb_T4(e["T4"], As[i], Pup[ym], Pdn[y])),
                  normalise(absorb_C4(e["C4"], e["T3"], Pdn[ym])))
    for y in range(Ly):
        j = _site(x + 1, y, Lx, Ly)
        envs[j]["C1"], envs[j]["T4"], envs[j]["C4"] = new[y]


def rotate_ccw(envs, As, Lx, Ly):
    """Rotate the lattice by 90 degrees counter-clockwise: site (x,y)->(-y,x).

    Top becomes left, so a left move of the rotated system is a top move of
    the original.  A'[s,l,u,r,d] = A[s,d,l,u,r]; C1'=C2, T1'=T2, C2'=C3,
    T2'=T3, C3'=C4, T3'=T4, C4'=C1, T4'=T1 (arrays unchanged)."""
    Lx2, Ly2 = Ly, Lx
    envs2 = [None] * (Lx * Ly)
    As2 = [None] * (Lx * Ly)
    for y in range(Ly):
        for x in range(Lx):
            i = _site(x, y, Lx, Ly)
            j = _site(-y, x, Lx2, Ly2)
            e = envs[i]
            envs2[j] = {"C1": e["C2"], "T1": e["T2"], "C2": e["C3"], "T2": e["T3"],
                        "C3": e["C4"], "T3": e["T4"], "C4": e["C1"], "T4": e["T1"]}
            As2[j] = np.ascontiguousarray(As[i].transpose(0, 2, 3, 4, 1))
    return envs2, As2, Lx2, Ly2


def sweep(envs, As, Lx, Ly, chi, cutoff=1e-12):
    """One CTMRG sweep: left, top, right, bottom moves (in place on envs)."""
    cur_e, cur_A, lx, ly = envs, As, Lx, Ly
    for _ in range(4):
        for x in range(lx):
            left_move_column(cur_e, cur_A, x, lx, ly, chi, cutoff)
        cur_e, cur_A, lx, ly = rotate_ccw(cur_e, cur_A, lx, ly)
    for i in range(Lx * Ly):
        envs[i] = cur_e[i]


def corner_spectra(envs):
    """Normalised singular values (sum = 1) of every corner, shape [sites, 4, chi]."""
    out = []
    for e in envs:
        row = []
        for name in ("C1", "C2", "C3", "C4"):
            s = np.linalg.svd(e[name], compute_uv=False)
            row.append(s / np.sum(s))
        out.append(row)
    return np.array(out)


def loop_spectra(envs, Lx=2, Ly=2):
    """Gauge-invariant corner spectra, shape [sites, chi].

    For the 2x2 block whose bottom-left site is i = (x, y), the four corners
    around it joined directly, L = C1(x, y+1) C2(x+1, y+1) C3(x+1, y) C4(x, y),
    close a loop: each corner leg meets the leg of its neighbour across the
    same chi bond (the network with no edge tensors and no sites, whose
    trace is the Z_00 of the free-energy ratio).  A change of basis G on any
    chi bond turns L into a similar matrix, so its eigenvalues do not depend
    on the gauge the projectors leave on the chi bonds, while the singular
    values of a single corner do.  Returned: the eigenvalue moduli, sorted
    descending, divided by their sum."""
    out = []
    for i in range(Lx * Ly):
        x, y = i % Lx, i // Lx
        L = (envs[_site(x, y + 1, Lx, Ly)]["C1"] @ envs[_site(x + 1, y + 1, Lx, Ly)]["C2"]
             @ envs[_site(x + 1, y, Lx, Ly)]["C3"] @ envs[_site(x, y, Lx, Ly)]["C4"])
        m = np.sort(np.abs(np.linalg.eigvals(L)))[::-1]
        out.append(m / np.sum(m))
    return np.array(out)


def cut_singular_values(envs, As, x, y, Lx=2, Ly=2):
    """All singular values of M = H_u^T H_d for the cut between rows y and
    y+1 at column x (left move, unrotated lattice): the gap at chi tells
    whether the truncation to chi is well posed."""
    Hu, Hd = half_systems(*cut_corners(envs, As, x, y, Lx, Ly))
    return np.linalg.svd(Hu.T @ Hd, compute_uv=False)


def run(As, envs, chi, max_sweeps, tol=0.0, Lx=2, Ly=2, cutoff=1e-12):
    """Iterate sweeps; stop early when the corner-spectrum change < tol.

    Returns (envs, sweeps_done, last_delta).  ``envs`` is copied first."""
    envs = [{k: v.copy() for k, v in e.items()} for e in envs]
    prev = corner_spectra(envs)
    delta = np.inf
    n = 0
    for n in range(1, max_sweeps + 1):
        sweep(envs, As, Lx, Ly, chi, cutoff)
        cur = corner_spectra(envs)
        delta = float(np.max(np.abs(cur - prev)))
        prev = cur
        if tol > 0 and delta < tol:
            break
    return envs, n, delta


# --------------------------------------------------------------------------
# reduced density matrices and expectation values (Sec. 5.3)
# rho[ket, bra]; <O> = Tr(O rho) with O[after, before].
# --------------------------------------------------------------------------
def rdm1(envs, As, i):
    """rho[s, t] = full network around site i with the ket index s and the
    bra index t left open, divided by its trace."""
    e, A = envs[i], As[i]
    # left column: C4 T4 C1 -> [c_T3, l, l', c_T1]
    left = np.einsum("mn,nlLa,ab->mlLb", e["C4"], e["T4"], e["C1"], optimize=PAIRWISE)
    # right column: C2 T2 C3 -> [c_T1, r, r', c_T3]
    right = np.einsum("ce,erRf,fg->crRg", e["C2"], e["T2"], e["C3"], optimize=PAIRWISE)
    top = np.einsum("mlLb,buUc->mlLuUc", left, e["T1"], optimize=PAIRWISE)          # + T1
    top = np.einsum("mlLuUc,crRg->mlLuUrRg", top, right, optimize=PAIRWISE)           # + right column
    ring = np.einsum("mlLuUrRg,gdDm->lLuUrRdD", top, e["T3"], optimize=PAIRWISE)      # + T3 closes the ring
    ket = np.einsum("lLuUrRdD,slurd->sLURD", ring, A, optimize=PAIRWISE)
    rho = np.einsum("sLURD,tLURD->st", ket, A, optimize=PAIRWISE)
    return rho / np.trace(rho)


def _half_h_left(e, A):
    """Left half of the horizontal pair: C4 T4 C1 T1 T3 around A, A*.
    Returns [c (T1.c_C2), x (A.r), X (A*.r), k (T3.c_C3), p (ket s), q (bra s)]."""
    t = np.einsum("mn,nlLa,ab->mlLb", e["C4"], e["T4"], e["C1"], optimize=PAIRWISE)
    t = np.einsum("mlLb,buUc->mlLuUc", t, e["T1"], optimize=PAIRWISE)
    t = np.einsum("kdDm,mlLuUc->kdDlLuUc", e["T3"], t, optimize=PAIRWISE)
    t = np.einsum("kdDlLuUc,pluxd->kDLUcpx", t, A, optimize=PAIRWISE)
    return np.einsum("kDLUcpx,qLUXD->cxXkpq", t, A, optimize=PAIRWISE)


def _half_h_right(e, A):
    """Right half: T1 C2 T2 C3 T3 around A, A*.
    Returns [c (T1.c_C1), x (A.l), X (A*.l), k (T3.c_C4), s, t]."""
    u = np.einsum("cvVe,ef,frRg,gh->cvVrRh", e["T1"], e["C2"], e["T2"], e["C3"], optimize=PAIRWISE)
    u = np.einsum("cvVrRh,hwWk->cvVrRwWk", u, e["T3"], optimize=PAIRWISE)
    u = np.einsum("cvVrRwWk,sxvrw->cVRWksx", u, A, optimize=PAIRWISE)
    return np.einsum("cVRWksx,tXVRW->cxXkst", u, A, optimize=PAIRWISE)


def rdm2_horizontal(envs, As, i, j):
    """i = left site, j = its right neighbour; rho[(s_i s_j), (t_i t_j)]."""
    L = _half_h_left(envs[i], As[i])
    Rh = _half_h_right(envs[j], As[j])
    rho = np.einsum("cxXkpq,cxXkst->psqt", L, Rh, optimize=PAIRWISE)
    dI, dJ = As[i].shape[0], As[j].shape[0]
    rho = rho.reshape(dI * dJ, dI * dJ)
    return rho / np.trace(rho)


def _half_v_top(e, A):
    """Top half of the vertical pair: T4 C1 T1 C2 T2 around A, A*.
    Returns [n (T4.c_C4), y (A.d), Y (A*.d), f (T2.c_C3), s, t]."""
    u = np.einsum("nvVa,ab,buUc,ce->nvVuUe", e["T4"], e["C1"], e["T1"], e["C2"], optimize=PAIRWISE)
    u = np.einsum("nvVuUe,erRf->nvVuUrRf", u, e["T2"], optimize=PAIRWISE)
    u = np.einsum("nvVuUrRf,svury->nVURfsy", u, A, optimize=PAIRWISE)
    return np.einsum("nVURfsy,tVURY->nyYfst", u, A, optimize=PAIRWISE)


def _half_v_bottom(e, A):
    """Bottom half: T2 C3 T3 C4 T4 around A, A*.
    Returns [n (T4.c_C1), y (A.u), Y (A*.u), f (T2.c_C2), p, q]."""
    t = np.einsum("fwWg,gh,hdDk,km->fwWdDm", e["T2"], e["C3"], e["T3"], e["C4"], optimize=PAIRWISE)
    t = np.einsum("fwWdDm,mlLn->fwWdDlLn", t, e["T4"], optimize=PAIRWISE)
    t = np.einsum("fwWdDlLn,plywd->fWDLnpy", t, A, optimize=PAIRWISE)
    return np.einsum("fWDLnpy,qLYWD->nyYfpq", t, A, optimize=PAIRWISE)


def rdm2_vertical(envs, As, i, j):
    """i = bottom site, j = its top neighbour; rho[(s_i s_j), (t_i t_j)]."""
    Tp = _half_v_top(envs[j], As[j])
    Bt = _half_v_bottom(envs[i], As[i])
    rho = np.einsum("nyYfst,nyYfpq->psqt", Tp, Bt, optimize=PAIRWISE)
    dI, dJ = As[i].shape[0], As[j].shape[0]
    rho = rho.reshape(dI * dJ, dI * dJ)
    return rho / np.trace(rho)


def swap_sites(rho, dI, dJ):
    """rho over (i, j) -> rho over (j, i)."""
    r = rho.reshape(dI, dJ, dI, dJ).transpose(1, 0, 3, 2)
    return r.reshape(dI * dJ, dI * dJ)


def rdm2(envs, As, i, dx, dy, Lx=2, Ly=2):
    """Two-site RDM of source site i and target i + (dx, dy), |dx|+|dy| = 1."""
    if abs(dx) + abs(dy) != 1:
        raise ValueError("nearest neighbours only")
    x, y = i % Lx, i // Lx
    j = _site(x + dx, y + dy, Lx, Ly)
    dI, dJ = As[i].shape[0], As[j].shape[0]
    if (dx, dy) == (1, 0):
        return rdm2_horizontal(envs, As, i, j)
    if (dx, dy) == (-1, 0):
        return swap_sites(rdm2_horizontal(envs, As, j, i), dJ, dI)
    if (dx, dy) == (0, 1):
        return rdm2_vertical(envs, As, i, j)
    return swap_sites(rdm2_vertical(envs, As, j, i), dJ, dI)


def expect(op, rho):
    return float(np.trace(op @ rho))


# --------------------------------------------------------------------------
# free energy per site from the converged environment (2x2 block ratio)
# --------------------------------------------------------------------------
def log_kappa_per_site(envs, As):
    """ln kappa per site = (1/4) ln(Z_22 Z_00 / (Z_20 Z_02)) for a 2x2 cell.

    Sites TL=(0,1), TR=(1,1), BL=(0,0), BR=(1,0).  Z_22: the 4 corners, the
    8 edge tensors around the cell and its 4 double-layer sites, evaluated as
    Tr(H_u^T H_d) of the cut through the block; Z_00: the
    four corners joined directly; Z_20: corners plus the top and bottom edge
    pairs, each T1 ket/bra leg joined to the T3 of the same column (a strip
    with no sites); Z_02: likewise with the right and left edge pairs.
    Environment normalisations cancel in the ratio; A -> c A adds 2 ln c.
    Returns (ln kappa, sign of the ratio).
    """
    TL, TR, BL, BR = 2, 3, 0, 1
    E = envs
    c1, c2, c3, c4 = E[TL]["C1"], E[TR]["C2"], E[BR]["C3"], E[BL]["C4"]
    t1a, t1b = E[TL]["T1"], E[TR]["T1"]
    t2a, t2b = E[TR]["T2"], E[BR]["T2"]
    t3a, t3b = E[BR]["T3"], E[BL]["T3"]
    t4a, t4b = E[BL]["T4"], E[TL]["T4"]
    z00 = np.einsum("ab,bc,cd,da->", c1, c2, c3, c4, optimize=PAIRWISE)
    z20 = np.einsum("ab,buUc,cvVe,ef,fg,gvVh,huUk,ka->",
                    c1, t1a, t1b, c2, c3, t3a, t3b, c4, optimize=True)
    z02 = np.einsum("ab,bc,crRd,dsSe,ef,fg,gsSh,hrRa->",
                    c1, c2, t2a, t2b, c3, c4, t4a, t4b, optimize=True)
    # Z_22 is the closed network of the block with its environment: the
    # half systems of the cut between rows 0 and 1 at column 0 (the same
    # four sites and environment tensors) give it as Tr(H_u^T H_d)
    Hu, Hd = half_systems(*cut_corners(envs, As, 0, 0, 2, 2))
    z22 = float(np.sum(Hu * Hd))
    ratio = z22 * z00 / (z20 * z02)
    return 0.25 * float(np.log(abs(ratio))), float(np.sign(ratio))
