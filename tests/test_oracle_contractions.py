"""Pin every contraction of the oracle against brute force on tiny shapes.

Enlarged corners and absorption steps: explicit Python index loops over
every summed index.  Reduced density matrices and the free-energy networks:
networks generated from grid geometry (tests/netlist.py) and contracted by
a generic pairwise contractor.  Shapes are deliberately non-square
(d=2, D=2, chi=3) so that a transposed operand cannot pass.
"""
import itertools

import numpy as np
import pytest

from oracle import ctmrg_ref as R
from paper_2112_13184_gb300 import inputs as I
import netlist as NL

d, D, chi = 2, 2, 3


@pytest.fixture(scope="module")
def state():
    rng = np.random.default_rng(123)
    As = [rng.standard_normal((d, D, D, D, D)) for _ in range(4)]
    envs = I.random_env(chi, [D] * 4, seed=7)
    # break the k<->k' symmetry so a swapped ket/bra leg is detected
    for e in envs:
        for n in ("T1", "T2", "T3", "T4"):
            e[n] = e[n] + 0.3 * rng.standard_normal(e[n].shape)
    return As, envs


def loops_ul(C1, T1, T4, A):
    N = chi * D * D
    Q = np.zeros((N, N))
    for a, dd, dp, b, r, rp in itertools.product(range(chi), range(D), range(D),
                                                 range(chi), range(D), range(D)):
        s_ = 0.0
        for g, h, u, up, l, lp, s in itertools.product(range(chi), range(chi), range(D), range(D),
                                                       range(D), range(D), range(d)):
            s_ += (C1[g, h] * T1[h, u, up, b] * T4[a, l, lp, g]
                   * A[s, l, u, r, dd] * A[s, lp, up, rp, dp])
        Q[(a * D + dd) * D + dp, (b * D + r) * D + rp] = s_
    return Q


def loops_ur(T1, C2, T2, A):
    N = chi * D * D
    Q = np.zeros((N, N))
    for b, l, lp, e, dd, dp in itertools.product(range(chi), range(D), range(D),
                                                 range(chi), range(D), range(D)):
        s_ = 0.0
        for g, h, u, up, r, rp, s in itertools.product(range(chi), range(chi), range(D), range(D),
                                                       range(D), range(D), range(d)):
            s_ += (T1[b, u, up, g] * C2[g, h] * T2[h, r, rp, e]
                   * A[s, l, u, r, dd] * A[s, lp, up, rp, dp])
        Q[(b * D + l) * D + lp, (e * D + dd) * D + dp] = s_
    return Q


def loops_br(T2, C3, T3, A):
    N = chi * D * D
    Q = np.zeros((N, N))
    for e, u, up, z, l, lp in itertools.product(range(chi), range(D), range(D),
                                                range(chi), range(D), range(D)):
        s_ = 0.0
        for g, h, r, rp, dd, dp, s in itertools.product(range(chi), range(chi), range(D), range(D),
                                                        range(D), range(D), range(d)):
            s_ += (T2[e, r, rp, g] * C3[g, h] * T3[h, dd, dp, z]
                   * A[s, l, u, r, dd] * A[s, lp, up, rp, dp])
        Q[(z * D + l) * D + lp, (e * D + u) * D + up] = s_
    return Q


def loops_bl(T4, C4, T3, A):
    N = chi * D * D
    Q = np.zeros((N, N))
    for a, u, up, z, r, rp in itertools.product(range(chi), range(D), range(D),
                                                range(chi), range(D), range(D)):
        s_ = 0.0
        for g, h, l, lp, dd, dp, s in itertools.product(range(chi), range(chi), range(D), range(D),
                                                        range(D), range(D), range(d)):
            s_ += (T4[g, l, lp, a] * C4[h, g] * T3[z, dd, dp, h]
                   * A[s, l, u, r, dd] * A[s, lp, up, rp, dp])
        Q[(a * D + u) * D + up, (z * D + r) * D + rp] = s_
    return Q


def test_enlarged_corners_vs_loops(state):
    As, envs = state
    e, A = envs[1], As[1]
    np.testing.assert_allclose(R.enlarged_ul(e["C1"], e["T1"], e["T4"], A),
                               loops_ul(e["C1"], e["T1"], e["T4"], A), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(R.enlarged_ur(e["T1"], e["C2"], e["T2"], A),
                               loops_ur(e["T1"], e["C2"], e["T2"], A), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(R.enlarged_br(e["T2"], e["C3"], e["T3"], A),
                               loops_br(e["T2"], e["C3"], e["T3"], A), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(R.enlarged_bl(e["T4"], e["C4"], e["T3"], A),
                               loops_bl(e["T4"], e["C4"], e["T3"], A), rtol=1e-12, atol=1e-12)


def test_loop_value_equals_block_network(state):
    """Tr(H_u^T H_d) = the closed network of the 2x2 block (geometry-built)."""
    As, envs = state
    for x, y in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        Qs = R.cut_corners(envs, As, x, y, 2, 2)
        Hu, Hd = R.half_systems(*Qs)
        z = np.trace(Hu.T @ Hd)
        zb = NL.contract(NL.block_network(envs, As, x, y, 2, 2), [])
        np.testing.assert_allclose(z, zb, rtol=1e-11)


def test_absorb_vs_loops(state):
    As, envs = state
    rng = np.random.default_rng(5)
    N = chi * D * D
    Pup = rng.standard_normal((N, chi))
    Pup2 = rng.standard_normal((N, chi))
    Pdn = rng.standard_normal((chi, N))
    e, A = envs[2], As[2]
    C1, T1, T4, C4, T3 = e["C1"], e["T1"], e["T4"], e["C4"], e["T3"]
    # C1'
    ref = np.zeros((chi, chi))
    for c, b in itertools.product(range(chi), range(chi)):
        for g, h, u, up in itertools.product(range(chi), range(chi), range(D), range(D)):
            ref[c, b] += Pup[(g * D + u) * D + up, c] * C1[g, h] * T1[h, u, up, b]
    np.testing.assert_allclose(R.absorb_C1(C1, T1, Pup), ref, rtol=1e-12, atol=1e-13)
    # C4'
    ref = np.zeros((chi, chi))
    for z, c in itertools.product(range(chi), range(chi)):
        for g, h, dd, dp in itertools.product(range(chi), range(chi), range(D), range(D)):
            ref[z, c] += C4[h, g] * T3[z, dd, dp, h] * Pdn[c, (g * D + dd) * D + dp]
    np.testing.assert_allclose(R.absorb_C4(C4, T3, Pdn), ref, rtol=1e-12, atol=1e-13)
    # T4'
    ref = np.zeros((chi, D, D, chi))
    for c1, r, rp, c2 in itertools.product(range(chi), range(D), range(D), range(chi)):
        acc = 0.0
        for ab, dd, dp, at, u, up, l, lp, s in itertools.product(
                range(chi), range(D), range(D), range(chi), range(D), range(D), range(D), range(D), range(d)):
            acc += (Pup2[(ab * D + dd) * D + dp, c1] * T4[ab, l, lp, at]
                    * A[s, l, u, r, dd] * A[s, lp, up, rp, dp] * Pdn[c2, (at * D + u) * D + up])
        ref[c1, r, rp, c2] = acc
    np.testing.assert_allclose(R.absorb_T4(T4, A, Pup2, Pdn), ref, rtol=1e-11, atol=1e-12)


def test_rdm1_vs_network(state):
    As, envs = state
    for i in range(4):
        x, y = i % 2, i // 2
        rho = NL.contract(NL.block_network(envs, As, x, y, 1, 1, open_sites=(i,)),
                          [("ket", i), ("bra", i)])
        np.testing.assert_allclose(R.rdm1(envs, As, i), rho / np.trace(rho), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("i,dx,dy", [(0, 1, 0), (1, 1, 0), (2, 1, 0), (3, 1, 0),
                                     (0, 0, 1), (1, 0, 1), (2, 0, 1), (3, 0, 1)])
def test_rdm2_vs_network(state, i, dx, dy):
    As, envs = state
    x, y = i % 2, i // 2
    j = ((x + dx) % 2) + 2 * ((y + dy) % 2)
    net = NL.block_network(envs, As, x, y, 1 + dx, 1 + dy, open_sites=(i, j))
    rho = NL.contract(net, [("ket", i), ("ket", j), ("bra", i), ("bra", j)]).reshape(d * d, d * d)
    np.testing.assert_allclose(R.rdm2(envs, As, i, dx, dy), rho / np.trace(rho), rtol=1e-10, atol=1e-12)


def test_rdm2_negative_offsets_are_swaps(state):
    As, envs = state
    # source 1, target to its left = site 0: same pair as (0, +1, 0) with sites swapped
    r = R.rdm2(envs, As, 1, -1, 0).reshape(d, d, d, d)
    r0 = R.rdm2(envs, As, 0, 1, 0).reshape(d, d, d, d)
    # site 1's left neighbour is 0 and (by periodicity) also its right neighbour,
    # but the bond 1->0 leftwards is the bond 0->1 rightwards
    np.testing.assert_allclose(r, r0.transpose(1, 0, 3, 2), rtol=1e-12)


def test_log_kappa_networks(state):
    As, envs = state
    z22 = NL.contract(NL.block_network(envs, As, 0, 0, 2, 2), [])
    z20 = NL.contract(NL.row_strip(envs, 0, 2, 0, 1), [])
    z02 = NL.contract(NL.column_strip(envs, 0, 1, 0, 2), [])
    z00 = NL.contract(NL.corners_only(envs, 0, 1, 0, 1), [])
    ratio = z22 * z00 / (z20 * z02)
    lk, sg = R.log_kappa_per_site(envs, As)
    assert sg == np.sign(ratio)
    np.testing.assert_allclose(lk, 0.25 * np.log(abs(ratio)), rtol=1e-11)


def test_double_layer_definition():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((2, 2, 3, 2, 2))
    a = R.double_layer(A)
    ref = np.zeros(a.shape)
    for l, L, u, U, r, Rr, dd, DD in itertools.product(range(2), range(2), range(3), range(3),
                                                       range(2), range(2), range(2), range(2)):
        ref[l * 2 + L, u * 3 + U, r * 2 + Rr, dd * 2 + DD] = sum(
            A[s, l, u, r, dd] * A[s, L, U, Rr, DD] for s in range(2))
    np.testing.assert_allclose(a, ref, rtol=1e-13)


def test_rotation_is_a_4_cycle(state):
    As, envs = state
    e, a, lx, ly = envs, As, 2, 2
    for _ in range(4):
        e, a, lx, ly = R.rotate_ccw(e, a, lx, ly)
    for i in range(4):
        np.testing.assert_array_equal(a[i], As[i])
        for n in R.ENV_NAMES:
            np.testing.assert_array_equal(e[i][n], envs[i][n])


def test_rotation_maps_vertical_to_horizontal(state):
    """After a CCW rotation the vertical pair (i below j) becomes the
    horizontal pair (j left of i): same two-site RDM up to the site order."""
    As, envs = state
    e2, a2, _, _ = R.rotate_ccw(envs, As, 2, 2)
    i, j = 0, 2                # (0,0) and its top neighbour (0,1)
    # (x,y)->(-y,x): (0,0)->(0,0) = 0, (0,1)->(1,0) = 1 ; top -> left
    rv = R.rdm2(envs, As, i, 0, 1)
    rh = R.rdm2(e2, a2, 1, 1, 0)   # site 1 (image of j) left of site 0 (image of i)
    np.testing.assert_allclose(rv, R.swap_sites(rh, d, d), rtol=1e-11, atol=1e-13)


def test_loop_spectra_vs_network(state):
    """loop_spectra: the corner loop of each 2x2 block, built here from the
    grid geometry with the closing bond left open, has the same eigenvalue
    moduli."""
    As, envs = state
    for i in range(4):
        x, y = i % 2, i // 2
        net = NL.corners_only(envs, x, x + 1, y, y + 1)
        net[3] = (net[3][0], [("B",), ("L'",)])      # open the bond C4 -> C1
        L = NL.contract(net, [("L",), ("L'",)])
        m = np.sort(np.abs(np.linalg.eigvals(L)))[::-1]
        np.testing.assert_allclose(R.loop_spectra(envs)[i], m / m.sum(), rtol=1e-10, atol=1e-14)


def test_test_side_loop_spectra_match_oracle(state):
    """The tests' own loop-spectrum helper (applied to GPU environments)
    computes the oracle's definition."""
    import invariants as INV
    As, envs = state
    np.testing.assert_allclose(INV.loop_spectra(envs), R.loop_spectra(envs), rtol=1e-12, atol=1e-15)
