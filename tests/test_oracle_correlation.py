"""Pins of the oracle's correlation functions and transfer-matrix spectrum
(paper Sec. 5.3, correlation and correlation_length).

  * the strip primitives against the whole strip network written out as one
    contraction (brute force on tiny random tensors), along x and y;
  * the dense period transfer matrix against its trace identities
    Tr(T) and Tr(T^2) = the ring networks of one and two periods;
  * rows that decouple into infinite matrix-product states (vertical legs
    carry only index 0): C along x equals the textbook infinite-MPS value
    built from the MPS transfer matrix E = sum_s a^s (x) a^s, C along y
    factorises, and the transfer-matrix eigenvalue ratios are those of
    E_(0,y) E_(1,y) (numpy eigvals of a D^2 x D^2 matrix);
  * the Ising network: C(1) = Onsager's nearest-neighbour correlation,
    C(r) -> M^2 (Yang) deep in the ordered phase, C_x = C_y, and the same
    values for the bond-gauged Ising tensors whose four sites all differ;
    the CTMRG correlation length lies below the exact axial one and within
    10% of it (the finite-chi transfer matrix resolves the edge of the
    Ornstein-Zernike continuum only as chi -> infinity);
  * a product state: C(r >= 1) = <A><B>, lambda_1 = 0.
"""
import math

import numpy as np
import pytest

from oracle import correlation_ref as CR
from oracle import ctmrg_ref as R
from oracle import exact as X
from paper_2112_13184_gb300 import inputs as I

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.diag([1.0, -1.0])


def random_case(chi=3, D=2, d=2, seed=0):
    rng = np.random.default_rng(seed)
    As = [rng.standard_normal((d, D, D, D, D)) for _ in range(4)]
    envs = I.random_env(chi, [D] * 4, seed=seed + 1, per_site=True)
    return As, envs


def brute_strip_x(envs, As, ops, x0, y0):
    """Three sites along +x from (x0, y0), every tensor listed once, one
    contraction with integer leg labels."""
    sites = [I.site_index(x0 + j, y0) for j in range(3)]
    L = iter(range(1000))
    b = [next(L) for _ in range(4)]  # T1 chain
    m = [next(L) for _ in range(4)]  # T3 chain
    h = [next(L) for _ in range(4)]  # ket horizontal legs
    H = [next(L) for _ in range(4)]  # bra horizontal legs
    n, a_, e, f = next(L), next(L), next(L), next(L)
    e0, eL = envs[sites[0]], envs[sites[2]]
    args = [e0["C4"], [m[0], n], e0["T4"], [n, h[0], H[0], a_], e0["C1"], [a_, b[0]]]
    for j, s in enumerate(sites):
        u, U, dd, DD, sk, sb = (next(L) for _ in range(6))
        A = As[s] if ops[j] is None else np.einsum("ts,slurd->tlurd", ops[j], As[s])
        args += [envs[s]["T1"], [b[j], u, U, b[j + 1]], A, [sk, h[j], u, h[j + 1], dd],
                 As[s], [sk, H[j], U, H[j + 1], DD], envs[s]["T3"], [m[j + 1], dd, DD, m[j]]]
    args += [eL["C2"], [b[3], e], eL["T2"], [e, h[3], H[3], f], eL["C3"], [f, m[3]]]
    return float(np.einsum(*args, [], optimize=("greedy", 1 << 40)))


def brute_strip_y(envs, As, ops, x0, y0):
    sites = [I.site_index(x0, y0 + j) for j in range(3)]
    L = iter(range(1000))
    w = [next(L) for _ in range(4)]  # T4 chain
    e = [next(L) for _ in range(4)]  # T2 chain
    v = [next(L) for _ in range(4)]  # ket vertical legs
    V = [next(L) for _ in range(4)]  # bra vertical legs
    m, g, bb, c = next(L), next(L), next(L), next(L)
    e0, eT = envs[sites[0]], envs[sites[2]]
    args = [e0["C4"], [m, w[0]], e0["T3"], [g, v[0], V[0], m], e0["C3"], [e[0], g]]
    for j, s in enumerate(sites):
        l, Lb, r, Rb, sk = (next(L) for _ in range(5))
        A = As[s] if ops[j] is None else np.einsum("ts,slurd->tlurd", ops[j], As[s])
        args += [envs[s]["T4"], [w[j], l, Lb, w[j + 1]], A, [sk, l, v[j + 1], r, v[j]],
                 As[s], [sk, Lb, V[j + 1], Rb, V[j]], envs[s]["T2"], [e[j + 1], r, Rb, e[j]]]
    args += [eT["C1"], [w[3], bb], eT["T1"], [bb, v[3], V[3], c], eT["C2"], [c, e[3]]]
    return float(np.einsum(*args, [], optimize=("greedy", 1 << 40)))


@pytest.mark.parametrize("x0,y0", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_strips_match_brute_force(x0, y0):
    As, envs = random_case(seed=3 + x0 + 2 * y0)
    ops = [SX, None, SZ]
    vx = CR.strip_value(envs, As, ops, 0, x0, y0)
    vy = CR.strip_value(envs, As, ops, 1, x0, y0)
    assert vx == pytest.approx(brute_strip_x(envs, As, ops, x0, y0), rel=1e-12)
    assert vy == pytest.approx(brute_strip_y(envs, As, ops, x0, y0), rel=1e-12)


def ring_trace(envs, As, direction, index, periods):
    """Tr(T^periods): the strip of `periods` cell periods closed on itself
    (edge-tensor chains and the site legs along the strip wrap around)."""
    if direction == 0:
        cols = [I.site_index(x, index) for x in range(2)] * periods
    else:
        cols = [I.site_index(index, y) for y in range(2)] * periods
    n = len(cols)
    L = iter(range(1000))
    p = [next(L) for _ in range(n)]   # chain above (x) / left (y)
    q = [next(L) for _ in range(n)]   # chain below / right
    h = [next(L) for _ in range(n)]   # ket legs along the strip
    H = [next(L) for _ in range(n)]
    args = []
    for j, s in enumerate(cols):
        jn = (j + 1) % n
        a1, A1, a2, A2, sk = (next(L) for _ in range(5))
        e = envs[s]
        if direction == 0:
            args += [e["T1"], [p[j], a1, A1, p[jn]], As[s], [sk, h[j], a1, h[jn], a2],
                     As[s], [sk, H[j], A1, H[jn], A2], e["T3"], [q[jn], a2, A2, q[j]]]
        else:
            args += [e["T4"], [p[j], a1, A1, p[jn]], As[s], [sk, a1, h[jn], a2, h[j]],
                     As[s], [sk, A1, H[jn], A2, H[j]], e["T2"], [q[jn], a2, A2, q[j]]]
    return float(np.einsum(*args, [], optimize=("greedy", 1 << 40)))


@pytest.mark.parametrize("direction,index", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_transfer_matrix_trace_identities(direction, index):
    As, envs = random_case(chi=2, D=2, seed=11 + index + 2 * direction)
    T = CR.transfer_matrix(envs, As, direction, index)
    assert np.trace(T) == pytest.approx(ring_trace(envs, As, direction, index, 1), rel=1e-11)
    assert np.trace(T @ T) == pytest.approx(ring_trace(envs, As, direction, index, 2), rel=1e-11)


# --------------------------------------------------------------------------
# decoupled rows: every row an infinite MPS
# --------------------------------------------------------------------------
def mps_E(a, op=None):
    d, D = a.shape[0], a.shape[1]
    op = np.eye(d) if op is None else op
    return np.einsum("ts,slr,tLR->lLrR", op, a, a).reshape(D * D, D * D)


def mps_correlation(a, y, x0, r, opA, opB, axis=0):
    """Infinite-MPS <A(x0) B(x0 + r)> along row y (axis 0: tensors
    a_(x mod 2, y)) or along column y (axis 1: a_(y, x mod 2))."""
    t = [a[I.site_index(x, y) if axis == 0 else I.site_index(y, x)] for x in range(2)]
    E = [mps_E(ti) for ti in t]

    def fixed(xs, left):
        T = E[xs % 2] @ E[(xs + 1) % 2]
        w, v = np.linalg.eig(T.T if left else T)
        return np.real(v[:, np.argmax(np.abs(w))])

    vL, vR = fixed(x0, True), fixed(x0 + r + 1, False)
    if r == 0:
        return (vL @ mps_E(t[x0 % 2], opA @ opB) @ vR) / (vL @ E[x0 % 2] @ vR)
    num, den = mps_E(t[x0 % 2], opA), E[x0 % 2]
    for j in range(1, r + 1):
        xj = (x0 + j) % 2
        num = num @ (mps_E(t[xj], opB) if j == r else E[xj])
        den = den @ E[xj]
    return (vL @ num @ vR) / (vL @ den @ vR)


@pytest.fixture(scope="module", params=[0, 1], ids=["rows", "columns"])
def mps_chains(request):
    axis = request.param
    As, a = I.decoupled_chain_tensors(2, 3, seed=3 + axis, axis=axis)
    envs = I.random_env(6, [3] * 4, seed=9)
    # fixed sweep count: the corners are rank one here, so their spectra do
    # not move while the edge tensors still converge
    envs, _, _ = R.run(As, envs, 6, 60, tol=0.0)
    return axis, As, a, envs


def test_decoupled_chains_correlation_along(mps_chains):
    axis, As, a, envs = mps_chains
    C = CR.correlation(envs, As, SX, SZ, 6, axis)
    for i in range(4):
        x, y = i % 2, i // 2
        along, across = (x, y) if axis == 0 else (y, x)
        ref = [mps_correlation(a, across, along, r, SX, SZ, axis) for r in range(7)]
        np.testing.assert_allclose(C[i], ref, rtol=0, atol=1e-13)


def test_decoupled_chains_correlation_across_factorises(mps_chains):
    axis, As, a, envs = mps_chains
    C = CR.correlation(envs, As, SX, SZ, 4, 1 - axis)
    one = lambda op, i: R.expect(op, R.rdm1(envs, As, i))
    for i in range(4):
        x, y = i % 2, i // 2
        for r in range(1, 5):
            j = I.site_index(x, y + r) if axis == 0 else I.site_index(x + r, y)
            assert C[i, r] == pytest.approx(one(SX, i) * one(SZ, j), abs=1e-13)
        assert C[i, 0] == pytest.approx(R.expect(SX @ SZ, R.rdm1(envs, As, i)), abs=1e-13)


@pytest.mark.parametrize("index", [0, 1])
def test_decoupled_chains_transfer_spectrum(mps_chains, index):
    axis, As, a, envs = mps_chains
    ratio, e, xi = CR.transfer_spectrum(envs, As, axis, index, nev=6)
    sites = [I.site_index(x, index) if axis == 0 else I.site_index(index, x) for x in range(2)]
    T = mps_E(a[sites[0]]) @ mps_E(a[sites[1]])
    lam = np.linalg.eigvals(T)
    lam = lam[np.argsort(-np.abs(lam), kind="stable")][:6]
    np.testing.assert_allclose(np.abs(ratio), np.abs(lam / lam[0]), atol=1e-11)
    # the complex pairs too (each pair's order within equal moduli aside)
    np.testing.assert_allclose(np.sort_complex(ratio), np.sort_complex(lam / lam[0]), atol=1e-11)
    assert xi == pytest.approx(2.0 / -np.log(np.abs(lam[1] / lam[0])), rel=1e-10)
    # across the chains the lattice is a product of uncorrelated chains:
    # one eigenvalue only
    ratio_x, _, _ = CR.transfer_spectrum(envs, As, 1 - axis, index, nev=3)
    assert np.max(np.abs(ratio_x[1:])) < 1e-12


# --------------------------------------------------------------------------
# Ising network
# --------------------------------------------------------------------------
def ising_env(As, beta, chi=8, sweeps=80):
    envs = I.random_env(chi, [2] * 4, seed=5)
    envs, _, _ = R.run(As, envs, chi, sweeps, tol=1e-13)
    return envs


@pytest.fixture(scope="module", params=[0.3, 0.6])
def ising(request):
    beta = request.param
    As = [I.ising_peps_tensor(beta)] * 4
    return beta, As, ising_env(As, beta)


def test_ising_correlation_closed_forms(ising):
    beta, As, envs = ising
    Cx = CR.correlation(envs, As, SZ, SZ, 24, 0)
    Cy = CR.correlation(envs, As, SZ, SZ, 24, 1)
    np.testing.assert_allclose(Cx, Cy, atol=1e-12)
    np.testing.assert_allclose(Cx[:, 0], 1.0, atol=1e-13)
    np.testing.assert_allclose(Cx[:, 1], X.onsager_nn_correlation(beta), atol=1e-10)
    if beta > X.K_CRITICAL:
        np.testing.assert_allclose(Cx[:, 24], X.yang_magnetisation(beta) ** 2, atol=1e-9)
    # connected correlations decay monotonically along the axis
    conn = Cx[0] - X.yang_magnetisation(beta) ** 2
    assert np.all(np.diff(conn[:12]) < 0)


def test_ising_correlation_length_below_exact(ising):
    beta, As, envs = ising
    K = beta
    Ks = 0.5 * math.log(1.0 / math.tanh(K))  # dual coupling, tanh K* = e^-2K
    # exact axial correlation length: 1/xi = 2 (K* - K) above T_c, twice
    # the single-particle gap, 4 (K - K*), below
    inv_exact = 2 * (Ks - K) if K < X.K_CRITICAL else 4 * (K - Ks)
    for direction in (0, 1):
        _, e, xi = CR.transfer_spectrum(envs, As, direction, 0, nev=3)
        assert 1.0 / xi > inv_exact
        assert 1.0 / xi < 1.1 * inv_exact


def test_gauged_ising_correlations_equal():
    """Gauged and plain Ising tensors at chi = 8, beta = 0.3.  The bond
    gauges act on the D legs crossing each cut as non-orthogonal maps, which
    change the singular values of M = H_u^T H_d and so the subspace the
    truncation keeps: the environments agree only to the truncation error
    (3e-9 at chi = 8, 4e-8 at chi = 5), and the subleading transfer-matrix
    eigenvalues, which resolve the edge of a continuum, to 1e-3.  (At beta =
    0.6 the gauged iteration stalls near 1e-5 above chi = 3, the noise floor
    the gauged Onsager pins avoid by running at chi = 3.)"""
    beta = 0.3
    As = [I.ising_peps_tensor(beta)] * 4
    envs = ising_env(As, beta)
    Cref = CR.correlation(envs, As, SZ, SZ, 6, 0)
    Ag = I.gauged_ising_tensors(beta, seed=7, strength=0.3)
    envs_g = ising_env(Ag, beta)
    for direction in (0, 1):
        C = CR.correlation(envs_g, Ag, SZ, SZ, 6, direction)
        np.testing.assert_allclose(C, Cref, atol=1e-8, rtol=0)
    _, e_ref, _ = CR.transfer_spectrum(envs, As, 0, 0, nev=3)
    _, e_g, _ = CR.transfer_spectrum(envs_g, Ag, 0, 1, nev=3)
    np.testing.assert_allclose(e_g, e_ref, rtol=1e-3)


def test_product_state():
    d, D, chi = 2, 2, 4
    phis = [np.array([1.0, 0.5]), np.array([0.3, 1.0]), np.array([1.0, -0.2]), np.array([0.6, 0.8])]
    As = []
    for ph in phis:
        A = np.zeros((d, D, D, D, D))
        A[:, 0, 0, 0, 0] = ph
        As.append(A)
    envs = I.random_env(chi, [D] * 4, seed=2)
    envs, _, _ = R.run(As, envs, chi, 10, tol=0.0)
    for direction in (0, 1):
        C = CR.correlation(envs, As, SX, SZ, 3, direction)
        for i in range(4):
            x, y = i % 2, i // 2
            for r in range(1, 4):
                j = I.site_index(x + (r if direction == 0 else 0), y + (r if direction == 1 else 0))
                ref = X.product_expectation(phis[i], SX) * X.product_expectation(phis[j], SZ)
                assert C[i, r] == pytest.approx(ref, abs=1e-13)
        ratio, _, _ = CR.transfer_spectrum(envs, As, direction, 0, nev=2)
        assert abs(ratio[1]) < 1e-12
