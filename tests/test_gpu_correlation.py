"""Correlation functions and the transfer-matrix spectrum on the GPU against
the oracle (paper Sec. 5.3) on the same environments.

Every environment here is the oracle's (a few or many CPU sweeps from a
seeded start); the GPU handle receives it through ctm_set_env, so the
comparison isolates ctm_correlation / ctm_transfer_spectrum.  Cases: the
decoupled-chain states (exact infinite-MPS values, sites all different),
the Neel workload d=2, D=3, chi=16 (N = 144) and a d=2, D=4, chi=24 case
(N = 384, strip vectors of 9216 entries) after 3 oracle sweeps.  Bars:
FP64 1e-11 relative on C, emulated FP64 (5 slices) 1e-9; the first four
eigenvalue ratios to 1e-9 (block iteration stopped at a change < 1e-12,
1e-10 emulated).
The small eigenvalue kernel is checked against numpy on random matrices
with complex pairs and clustered moduli.
"""
import numpy as np
import pytest

from oracle import correlation_ref as CR
from oracle import ctmrg_ref as R
from paper_2112_13184_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SX = np.array([[0.0, 1.0], [1.0, 0.0]])
SZ = np.diag([1.0, -1.0])


@pytest.fixture(scope="module")
def ctm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_13184_gb300 import ctm as m
    return m


def match_eigs(got, ref, conj=False):
    """Largest distance between each reference eigenvalue and a distinct
    nearest computed one (the order within equal moduli is arbitrary).
    conj: a real matrix's spectrum is closed under conjugation, and a list
    cut at nev may hold either member of a pair, so z and conj(z) match."""
    got = list(got)
    worst = 0.0
    for z in ref:
        dist = [min(abs(z - g), abs(np.conj(z) - g)) if conj else abs(z - g) for g in got]
        j = int(np.argmin(dist))
        worst = max(worst, dist[j])
        got.pop(j)
    return worst


@pytest.mark.parametrize("m", [1, 2, 3, 5, 8, 12, 16, 24, 32])
@pytest.mark.parametrize("kind", ["random", "rotations", "clustered"])
def test_small_eig_vs_numpy(ctm, m, kind):
    rng = np.random.default_rng(m + 100 * len(kind))
    if kind == "random":
        H = rng.standard_normal((m, m))
    elif kind == "rotations":
        # block diagonal 2x2 rotations (complex pairs of equal modulus), similar-transformed
        B = np.zeros((m, m))
        for k in range(0, m - 1, 2):
            r, t = rng.uniform(0.2, 2.0), rng.uniform(0, np.pi)
            B[k:k + 2, k:k + 2] = r * np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
        if m % 2:
            B[-1, -1] = rng.uniform(-1, 1)
        S = np.eye(m) + 0.3 * rng.standard_normal((m, m))
        H = S @ B @ np.linalg.inv(S)
    else:
        # a transfer-matrix-like spectrum: one dominant eigenvalue, then a
        # slowly decaying cluster
        lam = np.concatenate([[1.0], 0.3 * 0.97 ** np.arange(m - 1)])
        S = np.eye(m) + 0.2 * rng.standard_normal((m, m))
        H = S @ np.diag(lam) @ np.linalg.inv(S)
    Hd = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    out = torch.zeros(4 * m, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctm.ctm_small_eig(Hd, m, m, 2.0, out, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    o = out.cpu().numpy()
    ref = np.linalg.eigvals(H)
    ref = ref[np.argsort(-np.abs(ref), kind="stable")]
    scale = np.abs(ref[0])
    np.testing.assert_allclose(o[2 * m:3 * m], np.abs(ref), rtol=0, atol=1e-11 * max(1.0, scale) * m)
    # the ratios lambda_i / lambda_0: lambda_0 is any eigenvalue of largest
    # modulus (a complex pair, or +-r), so take the best candidate
    got = o[:m] + 1j * o[m:2 * m]
    cands = [z for z in ref if abs(abs(z) - scale) <= 1e-9 * scale]
    assert min(match_eigs(got, ref / z0) for z0 in cands) < 1e-8 * m
    with np.errstate(divide="ignore"):
        e = -np.log(np.abs(ref) / np.abs(ref[0])) / 2.0
    fin = np.isfinite(e)
    np.testing.assert_allclose(o[3 * m:][fin], e[fin], rtol=1e-9, atol=1e-10)


def set_case(ctm, As, envs, d, D, chi, precision):
    c = ctm.CTMRG(d, D, chi, precision=precision)
    c.set_tensors(As)
    c.set_envs(envs)
    return c


@pytest.fixture(scope="module")
def cases():
    out = {}
    for axis in (0, 1):
        As, a = I.decoupled_chain_tensors(2, 3, seed=3 + axis, axis=axis)
        envs = I.random_env(6, [3] * 4, seed=9)
        envs, _, _ = R.run(As, envs, 6, 60, tol=0.0)
        out[f"chain{axis}"] = (As, envs, 2, 3, 6)
    w = I.workload("neel_d2_D3_chi16")
    envs, _, _ = R.run(w["As"], w["envs"], 16, 30, tol=0.0)
    out["neel_d2_D3_chi16"] = (w["As"], envs, 2, 3, 16)
    As = I.neel_tensors(2, 4, 0.1, seed=21)
    envs = I.random_env(24, [4] * 4, seed=22)
    envs, _, _ = R.run(As, envs, 24, 3, tol=0.0)
    out["neel_d2_D4_chi24"] = (As, envs, 2, 4, 24)
    return out


CASES = ["chain0", "chain1", "neel_d2_D3_chi16", "neel_d2_D4_chi24"]
_SPECTRA = {}


def oracle_spectrum(cases, name, direction, index):
    key = (name, direction, index)
    if key not in _SPECTRA:
        As, envs = cases[name][:2]
        _SPECTRA[key] = CR.transfer_spectrum(envs, As, direction, index, nev=4)
    return _SPECTRA[key]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_correlation_vs_oracle(ctm, cases, name, precision):
    As, envs, d, D, chi = cases[name]
    rmax = 5
    prec = ctm.CTM_OZAKI_BF16 if precision == "mixed" else ctm.CTM_FP64
    c = set_case(ctm, As, envs, d, D, chi, prec)
    got = c.correlation(SX, SZ, rmax)
    c.close()
    # |error| <= rtol |C| + atol: the emulated products' error follows the
    # operands' magnitudes, not the value (C(0) = <SX SZ> is 0 here).  The
    # D = 4 environment is three sweeps from random: its strips cancel
    # strongly, and the emulated bound 2^-36 K max|row| max|col| per product
    # (K up to N = 384) allows a few 1e-9 there (measured 2e-8 relative).
    if precision == "fp64":
        rtol, atol = 1e-11, 1e-14
    else:
        rtol, atol = (5e-8, 5e-9) if name == "neel_d2_D4_chi24" else (1e-9, 1e-10)
    for direction in (0, 1):
        ref = CR.correlation(envs, As, SX, SZ, rmax, direction)
        err = np.abs(got[direction] - ref)
        print(f"{name} {precision} dir {direction}: max |dC| {err.max():.2e}, "
              f"max |dC|/|C| over |C| > 1e-3 {np.max(err[np.abs(ref) > 1e-3] / np.abs(ref[np.abs(ref) > 1e-3])):.2e}")
        assert np.all(err <= rtol * np.abs(ref) + atol), (got[direction], ref)


@pytest.mark.parametrize("name", CASES[:3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_transfer_spectrum_vs_oracle(ctm, cases, name, precision):
    As, envs, d, D, chi = cases[name]
    prec = ctm.CTM_OZAKI_BF16 if precision == "mixed" else ctm.CTM_FP64
    c = set_case(ctm, As, envs, d, D, chi, prec)
    for direction in (0, 1):
        for index in (0, 1):
            # the emulated products leave a change of ~1e-11 per iteration
            ratio, mod, e, it, ch, st = c.transfer_spectrum(direction, index, nev=4, block=10, max_iter=400,
                                                            tol=1e-12 if precision == "fp64" else 1e-10)
            ref, e_ref, _ = oracle_spectrum(cases, name, direction, index)
            print(f"{name} {precision} dir {direction} index {index}: {it} iterations, change {ch:.1e}, "
                  f"|ratio| {np.abs(ratio)}")
            assert st == ctm.CTM_OK
            np.testing.assert_allclose(np.abs(ratio), np.abs(ref), atol=1e-9)
            assert match_eigs(ratio, ref, conj=True) < 1e-8
    c.close()


def test_correlation_rmax_zero_and_errors(ctm, cases):
    As, envs, d, D, chi = cases["neel_d2_D3_chi16"]
    c = set_case(ctm, As, envs, d, D, chi, ctm.CTM_FP64)
    got = c.correlation(SZ, SZ, 0)
    for direction in (0, 1):
        ref = CR.correlation(envs, As, SZ, SZ, 0, direction)
        np.testing.assert_allclose(got[direction], ref, rtol=1e-12)
    with pytest.raises(RuntimeError):
        ctm.ctm_correlation(c.h, SZ, SZ, -1)
    with pytest.raises(RuntimeError):
        c.transfer_spectrum(2, 0)
    with pytest.raises(RuntimeError):
        c.transfer_spectrum(0, 0, nev=4, block=40)
    c.close()
