"""Parity of the CUDA CTMRG with the oracle's converged results at the larger
sizes: the precision workload (d=2, D=6, chi=72, N = 2592) and the D = 8
workload at chi = 32 (d=3, N = 2048).  The expected values were written by
tests/golden/make_ctmrg_goldens.py, which runs only the CPU oracle.

Both run through the randomised, warm-started range finder (N above the
exact-SVD limit) and the persistent QR, on multi-tile GEMMs.  The GPU runs
more sweeps than the oracle needed; past the fixed point extra sweeps change
nothing gauge-invariant.  Bars: FP64 -- every observable and every RDM entry
to 1e-10, ln kappa to 1e-10 relative, the loop spectra (the gauge-invariant
normalised corner spectra) to 1e-9; emulated FP64 (5 BF16 slices) -- every
observable within 1e-8 of the oracle, the loop spectra within 1e-8.
"""
import json
import os

import numpy as np
import pytest

from paper_2112_13184_gb300 import inputs as I
import invariants as INV

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_13184_gb300 import ctm as m
    return m


def case(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        g = json.load(f)
    if name == "neel_d2_D6_chi72":
        w = I.workload(name)
        return g, w["As"], w["envs"], w["d"], w["D"], w["chi"], w["op1"], w["op2"]
    d, D, chi = 3, 8, 32
    As = I.x_polarised_tensors(d, D, 0.05, seed=3)
    envs = I.random_env(chi, [D] * 4, seed=4)
    return g, As, envs, d, D, chi, I.spin_ops(3)["Sx"], I.blbq_bond(3, 1.0, 0.1)


def run_gpu(ctm, name, precision, sweeps):
    """Sweeps until the gauge-invariant loop moments change by < 1e-12 per
    sweep (FP64; 1e-10 emulated) or `sweeps` are done."""
    g, As, envs, d, D, chi, op1, op2 = case(name)
    prec = ctm.CTM_OZAKI_BF16 if precision == "mixed" else ctm.CTM_FP64
    c = ctm.CTMRG(d, D, chi, precision=prec, conv_measure=1, max_sweeps=sweeps,
                  tol=1e-12 if precision == "fp64" else 1e-10)
    c.set_tensors(As)
    c.set_envs(envs)
    st, n, delta = c.run()
    print(f"{name} {precision}: {n} sweeps, loop-moment change {delta:.1e}")
    obs = np.array([c.measure1(i, op1) for i in range(4)]
                   + [c.measure2(i, dx, dy, op2) for (i, dx, dy) in I.SQUARE_2X2_BONDS])
    out = dict(obs=obs, loop=INV.loop_spectra(c.get_envs()), lnk=c.log_norm_per_site(),
               rdm1=[c.rdm1(i) for i in range(4)],
               rdm2=[c.rdm2(i, dx, dy) for (i, dx, dy) in I.SQUARE_2X2_BONDS])
    c.close()
    return g, out


CASES = [("neel_d2_D6_chi72", 150), ("xpol_d3_D8_chi32", 100)]


@pytest.mark.parametrize("name,sweeps", CASES)
def test_golden_fp64(ctm, name, sweeps):
    g, out = run_gpu(ctm, name, "fp64", sweeps)
    ref = np.array(g["observables"])
    err = np.abs(out["obs"] - ref) / np.maximum(np.abs(ref), 1e-3)
    print(f"{name} FP64: max rel |dO| {err.max():.2e}, loop {np.abs(out['loop'] - g['loop_spectra']).max():.2e}")
    assert err.max() < 1e-10, (out["obs"], ref)
    # Hermitian observables see the symmetric part of rho, held to 1e-10;
    # the ket/bra-antisymmetric part the randomised range finder leaves at a
    # cut with a small gap at chi (1e-4 relative at one cut of the precision
    # workload) is bounded separately
    for a, b in zip(out["rdm1"] + out["rdm2"], g["rdm1"] + g["rdm2"]):
        b = np.array(b)
        np.testing.assert_allclose(0.5 * (a + a.T), 0.5 * (b + b.T), atol=1e-10, rtol=0)
        assert np.max(np.abs(a - a.T)) < 1e-8
    np.testing.assert_allclose(out["loop"], np.array(g["loop_spectra"]), atol=1e-9, rtol=0)
    np.testing.assert_allclose(out["lnk"], g["log_kappa_per_site"], rtol=1e-10)


@pytest.mark.parametrize("name,sweeps", CASES)
def test_golden_emulated_fp64(ctm, name, sweeps):
    g, out = run_gpu(ctm, name, "mixed", sweeps)
    err = np.abs(out["obs"] - np.array(g["observables"]))
    print(f"{name} emulated FP64 (5 slices): |dO| per observable vs the oracle {err}")
    assert err.max() <= 1e-8, err
    np.testing.assert_allclose(out["loop"], np.array(g["loop_spectra"]), atol=1e-8, rtol=0)


def run_scheme(ctm, name, precision, slices, sweeps, tol, refine=0):
    g, As, envs, d, D, chi, op1, op2 = case(name)
    c = ctm.CTMRG(d, D, chi, precision=precision, ozaki_slices=slices, conv_measure=1, max_sweeps=sweeps,
                  tol=tol, fp64_refine=refine)
    c.set_tensors(As)
    c.set_envs(envs)
    st, n, delta = c.run()
    obs = np.array([c.measure1(i, op1) for i in range(4)]
                   + [c.measure2(i, dx, dy, op2) for (i, dx, dy) in I.SQUARE_2X2_BONDS])
    loop = INV.loop_spectra(c.get_envs())
    c.close()
    return g, n, delta, obs, loop


# (label, precision constant name, slices, bound on |dO| and on the loop
# spectra).  Measured on a GB300 (max |dO|): split-BF16 9.2e-6, 3xTF32
# 2.4e-5, emulated FP64 with 3 / 4 / 6 slices 1.4e-6 / 1.4e-8 / 4.0e-10; the
# bounds leave a factor of 4 to 10.  The FP32-summed schemes stall at a loop-
# moment change near 1e-5, the fixed point of FP32 rounding of sums over K up
# to chi D^2.
SCHEMES = [("split-BF16 (3 slices, FP32 sums)", "CTM_SPLIT_BF16", 3, 1e-4),
           ("3xTF32 (FP32 sums)", "CTM_3XTF32", 2, 1e-4),
           ("emulated FP64, 3 slices", "CTM_OZAKI_BF16", 3, 1e-5),
           ("emulated FP64, 4 slices", "CTM_OZAKI_BF16", 4, 1e-7),
           ("emulated FP64, 6 slices", "CTM_OZAKI_BF16", 6, 4e-9)]


@pytest.mark.parametrize("label,pname,slices,bound", SCHEMES)
def test_golden_precision_schemes(ctm, label, pname, slices, bound):
    """Error of every observable of the precision workload (d=2, D=6,
    chi=72) against the oracle, per contraction scheme, after up to 150
    sweeps with the loop-moment stopping rule at 1e-10."""
    g, n, delta, obs, loop = run_scheme(ctm, "neel_d2_D6_chi72", getattr(ctm, pname), slices, 150, 1e-10)
    err = np.abs(obs - np.array(g["observables"]))
    lerr = np.abs(loop - np.array(g["loop_spectra"])).max()
    print(f"SCHEME {label}: {n} sweeps, loop-moment change {delta:.1e}, max |dO| {err.max():.2e} "
          f"(site {err[:4].max():.2e}, bond {err[4:].max():.2e}), loop spectra {lerr:.2e}")
    assert err.max() <= bound and lerr <= bound


def test_split_bf16_with_fp64_refine(ctm):
    """split-BF16 until its loop-moment change falls below 1e-4, then FP64
    to 1e-12: the observables reach the FP64 bar of the oracle."""
    g, n, delta, obs, loop = run_scheme(ctm, "neel_d2_D6_chi72", ctm.CTM_SPLIT_BF16, 3, 150, 1e-12, refine=1)
    err = np.abs(obs - np.array(g["observables"]))
    print(f"split-BF16 + FP64 refinement: {n} sweeps, max |dO| {err.max():.2e}")
    assert err.max() < 1e-9
    np.testing.assert_allclose(loop, np.array(g["loop_spectra"]), atol=1e-9, rtol=0)
