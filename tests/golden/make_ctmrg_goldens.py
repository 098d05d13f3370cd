#!/usr/bin/env python
"""Write the oracle's converged CTMRG results for the larger parity cases.

Every value written here comes from the CPU oracle (``oracle/``) run on the
seeded inputs of ``paper_2112_13184_gb300.inputs``; nothing comes from the
CUDA path.  The GPU parity tests (tests/test_gpu_goldens.py) compare the
library's results with these files.

Cases
  neel_d2_D6_chi72   d=2, D=6, chi=72 (N = chi D^2 = 2592): Neel + 0.1 N(0,1)
                     (seed 2), environment seed 3; S^z per site and the
                     S=1/2 Heisenberg bond energy on the 8 bonds.
  xpol_d3_D8_chi32   d=3, D=8, chi=32 (N = 2048): S=1 polarised along +x +
                     0.05 N(0,1) (seed 3), environment seed 4 -- the D = 8
                     workload at a chi the oracle's dense O(N^3) projectors
                     can afford; S^x per site and J S.S + 0.1 (S.S)^2.

Each case runs directional CTMRG sweeps (Sec. 2.2) until the gauge-invariant
loop spectra (eigenvalues of the corner loop around each 2x2 block; the
singular values of single corners move with the chi-bond gauge the
projectors leave) change by less than 1e-12, or the sweep cap is reached, then
records: the per-sweep spectrum change, the one-site and two-site reduced
density matrices and observables (Sec. 5.3), the normalised corner spectra,
the gauge-invariant loop spectra, ln kappa per site, and the singular values
of M = H_u^T H_d around chi for the four cuts of the left move (the
truncation gap).

Usage:  python tests/golden/make_ctmrg_goldens.py CASE [--checkpoint DIR]
(BLAS threads as set by OMP_NUM_THREADS).  With --checkpoint the
environment is saved every 2 sweeps and a rerun resumes from it.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import ctmrg_ref as R  # noqa: E402
from paper_2112_13184_gb300 import inputs as I  # noqa: E402

CASES = {
    "neel_d2_D6_chi72": dict(max_sweeps=100, tol=1e-12),
    "xpol_d3_D8_chi32": dict(max_sweeps=100, tol=1e-12),
}


def case_inputs(name):
    if name == "neel_d2_D6_chi72":
        w = I.workload(name)
        return w["As"], w["envs"], w["chi"], w["op1"], w["op2"]
    if name == "xpol_d3_D8_chi32":
        d, D, chi = 3, 8, 32
        As = I.x_polarised_tensors(d, D, 0.05, seed=3)
        envs = I.random_env(chi, [D] * 4, seed=4)
        return As, envs, chi, I.spin_ops(3)["Sx"], I.blbq_bond(3, 1.0, 0.1)
    raise KeyError(name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--checkpoint", default=None)
    args = ap.parse_args()
    cfg = CASES[args.case]
    As, envs, chi, op1, op2 = case_inputs(args.case)
    envs = [{k: v.copy() for k, v in e.items()} for e in envs]
    deltas, loop_deltas = [], []
    ck = os.path.join(args.checkpoint, args.case + ".npz") if args.checkpoint else None
    if ck and os.path.exists(ck):
        z = np.load(ck)
        deltas = list(z["deltas"])
        loop_deltas = list(z["loop_deltas"]) if "loop_deltas" in z else [float("inf")] * len(deltas)
        envs = [{n: z[f"{i}_{n}"] for n in R.ENV_NAMES} for i in range(4)]
        print(f"resumed at sweep {len(deltas)}", flush=True)
    prev = R.corner_spectra(envs)
    prev_loop = R.loop_spectra(envs)
    t0 = time.time()
    while len(deltas) < cfg["max_sweeps"] and not (loop_deltas and loop_deltas[-1] < cfg["tol"]):
        R.sweep(envs, As, 2, 2, chi)
        cur, cur_loop = R.corner_spectra(envs), R.loop_spectra(envs)
        deltas.append(float(np.max(np.abs(cur - prev))))
        loop_deltas.append(float(np.max(np.abs(cur_loop - prev_loop))))
        prev, prev_loop = cur, cur_loop
        print(f"sweep {len(deltas)} corner delta {deltas[-1]:.3e} loop delta {loop_deltas[-1]:.3e} "
              f"({time.time() - t0:.0f} s)", flush=True)
        if ck and len(deltas) % 2 == 0:
            os.makedirs(args.checkpoint, exist_ok=True)
            arrs = {f"{i}_{n}": envs[i][n] for i in range(4) for n in R.ENV_NAMES}
            np.savez(ck + ".tmp.npz", deltas=np.array(deltas), loop_deltas=np.array(loop_deltas), **arrs)
            os.replace(ck + ".tmp.npz", ck)
    rho1 = [R.rdm1(envs, As, i) for i in range(4)]
    rho2 = [R.rdm2(envs, As, i, dx, dy) for (i, dx, dy) in I.SQUARE_2X2_BONDS]
    obs1 = [R.expect(op1, r) for r in rho1]
    obs2 = [R.expect(op2, r) for r in rho2]
    lk, sign = R.log_kappa_per_site(envs, As)
    cuts = {}
    for x in range(2):
        for y in range(2):
            s = R.cut_singular_values(envs, As, x, y)
            cuts[f"x{x}y{y}"] = {"s_chi_minus_2..chi+1_over_s0": list(s[chi - 2:chi + 2] / s[0]),
                                 "rel_gap_at_chi": float((s[chi - 1] - s[chi]) / s[chi - 1])}
    out = {
        "case": args.case,
        "provenance": ("tests/golden/make_ctmrg_goldens.py: CPU oracle (oracle/ctmrg_ref.py, dense "
                       "half systems, full LAPACK SVD) on paper_2112_13184_gb300.inputs; numpy "
                       + np.__version__),
        "chi": chi, "sweeps": len(deltas), "corner_spectrum_deltas": deltas, "loop_spectrum_deltas": loop_deltas,
        "sites_then_bonds": {"one_site": [0, 1, 2, 3], "bonds": [list(b) for b in I.SQUARE_2X2_BONDS]},
        "observables": obs1 + obs2,
        "rdm1": [r.tolist() for r in rho1],
        "rdm2": [r.tolist() for r in rho2],
        "corner_spectra": R.corner_spectra(envs).tolist(),
        "loop_spectra": R.loop_spectra(envs).tolist(),
        "log_kappa_per_site": lk, "log_kappa_sign": sign,
        "cuts": cuts,
    }
    path = os.path.join(HERE, args.case + ".json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, flush=True)


if __name__ == "__main__":
    main()
