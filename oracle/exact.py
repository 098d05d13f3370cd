"""Closed forms the CTMRG oracle is pinned to.

TEST INFRASTRUCTURE ONLY -- see ``oracle/__init__.py``.

The Ising PEPS (inputs.ising_peps_tensor) has <psi|psi> = Z_Ising(K = beta)
on the square lattice with J = 1, so the CTMRG environment of that network
must reproduce Onsager's exact solution:
  * free energy per site  -beta f = ln 2 + (1/8 pi^2) int int
        ln[cosh^2 2K - sinh 2K (cos t1 + cos t2)] dt1 dt2     (Onsager 1944)
  * internal energy per site u = -coth 2K [1 + (2/pi)(2 tanh^2 2K - 1) K(k)],
        k = 2 sinh 2K / cosh^2 2K,  K(k) the complete elliptic integral
  * spontaneous magnetisation M = (1 - sinh^-4 2K)^(1/8) for K > K_c
        = ln(1 + sqrt 2)/2                                      (Yang 1952)
All are written here from these formulas with our own quadrature and AGM.
"""
from __future__ import annotations

import math

import numpy as np

K_CRITICAL = 0.5 * math.log(1.0 + math.sqrt(2.0))


def agm(a: float, b: float) -> float:
    for _ in range(100):
        a2, b2 = 0.5 * (a + b), math.sqrt(a * b)
        if abs(a2 - b2) <= 1e-17 * abs(a2):
            return a2
        a, b = a2, b2
    return 0.5 * (a + b)


def elliptic_k(k: float) -> float:
    """Complete elliptic integral of the first kind, modulus k: pi / (2 AGM(1, k'))."""
    return math.pi / (2.0 * agm(1.0, math.sqrt(1.0 - k * k)))


def onsager_log_z_per_site(K: float, n: int = 512) -> float:
    """-beta f per site by the periodic trapezoid rule on [0, 2pi)^2.

    The integrand is smooth and periodic away from K_c, so the rule
    converges exponentially in n."""
    t = 2.0 * np.pi * np.arange(n) / n
    c = np.cos(t)
    ch, sh = math.cosh(2 * K), math.sinh(2 * K)
    integrand = np.log(ch * ch - sh * (c[:, None] + c[None, :]))
    integral = integrand.mean() * (2 * np.pi) ** 2
    return math.log(2.0) + integral / (8 * np.pi ** 2)


def onsager_energy_per_site(K: float) -> float:
    """u = <-sum_bonds s_i s_j> per site (J = 1)."""
    k = 2.0 * math.sinh(2 * K) / math.cosh(2 * K) ** 2
    t = math.tanh(2 * K)
    return -(1.0 / math.tanh(2 * K)) * (1.0 + (2.0 / math.pi) * (2 * t * t - 1.0) * elliptic_k(k))


def onsager_nn_correlation(K: float) -> float:
    """<s_i s_j> for nearest neighbours: two bonds per site, so -u/2."""
    return -0.5 * onsager_energy_per_site(K)


def yang_magnetisation(K: float) -> float:
    if K <= K_CRITICAL:
        return 0.0
    return (1.0 - math.sinh(2 * K) ** -4) ** 0.125


def product_expectation(phi, op) -> float:
    """<phi|O|phi>/<phi|phi> for a real product state."""
    phi = np.asarray(phi, dtype=np.float64)
    return float(phi @ op @ phi / (phi @ phi))
