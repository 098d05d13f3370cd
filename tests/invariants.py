"""Gauge-invariant quantities computed in the tests from any environment
(the library's or the oracle's), so that both sides go through the same
post-processing and no oracle function ever takes the library's output.

loop_spectra(envs): for the 2x2 block with bottom-left site i = (x, y), the
four corners joined directly around it, L = C1(x,y+1) C2(x+1,y+1) C3(x+1,y)
C4(x,y), are the network Z_00; a change of basis on any chi bond turns L into
a similar matrix, so the moduli of its eigenvalues (sorted, normalised to sum
1) are invariant, while the singular values of a single corner are not.
"""
import numpy as np


def _site(x, y):
    return (x % 2) + 2 * (y % 2)


def loop_spectra(envs):
    out = []
    for i in range(4):
        x, y = i % 2, i // 2
        L = (envs[_site(x, y + 1)]["C1"] @ envs[_site(x + 1, y + 1)]["C2"]
             @ envs[_site(x + 1, y)]["C3"] @ envs[_site(x, y)]["C4"])
        m = np.sort(np.abs(np.linalg.eigvals(L)))[::-1]
        out.append(m / m.sum())
    return np.array(out)
