"""Small, self-contained launches of single libctm kernels for profiling.

    python -m paper_2112_13184_gb300.profile_cases <case>

Each case allocates its inputs on cuda:0 (seeded), launches the kernel a
few times through the C ABI and exits; sized so that an ncu capture of one
launch ends in seconds while the operands still exceed the 129 MB L2.
"""
from __future__ import annotations

import sys

import numpy as np


def apply_fp64():
    """One corner apply of the D=8, chi=128 sweep: Y = E X, E 8192 x 8192
    (537 MB), X 8192 x 144, FP64."""
    import torch
    from paper_2112_13184_gb300 import ctm
    N, k = 8192, 144
    g = torch.Generator(device="cuda").manual_seed(0)
    E = torch.randn(N, N, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn(N, k, dtype=torch.float64, device="cuda", generator=g)
    Y = torch.empty(N, k, dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctm.ctm_dgemm(0, 0, N, k, N, 1.0, E, N, X, k, 0.0, Y, k)
    torch.cuda.synchronize()
    print("apply_fp64 done", float(Y[0, 0]))


CASES = {"apply_fp64": apply_fp64}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        print("cases:", ", ".join(CASES))
        sys.exit(2)
    CASES[sys.argv[1]]()
