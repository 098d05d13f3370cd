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


def _oz(M, N, K, slices=5, tA=0):
    import torch
    from paper_2112_13184_gb300 import ctm
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((K, M) if tA else (M, K), dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(K, N, dtype=torch.float64, device="cuda", generator=g)
    C = torch.empty(M, N, dtype=torch.float64, device="cuda")
    ws = torch.empty(ctm.ctm_gemm_ozaki_workspace_bytes(M, N, K, slices), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ctm.ctm_gemm_ozaki(tA, 0, M, N, K, 1.0, A, A.shape[1], B, N, 0.0, C, N, slices, ws)
    torch.cuda.synchronize()
    print("done", float(C[0, 0]))


def apply_oz():
    """Corner apply of the D=8, chi=128 sweep on the tensor cores (5 slices)."""
    _oz(8192, 144, 8192)


def x2_oz():
    """First corner-formation product of the D=8, chi=128 sweep: 8192 x 8192 x 128."""
    _oz(8192, 8192, 128)


def x3_oz():
    """Second corner-formation product of the D=8, chi=128 sweep: 1048576 x 192 x 64."""
    _oz(1048576, 192, 64)


def x4t_oz():
    """Third product's shape with a transposed (column-layout) A: 1048576 x 64 x 192."""
    _oz(1048576, 64, 192, tA=1)


def split_e():
    """Slicing of an enlarged corner E (8192 x 8192) as a row-layout operand
    (E X) and as a column-layout one (E^T X), one emulated product each."""
    import torch
    from paper_2112_13184_gb300 import ctm
    N, k, slices = 8192, 144, 5
    g = torch.Generator(device="cuda").manual_seed(0)
    E = torch.randn(N, N, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn(N, k, dtype=torch.float64, device="cuda", generator=g)
    Y = torch.empty(N, k, dtype=torch.float64, device="cuda")
    ws = torch.empty(ctm.ctm_gemm_ozaki_workspace_bytes(N, k, N, slices), dtype=torch.uint8, device="cuda")
    for tA in (0, 1):
        ctm.ctm_gemm_ozaki(tA, 0, N, k, N, 1.0, E, N, X, k, 0.0, Y, k, slices, ws)
    torch.cuda.synchronize()
    print("split_e done", float(Y[0, 0]))


def sweep_mixed_chi64():
    """One emulated-FP64 sweep at d=3, D=8, chi=64 (N = 4096, corners 134 MB):
    every kernel of the sweep in its real operand layouts (strided corner
    views, slice caches), on a case small enough for full ncu captures."""
    import torch
    from paper_2112_13184_gb300 import ctm, inputs
    d, D, chi = 3, 8, 64
    c = ctm.CTMRG(d, D, chi, precision=ctm.CTM_OZAKI_BF16, ozaki_slices=5)
    c.set_tensors(inputs.x_polarised_tensors(d, D, 0.05, seed=3))
    c.set_envs(inputs.random_env(chi, [D] * 4, seed=4))
    c.sweep(1)
    torch.cuda.synchronize()
    print("sweep_mixed_chi64 done", c.measure1(0, inputs.spin_ops(d)["Sx"]))
    c.close()


CASES = {"split_e": split_e, "sweep_mixed_chi64": sweep_mixed_chi64, "apply_fp64": apply_fp64, "apply_oz": apply_oz, "x2_oz": x2_oz, "x3_oz": x3_oz, "x4t_oz": x4t_oz}

if __name__ == "__main__":
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        print("cases:", ", ".join(CASES))
        sys.exit(2)
    CASES[sys.argv[1]]()
