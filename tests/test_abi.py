"""C ABI checks that need no GPU: the library loads, exports every function
include/ctm.h declares, and its host-only logic behaves."""
import os
import re

import numpy as np
import pytest

from oracle import elements as EL
from paper_2112_13184_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ctm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2112_13184_gb300 import ctm
    lib = ctypes.CDLL(ctm.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi():
    from paper_2112_13184_gb300 import ctm
    for n in _declared():
        if n in ("ctm_last_error", "ctm_status_string"):
            continue
        assert hasattr(ctm, n), n


def test_default_options_and_footprint():
    from paper_2112_13184_gb300 import ctm
    o = ctm.ctm_default_options()
    assert o.chi == 16 and o.rsvd_power_iters == 2 and o.sv_cutoff_rel == 1e-12
    assert o.exact_svd_max_n == 256
    o = ctm.ctm_default_options(chi=128)
    b = ctm.ctm_footprint_bytes(3, 8, o)
    N = 128 * 64
    # dominated by the four N x N corners and the open-index RDM scratch
    assert 4 * N * N * 8 < b < 40 * N * N * 8


def test_invalid_create_is_rejected_without_gpu():
    from paper_2112_13184_gb300 import ctm
    o = ctm.ctm_default_options(chi=0)
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_create(2, 2, o)
    assert e.value.status == ctm.CTM_ERR_ARG


def test_op_from_elements_matches_oracle_and_golden():
    from paper_2112_13184_gb300 import ctm
    lines = EL.parse_elements("\n".join(l for l in open(os.path.join(ROOT, "tests", "golden",
                                                                      "heisenberg_elements.txt"))
                                        if not l.startswith("#")))
    op = ctm.ctm_op_from_elements(2, 2, lines)
    np.testing.assert_array_equal(op, EL.op_from_elements(2, 2, lines))
    np.testing.assert_allclose(op, I.heisenberg_bond(2), atol=0)
    # orientation: before (1,0) -> after (0,1) is <up down| S+ S- |down up>
    op = ctm.ctm_op_from_elements(2, 2, [(1, 0, 0, 1, 1.0, 0.0)])
    o = I.spin_ops(2)
    np.testing.assert_array_equal(op, np.kron(o["Sp"], o["Sm"]))
    with pytest.raises(ctm.CtmError):
        ctm.ctm_op_from_elements(2, 2, [(2, 0, 0, 0, 1.0, 0.0)])


def test_footprint_follows_batched_cuts_and_scheme():
    """Host arithmetic of ctm_footprint_bytes: batch_cuts keeps a second
    cut's four N x N corners (and, in a tensor-core mode, their eight slice
    caches) resident; the schemes' slice caches order FP64 < 3xTF32 (2 FP32
    slices) ~ split-BF16 (3 BF16 slices) < emulated FP64 with 5 BF16 slices."""
    from paper_2112_13184_gb300 import ctm
    d, D, chi = 3, 8, 64
    N = chi * D * D

    def fp(prec, batch):
        return ctm.ctm_footprint_bytes(d, D, ctm.ctm_default_options(chi=chi, precision=prec, batch_cuts=batch))

    assert fp(ctm.CTM_FP64, 1) - fp(ctm.CTM_FP64, 0) >= 4 * N * N * 8
    # eight more slice caches of 5 BF16 slices of an N x N corner
    assert fp(ctm.CTM_OZAKI_BF16, 1) - fp(ctm.CTM_OZAKI_BF16, 0) >= 4 * N * N * 8 + 8 * 5 * N * N * 2
    f64, tf32, bf3, oz5 = (fp(p, 1) for p in (ctm.CTM_FP64, ctm.CTM_3XTF32, ctm.CTM_SPLIT_BF16, ctm.CTM_OZAKI_BF16))
    assert f64 < bf3 < oz5 and f64 < tf32 < oz5


def test_unbuilt_scheme_and_bad_arena_are_rejected_without_gpu():
    from paper_2112_13184_gb300 import ctm
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_create(2, 2, ctm.ctm_default_options(chi=8, precision=ctm.CTM_OZAKI_INT8))
    assert e.value.status == ctm.CTM_ERR_ARG
    o = ctm.ctm_default_options(chi=8)
    need = ctm.ctm_footprint_bytes(2, 2, o)
    with pytest.raises(ctm.CtmError) as e:  # not 256-byte aligned
        ctm.ctm_create_in(2, 2, o, 1, need)
    assert e.value.status == ctm.CTM_ERR_ARG
    with pytest.raises(ctm.CtmError) as e:  # smaller than the footprint
        ctm.ctm_create_in(2, 2, o, 256, need - 1)
    assert e.value.status == ctm.CTM_ERR_ARG


def test_split_gemm_workspace_sizes():
    from paper_2112_13184_gb300 import ctm
    assert ctm.ctm_gemm_split_workspace_bytes(ctm.CTM_OZAKI_BF16, 64, 64, 64) == 0
    assert ctm.ctm_gemm_split_workspace_bytes(ctm.CTM_SPLIT_BF16, 0, 64, 64) == 0
    small = ctm.ctm_gemm_split_workspace_bytes(ctm.CTM_SPLIT_BF16, 200, 144, 1000)
    big = ctm.ctm_gemm_split_workspace_bytes(ctm.CTM_SPLIT_BF16, 400, 144, 1000)
    # three BF16 slices of both operands, padded rows: at least 2 s (M + N) K bytes
    assert small >= 2 * 3 * (200 + 144) * 1000 and big > small
    tf = ctm.ctm_gemm_split_workspace_bytes(ctm.CTM_3XTF32, 200, 144, 1000)
    assert tf >= 4 * 2 * (200 + 144) * 1000  # two FP32-held TF32 slices
