"""Host-side pieces of bench.py and the seeded input families (no GPU)."""
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gemm_roofline_arithmetic():
    if not os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        pytest.skip("no measured peaks on this machine")
    import bench
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    tc, bw = peaks["bf16_tflops_sustained"] * 1e12, peaks["hbm_gbs"] * 1e9
    # one tensor-bound and one HBM-bound operation, each taking 10x its roofline time
    f1, b1 = 1e12, 1e6
    f2, b2 = 1e6, 1e10
    t1, t2 = 10 * f1 / tc, 10 * b2 / bw
    by_op = {"a/gemm": {"ms": t1 * 1e3, "flops": f1, "bytes": b1},
             "b/gemm": {"ms": t2 * 1e3, "flops": f2, "bytes": b2},
             "c/split": {"ms": 5.0, "flops": 0.0, "bytes": 1e9}}
    r = bench.oz_gemm_roofline(by_op)
    assert r["ops"]["a/gemm"]["bound"] == "tensor" and r["ops"]["b/gemm"]["bound"] == "hbm"
    assert r["ops"]["a/gemm"]["roofline_frac"] == pytest.approx(0.1, rel=1e-3)
    assert r["roofline_time_frac"] == pytest.approx(0.1, rel=1e-6)
    tensor = f1 / tc + f2 / tc >= b1 / bw + b2 / bw
    assert r["bound"] == ("tensor" if tensor else "hbm")
    total_t = t1 + t2
    expect = (f1 + f2) / total_t / 1e12 if tensor else (b1 + b2) / total_t / 1e9
    assert r["achieved"] == pytest.approx(expect) and r["frac"] == pytest.approx(expect / r["peak"])
    assert r["class_ms"] == pytest.approx(total_t * 1e3)


def test_input_families_are_seeded():
    from paper_2112_13184_gb300 import inputs as I
    for j in (0, 7):
        a, b = I.serving_request(j), I.serving_request(j)
        assert (a["d"], a["D"], a["chi"]) == (b["d"], b["D"], b["chi"])
        assert a["d"] in (2, 3) and a["D"] in (4, 6, 8) and a["chi"] in (32, 64, 128)
        np.testing.assert_array_equal(a["As"][0], b["As"][0])
        assert a["As"][0].shape == (a["d"],) + (a["D"],) * 4
        assert a["op2"].shape == (a["d"] ** 2, a["d"] ** 2)
    seen = set()
    for i in range(64):
        q = I.batch_instance(i)
        assert q["D"] in (3, 4, 5, 6) and q["chi"] in (24, 32, 48, 64)
        seen.add((q["D"], q["chi"]))
    assert len(seen) > 4  # uneven sizes
