"""FP32-accumulated tensor-core GEMMs (ctm_gemm_split): split-BF16 (3 BF16
base-256 digit slices, every product of levels <= 2 kept) and 3xTF32 (2 TF32
base-2^11 digit slices, hi*hi + hi*lo + lo*hi kept), against numpy FP64.

Both schemes scale each row of op(A) and column of op(B) by 2^-e with
max|x| < 2^e and cut round(x 2^(Ls - e)) into digits (L = 8 or 11 bits, s
slices); the kept slice products are summed in FP32 on the tensor cores.

Exactness pins: integer operands whose digits the scheme keeps, arranged so
that every FP32 partial sum is a whole number of its unit below 2^24, give
numpy's result bit for bit.  The row and column maxima that fix the
exponents are planted at k = 0 (A) and k = 1 (B) with the other operand zero
there, so their large products never enter the sum.  One pin per kept level
path: leading digits only; one operand on two digits (level 1: d0*d1, and
for 3xTF32 hi*lo and lo*hi); one operand on three digits (level 2: d0*d2);
both operands on two digits (level 2: d1*d1).

Random data: per entry, |error| <= T + 2^-22 (p sum_g |P_g| + 2 sum_k |a_k b_k|)
with the slicing term T = 2^-22 sum_k (|a_k| max|b| + max|a| |b_k| + max|a| max|b|)
(the representation error of each operand is below 2^-22 of its row or
column maximum; the dropped products below 2^-22 max|a| max|b|), the FP32
accumulation bounded by one rounding of 2^-22 (either rounding mode) of each
partial sum P_g after every group of 8 k, for each of the p kept slice-product
pairs, plus the in-group sums.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_13184_gb300 import ctm as m
    return m


def prec_of(ctm, name):
    return ctm.CTM_SPLIT_BF16 if name == "bf16x3" else ctm.CTM_3XTF32


def run(ctm, name, A, B, tA, tB, alpha=1.0, beta=0.0, C0=None):
    M = A.shape[1] if tA else A.shape[0]
    K = A.shape[0] if tA else A.shape[1]
    N = B.shape[0] if tB else B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(C0 if C0 is not None else np.zeros((M, N)))).cuda()
    p = prec_of(ctm, name)
    ws = torch.zeros(ctm.ctm_gemm_split_workspace_bytes(p, M, N, K), dtype=torch.uint8, device="cuda")
    ctm.ctm_gemm_split(p, tA, tB, M, N, K, alpha, dA, A.shape[1], dB, B.shape[1], beta, dC, N, ws)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0, "a bounded device wait gave up"
    return dC.cpu().numpy()


def planted(rng, M, N, K, a_lim, b_lim, a_max, b_max):
    """A (M x K), B (K x N): integers |a| <= a_lim, |b| <= b_lim; A's row
    maxima a_max at k = 0 (B zero there), B's column maxima b_max at k = 1
    (A zero there)."""
    A = rng.integers(-a_lim, a_lim + 1, size=(M, K)).astype(np.float64)
    B = rng.integers(-b_lim, b_lim + 1, size=(K, N)).astype(np.float64)
    A[:, 0] = a_max
    B[0, :] = 0.0
    if K > 1:
        A[:, 1] = 0.0
        B[1, :] = b_max
    return A, B


def check_exact(ctm, name, A, B, tA, tB):
    ref = A @ B
    assert np.abs(ref).max() < 2 ** 53
    a_in = np.ascontiguousarray(A.T) if tA else A
    b_in = np.ascontiguousarray(B.T) if tB else B
    got = run(ctm, name, a_in, b_in, tA, tB)
    np.testing.assert_array_equal(got, ref)


SHAPES = [(128, 16, 32), (200, 144, 160), (129, 33, 250), (64, 64, 64), (300, 200, 256), (1, 1, 1), (257, 100, 96)]
TRANS = [(0, 0), (1, 0), (0, 1), (1, 1)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("tA,tB", TRANS)
def test_bf16x3_leading_digit(ctm, M, N, K, tA, tB):
    """|a|, |b| <= 255 with maxima 255 (e = 8): one digit each; level 0 only,
    partial sums <= 256 * 255^2 < 2^24."""
    rng = np.random.default_rng(M + 3 * N + 7 * K + tA + 2 * tB)
    A, B = planted(rng, M, N, K, 255, 255, 255.0, 255.0)
    check_exact(ctm, "bf16x3", A, B, tA, tB)


@pytest.mark.parametrize("swap", [False, True])
@pytest.mark.parametrize("tA,tB", TRANS)
def test_bf16x3_level1(ctm, swap, tA, tB):
    """One operand on two base-256 digits (max 65535, e = 16; |x| <= 2047):
    sum a b / 2^8 in FP32, exact while sum |a b| < 2^24 (|a| <= 31, K = 256)."""
    rng = np.random.default_rng(11 + tA + 2 * tB + 4 * swap)
    M, N, K = 200, 144, 256
    if not swap:
        A, B = planted(rng, M, N, K, 31, 2047, 255.0, 65535.0)
    else:
        A, B = planted(rng, M, N, K, 2047, 31, 65535.0, 255.0)
    check_exact(ctm, "bf16x3", A, B, tA, tB)


@pytest.mark.parametrize("tA,tB", TRANS)
def test_bf16x3_level2_d0_d2(ctm, tA, tB):
    """B on three digits (max 2^24 - 1, e = 24; |b| <= 2^15): the d0*d2
    products; sum a b / 2^16 exact while sum |a b| < 2^24 (|a| <= 3, K = 160)."""
    rng = np.random.default_rng(21 + tA + 2 * tB)
    A, B = planted(rng, 130, 40, 160, 3, 2 ** 15, 255.0, 2.0 ** 24 - 1)
    check_exact(ctm, "bf16x3", A, B, tA, tB)


@pytest.mark.parametrize("tA,tB", TRANS)
def test_bf16x3_level2_d1_d1(ctm, tA, tB):
    """Both operands on two digits (maxima 65535, |x| <= 300): the d1*d1
    products; sum a b / 2^16 exact while sum |a b| < 2^24 (K = 160)."""
    rng = np.random.default_rng(31 + tA + 2 * tB)
    A, B = planted(rng, 150, 70, 160, 300, 300, 65535.0, 65535.0)
    check_exact(ctm, "bf16x3", A, B, tA, tB)


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("tA,tB", TRANS)
def test_tf32x3_leading_digit(ctm, M, N, K, tA, tB):
    """Maxima 2047 (e = 11, hi = x, lo = 0), other entries |x| <= 15: hi*hi
    only, partial sums <= 2 * 2047 * 15 + K * 225 < 2^24."""
    rng = np.random.default_rng(5 + M + 3 * N + 7 * K + tA + 2 * tB)
    A, B = planted(rng, M, N, K, 15, 15, 2047.0, 2047.0)
    check_exact(ctm, "tf32x3", A, B, tA, tB)


@pytest.mark.parametrize("swap", [False, True])
@pytest.mark.parametrize("tA,tB", TRANS)
def test_tf32x3_hi_lo(ctm, swap, tA, tB):
    """One operand on both TF32 slices (max 2^22 - 1, e = 22: hi =
    round(x / 2^11), lo = x - 2^11 hi; |x| <= 4095), the other on hi only
    (|x| <= 7): hi*hi + hi*lo (lo*hi with swap), sum a b / 2^11 exact while
    sum |a b| < 2^24 (K = 520)."""
    rng = np.random.default_rng(41 + tA + 2 * tB + 4 * swap)
    M, N, K = 200, 144, 520
    if not swap:
        A, B = planted(rng, M, N, K, 7, 4095, 2047.0, 2.0 ** 22 - 1)
    else:
        A, B = planted(rng, M, N, K, 4095, 7, 2.0 ** 22 - 1, 2047.0)
    check_exact(ctm, "tf32x3", A, B, tA, tB)


def rigorous_bound(A, B, pairs):
    """Per-entry bound of the module docstring, A (M x K), B (K x N)."""
    K = A.shape[1]
    ma = np.abs(A).max(axis=1)[:, None]
    mb = np.abs(B).max(axis=0)[None, :]
    aa, ab = np.abs(A), np.abs(B)
    T = 2.0 ** -22 * (aa.sum(1)[:, None] * mb + ma * ab.sum(0)[None, :] + K * ma * mb)
    absum = aa @ ab
    g = 8
    ng = (K + g - 1) // g
    Kp = ng * g
    Ap = np.zeros((A.shape[0], Kp)); Ap[:, :K] = A
    Bp = np.zeros((Kp, B.shape[1])); Bp[:K] = B
    P = np.zeros(absum.shape)
    acc = np.zeros(absum.shape)
    for i in range(ng):
        P += Ap[:, i * g:(i + 1) * g] @ Bp[i * g:(i + 1) * g]
        acc += np.abs(P)
    return T + 2.0 ** -22 * (pairs * acc + 2.0 * absum)


@pytest.mark.parametrize("name,pairs", [("bf16x3", 6), ("tf32x3", 3)])
@pytest.mark.parametrize("M,N,K", [(200, 144, 1000), (300, 200, 520), (2048, 144, 4096), (129, 33, 7)])
def test_random_within_bound(ctm, name, pairs, M, N, K):
    rng = np.random.default_rng(M + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-3, 3, size=(1, N)))
    ref = A @ B
    got = run(ctm, name, A, B, 0, 0)
    err = np.abs(got - ref)
    bound = rigorous_bound(A, B, pairs)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"{name} {M}x{N}x{K}: Frobenius-relative error {rel:.2e}, max error / bound {np.max(err / bound):.2e}")
    assert np.all(err <= bound)
    assert rel < 2.0 ** -14  # a dropped hi*lo (3xTF32) or level-1 product (BF16) sits near 2^-11 .. 2^-8


@pytest.mark.parametrize("name", ["bf16x3", "tf32x3"])
def test_alpha_beta(ctm, name):
    rng = np.random.default_rng(7)
    A, B = planted(rng, 150, 60, 200, 15, 15, 255.0 if name == "bf16x3" else 2047.0,
                   255.0 if name == "bf16x3" else 2047.0)
    C0 = rng.integers(-100, 101, size=(150, 60)).astype(np.float64)
    got = run(ctm, name, A, B, 0, 0, alpha=2.0, beta=-0.5, C0=C0)
    np.testing.assert_array_equal(got, 2.0 * (A @ B) - 0.5 * C0)


def test_rejects_other_precisions(ctm):
    assert ctm.ctm_gemm_split_workspace_bytes(ctm.CTM_OZAKI_BF16, 8, 8, 8) == 0
    assert ctm.ctm_gemm_split_workspace_bytes(ctm.CTM_FP64, 8, 8, 8) == 0
