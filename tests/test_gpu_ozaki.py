"""Emulated-FP64 tensor-core GEMM (ctm_gemm_ozaki) against numpy FP64.

Exactness pins: when every operand entry is a whole number of the slice
unit (integers below 2^8 of the row/column maximum use only the leading
digit; below 2^16 only the two leading digits), every slice product the
kernel keeps is accumulated exactly (levels 0 and 1), nothing is dropped,
and the FP64 result must equal numpy's bit for bit (all partial sums stay
far below 2^53).  Shapes cross the 128-row and 16..144-column tiles with
ragged tails, several 256-wide K chunks, split-K and both transposes.
General data: error within (2^(2-8s) + 2^-36) max|row| max|col| K: the
slicing, plus the tensor cores' FP32 rounding of the levels >= 2, which are
summed in FP32 only within one 256-wide K chunk.
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


def run(ctm, A, B, tA, tB, slices, alpha=1.0, beta=0.0, C0=None):
    M = A.shape[1] if tA else A.shape[0]
    K = A.shape[0] if tA else A.shape[1]
    N = B.shape[0] if tB else B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(C0 if C0 is not None else np.zeros((M, N)))).cuda()
    ws = torch.zeros(ctm.ctm_gemm_ozaki_workspace_bytes(M, N, K, slices), dtype=torch.uint8, device="cuda")
    ctm.ctm_gemm_ozaki(tA, tB, M, N, K, alpha, dA, A.shape[1], dB, B.shape[1], beta, dC, N, slices, ws)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0, "a bounded device wait gave up"
    return dC.cpu().numpy()


def bound_of(A, B, slices):
    """Per-entry error bound of the emulated product of A (M x K) and B (K x N)."""
    K = A.shape[1]
    return (2.0 ** (2 - 8 * slices) + 2.0 ** -36) * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * K


SHAPES = [(128, 16, 32), (200, 144, 1000), (129, 33, 300), (64, 64, 64), (300, 200, 520), (1, 1, 1),
          (257, 100, 2048)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_exact_leading_digit(ctm, M, N, K, tA, tB):
    rng = np.random.default_rng(M + 3 * N + 7 * K + tA + 2 * tB)
    A = rng.integers(-255, 256, size=(K, M) if tA else (M, K)).astype(np.float64)
    B = rng.integers(-255, 256, size=(N, K) if tB else (K, N)).astype(np.float64)
    ref = (A.T if tA else A) @ (B.T if tB else B)
    got = run(ctm, A, B, tA, tB, slices=3)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("M,N,K", [(200, 144, 1000), (300, 200, 520), (257, 100, 2048)])
def test_exact_two_digits(ctm, M, N, K):
    """A uses one digit, B two (integers below 2^16 with a row maximum near
    2^16): the level-1 accumulator is exercised and stays exact."""
    rng = np.random.default_rng(K)
    A = rng.integers(-255, 256, size=(M, K)).astype(np.float64)
    B = rng.integers(-65535, 65536, size=(K, N)).astype(np.float64)
    B[0, :] = 65535.0  # pin every column maximum just below 2^16
    ref = A @ B
    got = run(ctm, A, B, 0, 0, slices=2)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("slices", [3, 4, 5])
@pytest.mark.parametrize("M,N,K", [(200, 144, 1000), (300, 200, 520)])
def test_random_within_slicing_bound(ctm, slices, M, N, K):
    rng = np.random.default_rng(slices * 100 + M)
    A = rng.standard_normal((M, K)) * np.logspace(0, -6, M)[:, None]
    B = rng.standard_normal((K, N)) * np.logspace(0, -6, N)[None, :]
    ref = A @ B
    got = run(ctm, A, B, 0, 0, slices)
    bound = bound_of(A, B, slices)
    assert np.all(np.abs(got - ref) <= bound)


def test_alpha_beta(ctm):
    rng = np.random.default_rng(5)
    A = rng.integers(-100, 100, size=(70, 90)).astype(np.float64)
    B = rng.integers(-100, 100, size=(90, 40)).astype(np.float64)
    C0 = rng.integers(-100, 100, size=(70, 40)).astype(np.float64)
    got = run(ctm, A, B, 0, 0, 3, alpha=2.0, beta=-0.5, C0=C0)
    np.testing.assert_array_equal(got, 2.0 * (A @ B) - 0.5 * C0)


def test_corner_apply_shape(ctm):
    """The projector's corner apply at D=8, chi=128: 8192 x 8192 times 8192 x 144."""
    N, k = 8192, 144
    g = torch.Generator(device="cuda").manual_seed(0)
    E = torch.randn(N, N, dtype=torch.float64, device="cuda", generator=g)
    X = torch.randn(N, k, dtype=torch.float64, device="cuda", generator=g)
    Y = torch.empty(N, k, dtype=torch.float64, device="cuda")
    ws = torch.zeros(ctm.ctm_gemm_ozaki_workspace_bytes(N, k, N, 4), dtype=torch.uint8, device="cuda")
    ctm.ctm_gemm_ozaki(0, 0, N, k, N, 1.0, E, N, X, k, 0.0, Y, k, 4, ws)
    ref = E @ X
    torch.cuda.synchronize()
    err = (Y - ref).abs().max().item()
    assert err < 2.0 ** -30 * E.abs().max().item() * X.abs().max().item() * N


# More tiles than the GB300's 152 SMs on the direct (non split-K) path: the
# persistent grid then walks several tiles per CTA, carrying the stage ring
# phases and the TMEM accumulator hand-off from one tile to the next.
MULTI_TILE = [(64000, 64, 64), (64000, 144, 256), (64000, 192, 256), (40000, 144, 600)]


def run_ld(ctm, A, B, tA, tB, slices, ldc, fill=7.0):
    """Like run(), with the output written at row stride ldc > N; the
    columns past N must keep their fill value."""
    M = A.shape[1] if tA else A.shape[0]
    K = A.shape[0] if tA else A.shape[1]
    N = B.shape[0] if tB else B.shape[1]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.full((M, ldc), fill, dtype=torch.float64, device="cuda")
    ws = torch.zeros(ctm.ctm_gemm_ozaki_workspace_bytes(M, N, K, slices), dtype=torch.uint8, device="cuda")
    ctm.ctm_gemm_ozaki(tA, tB, M, N, K, 1.0, dA, A.shape[1], dB, B.shape[1], 0.0, dC, ldc, slices, ws)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0, "a bounded device wait gave up"
    return dC.cpu().numpy()


@pytest.mark.parametrize("M,N,K", MULTI_TILE)
@pytest.mark.parametrize("tA", [0, 1])
def test_exact_multi_tile_persistent(ctm, M, N, K, tA):
    """Integer operands using the leading digit only: bit-exact over
    hundreds of tiles per launch (tiles = ceil(M/128) x N-tiles > 152)."""
    rng = np.random.default_rng(M + N + K + tA)
    A = rng.integers(-255, 256, size=(K, M) if tA else (M, K)).astype(np.float64)
    B = rng.integers(-255, 256, size=(K, N)).astype(np.float64)
    ref = (A.T if tA else A) @ B
    got = run(ctm, A, B, tA, 0, slices=3)
    np.testing.assert_array_equal(got, ref)


def test_exact_multi_tile_two_digits(ctm):
    """Two-digit B on the persistent multi-tile path: level-1 sums drained
    from TMEM every 256-wide chunk, across tiles."""
    M, N, K = 40000, 144, 600
    rng = np.random.default_rng(9)
    A = rng.integers(-255, 256, size=(M, K)).astype(np.float64)
    B = rng.integers(-65535, 65536, size=(K, N)).astype(np.float64)
    B[0, :] = 65535.0
    got = run(ctm, A, B, 0, 0, slices=2)
    np.testing.assert_array_equal(got, A @ B)


def test_exact_multi_tile_strided_output(ctm):
    """Output rows at stride ldc = N + 40: exact values in the first N
    columns, the rest untouched."""
    M, N, K, ldc = 64000, 144, 256, 184
    rng = np.random.default_rng(11)
    A = rng.integers(-255, 256, size=(M, K)).astype(np.float64)
    B = rng.integers(-255, 256, size=(N, K)).astype(np.float64)
    got = run_ld(ctm, A, B, 0, 1, 3, ldc)
    np.testing.assert_array_equal(got[:, :N], A @ B.T)
    assert np.all(got[:, N:] == 7.0)


@pytest.mark.parametrize("M,N,K", [(64000, 144, 256), (40000, 192, 600), (2048, 144, 8192), (256, 144, 256)])
def test_random_multi_tile_within_slicing_bound(ctm, M, N, K):
    """General FP64 data, 5 slices, multi-tile persistent path: every entry
    within 2^(2-8s) max|row| max|col| K of the FP64 product."""
    rng = np.random.default_rng(M + K)
    A = rng.standard_normal((M, K)) * np.logspace(0, -6, M)[:, None]
    B = rng.standard_normal((K, N)) * np.logspace(0, -6, N)[None, :]
    ref = A @ B
    got = run(ctm, A, B, 0, 0, 5)
    assert np.all(np.abs(got - ref) <= bound_of(A, B, 5))


@pytest.mark.parametrize("M,N,K", [(200, 144, 1000), (25600, 144, 64), (64000, 192, 256), (40000, 144, 600)])
def test_exact_three_levels(ctm, M, N, K):
    """Both operands two-digit integers (below 2^16, row/column maxima pinned
    at 65535) with 3 slices: the level-2 products a1 b1 2^-16 land in the
    FP32 accumulator, and for K <= 1000 their sums stay below 2^8 in 2^-16
    steps, so they are exact too and the whole product must equal numpy's
    bit for bit -- on the split-K path (first shape) and on the direct
    persistent path (the others, 200 to 1000 tiles)."""
    rng = np.random.default_rng(M + 7 * K)
    A = rng.integers(-65535, 65536, size=(M, K)).astype(np.float64)
    B = rng.integers(-65535, 65536, size=(K, N)).astype(np.float64)
    A[:, 0] = 65535.0
    B[0, :] = 65535.0
    got = run(ctm, A, B, 0, 0, slices=3)
    np.testing.assert_array_equal(got, A @ B)
