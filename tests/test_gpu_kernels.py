"""Per-kernel parity of libctm's FP64 building blocks against numpy (FP64).

Sizes span several 64-wide tiles with ragged tails.  Tolerances follow
the FP64 arithmetic: GEMM to 1e-13 relative of |A||B| scale; permute bit-exact;
QR to 1e-13 (orthogonality, reconstruction, unique R with diag >= 0);
Jacobi SVD to 1e-13 relative on graded singular values."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("tA,tB", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (67, 130, 45), (200, 33, 257), (129, 129, 16)])
def test_dgemm(ctm, tA, tB, M, N, K):
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((K, M) if tA else (M, K))
    B = rng.standard_normal((N, K) if tB else (K, N))
    C0 = rng.standard_normal((M, N))
    ref = 1.5 * (A.T if tA else A) @ (B.T if tB else B) - 0.5 * C0
    dA, dB, dC = dev(A), dev(B), dev(C0)
    ctm.ctm_dgemm(tA, tB, M, N, K, 1.5, dA, A.shape[1], dB, B.shape[1], -0.5, dC, N)
    torch.cuda.synchronize()
    scale = np.abs(A).max() * np.abs(B).max() * K
    assert np.max(np.abs(dC.cpu().numpy() - ref)) < 1e-14 * scale + 1e-15


@pytest.mark.parametrize("dims,perm", [((3, 4, 5), (2, 0, 1)), ((5, 2, 2, 3, 7, 2), (0, 3, 5, 1, 2, 4)),
                                       ((2, 3, 2, 5, 4, 2, 2, 3), (4, 5, 0, 1, 2, 3, 6, 7)),
                                       ((1000, 37), (1, 0))])
def test_permute_exact(ctm, dims, perm):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(dims)
    out = torch.empty(int(np.prod(dims)), dtype=torch.float64, device="cuda")
    ctm.ctm_permute(dev(x), out, dims, perm)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().reshape([dims[p] for p in perm]), x.transpose(perm))


@pytest.mark.parametrize("N,k", [(300, 24), (1000, 144), (144, 144), (77, 5)])
def test_qr(ctm, N, k):
    rng = np.random.default_rng(N + k)
    # graded columns: condition ~1e12, as the range finder produces
    Y = rng.standard_normal((N, k)) * np.logspace(0, -12, k)[None, :]
    dY = dev(Y)
    Q = torch.empty((N, k), dtype=torch.float64, device="cuda")
    R = torch.empty((k, k), dtype=torch.float64, device="cuda")
    ws = torch.empty(ctm.ctm_qr_workspace_bytes(N, k), dtype=torch.uint8, device="cuda")
    ctm.ctm_qr(dY, N, k, Q, R, ws)
    torch.cuda.synchronize()
    Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
    assert np.max(np.abs(Qh.T @ Qh - np.eye(k))) < 1e-13 * N
    assert np.max(np.abs(np.tril(Rh, -1))) == 0.0
    assert np.all(np.diag(Rh) >= 0)
    assert np.max(np.abs(Qh @ Rh - Y)) < 1e-14 * np.abs(Y).max() * N
    np.testing.assert_array_equal(dY.cpu().numpy(), Y)  # input untouched
    # uniqueness (full rank, diag > 0): compare with numpy's QR after sign fix
    Qn, Rn = np.linalg.qr(Y)
    s = np.sign(np.diag(Rn))
    Rn = Rn * s[:, None]
    assert np.max(np.abs(Rh - Rn) / (np.abs(Rn).max(axis=1, keepdims=True))) < 1e-9


@pytest.mark.parametrize("k", [1, 5, 24, 33, 144])
def test_svd(ctm, k):
    rng = np.random.default_rng(k)
    G = rng.standard_normal((k, k)) * np.logspace(0, -13, k)[None, :]
    U = torch.empty((k, k), dtype=torch.float64, device="cuda")
    V = torch.empty((k, k), dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    ws = torch.empty(ctm.ctm_svd_workspace_bytes(k), dtype=torch.uint8, device="cuda")
    ctm.ctm_svd(dev(G), k, U, S, V, ws)
    torch.cuda.synchronize()
    Uh, Sh, Vh = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    sref = np.linalg.svd(G, compute_uv=False)
    assert np.all(np.diff(Sh) <= 0)
    # LAPACK's small singular values are accurate to ~eps * s_max only
    assert np.all(np.abs(Sh - sref) < 1e-12 * sref + 1e-14 * k * sref[0])
    assert np.max(np.abs((Uh * Sh) @ Vh.T - G)) < 1e-14 * k
    assert np.max(np.abs(Vh.T @ Vh - np.eye(k))) < 1e-13 * k
    assert np.max(np.abs(Uh.T @ Uh - np.eye(k))) < 1e-12 * k


def test_svd_rank_deficient(ctm):
    k = 12
    rng = np.random.default_rng(3)
    G = rng.standard_normal((k, 5)) @ rng.standard_normal((5, k))
    U = torch.empty((k, k), dtype=torch.float64, device="cuda")
    V = torch.empty((k, k), dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    ws = torch.empty(ctm.ctm_svd_workspace_bytes(k), dtype=torch.uint8, device="cuda")
    ctm.ctm_svd(dev(G), k, U, S, V, ws)
    torch.cuda.synchronize()
    Sh = S.cpu().numpy()
    sref = np.linalg.svd(G, compute_uv=False)
    assert np.max(np.abs(Sh[:5] - sref[:5]) / sref[:5]) < 1e-12
    assert np.max(Sh[5:]) < 1e-13 * Sh[0]
    assert np.max(np.abs((U.cpu().numpy() * Sh) @ V.cpu().numpy().T - G)) < 1e-13


def test_svd_reports_converged(ctm):
    """The first int of the SVD workspace is the Jacobi status: 0 when the
    rotations settled within the sweep cap."""
    k = 144
    rng = np.random.default_rng(5)
    G = rng.standard_normal((k, k)) * np.logspace(0, -12, k)[None, :]
    U = torch.empty((k, k), dtype=torch.float64, device="cuda")
    V = torch.empty((k, k), dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    ws = torch.full((ctm.ctm_svd_workspace_bytes(k),), 0xFF, dtype=torch.uint8, device="cuda")
    ctm.ctm_svd(dev(G), k, U, S, V, ws)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0


def test_bounded_wait_gives_up_and_context_survives(ctm):
    """Failure detection without a fault: a thread waits on an mbarrier that
    nothing arrives on, with a short limit (1e6 cycles, ~0.5 ms).  The wait
    must give up, the call report CTM_ERR_TIMEOUT, and the device keep
    working: the same probe with an arrival succeeds and a GEMM runs."""
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert ctm.ctm_wait_probe(1_000_000, 0, flag) == ctm.CTM_ERR_TIMEOUT
    assert int(flag.item()) == 1
    assert ctm.ctm_wait_probe(1_000_000, 1, flag) == ctm.CTM_OK
    assert int(flag.item()) == 0
    rng = np.random.default_rng(2)
    A = rng.integers(-100, 100, size=(130, 70)).astype(np.float64)
    B = rng.integers(-100, 100, size=(70, 50)).astype(np.float64)
    C = torch.zeros((130, 50), dtype=torch.float64, device="cuda")
    ws = torch.zeros(ctm.ctm_gemm_ozaki_workspace_bytes(130, 50, 70, 3), dtype=torch.uint8, device="cuda")
    ctm.ctm_gemm_ozaki(0, 0, 130, 50, 70, 1.0, dev(A), 70, dev(B), 50, 0.0, C, 50, 3, ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.cpu().numpy(), A @ B)
    with pytest.raises(ctm.CtmError):
        ctm.ctm_wait_probe(0, 0, flag)
