"""ctm_svd_noalloc: the Jacobi SVD with the library's static scratch array.

It exists for callers that cannot call cudaMalloc where they need the SVD
(graph capture in global mode, latency-bound serving loops, fixed memory
budgets).  This file is collected last so that a failure here cannot stop
the rest of a run that stops at the first failure; it must also pass alone
in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctm():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2112_13184_gb300 import ctm as m
    return m


def _run(ctm, fn, G, k, ws=None):
    U = torch.empty((k, k), dtype=torch.float64, device="cuda")
    V = torch.empty((k, k), dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    if ws is None:
        fn(G, k, U, S, V)
    else:
        fn(G, k, U, S, V, ws)
    torch.cuda.synchronize()
    return U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()


@pytest.mark.gpu
def test_svd_noalloc_matches_workspace_svd_twice(ctm):
    for call, k in enumerate((144, 37)):   # two calls in a row, the second smaller
        rng = np.random.default_rng(100 + call)
        Gh = rng.standard_normal((k, k)) * np.logspace(0, -13, k)[None, :]
        G = torch.from_numpy(Gh).cuda()
        ws = torch.empty(ctm.ctm_svd_workspace_bytes(k), dtype=torch.uint8, device="cuda")
        U0, S0, V0 = _run(ctm, ctm.ctm_svd, G, k, ws)
        U1, S1, V1 = _run(ctm, ctm.ctm_svd_noalloc, G, k)
        # same tolerance as the workspace SVD's own test
        assert np.all(np.abs(S1 - S0) < 1e-12 * S0 + 1e-14 * k * S0[0])
        assert np.max(np.abs((U1 * S1) @ V1.T - Gh)) < 1e-14 * k
        assert np.max(np.abs((U1 * S1) @ V1.T - (U0 * S0) @ V0.T)) < 1e-14 * k
        assert np.max(np.abs(V1.T @ V1 - np.eye(k))) < 1e-13 * k


@pytest.mark.gpu
def test_svd_noalloc_rejects_k_above_its_scratch(ctm):
    k = 257
    G = torch.zeros((k, k), dtype=torch.float64, device="cuda")
    U = torch.empty((k, k), dtype=torch.float64, device="cuda")
    V = torch.empty((k, k), dtype=torch.float64, device="cuda")
    S = torch.empty(k, dtype=torch.float64, device="cuda")
    with pytest.raises(ctm.CtmError) as e:
        ctm.ctm_svd_noalloc(G, k, U, S, V)
    assert e.value.status == ctm.CTM_ERR_ARG
