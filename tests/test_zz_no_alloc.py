"""The allocation-free Gram entry point (ekcg_gram_noalloc) against the context-based one
(ekcg_gram), two calls in a row through the C ABI.  Kept in a file that pytest collects
last; it also passes on its own in a fresh process."""
import os

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_10629_gb300 import ekcg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()


def test_noalloc_gram_matches_context_gram_on_two_calls_in_a_row():
    A = wl.stencil_matrix((45, 37))                     # n = 1665 rows, ragged
    S = ekcg.Solver(A, 16, wl.partition_boxes((45, 37), 16), max_s=4)
    rng = np.random.default_rng(7)
    for (p, q) in [(64, 32), (32, 16)]:                 # two calls in a row, other shapes
        X = rng.standard_normal((A.n, p))
        Y = rng.standard_normal((A.n, q))
        Xd = torch.as_tensor(X, device="cuda")
        Yd = torch.as_tensor(Y, device="cuda")
        C_ref = torch.empty(p * q, dtype=torch.float64, device="cuda")
        C_na = torch.full((p * q,), np.nan, dtype=torch.float64, device="cuda")
        ekcg.ekcg_gram(S.ctx, Xd, p, Yd, q, C_ref)
        ekcg.ekcg_gram_noalloc(A.n, Xd, p, Yd, q, C_na)
        torch.cuda.synchronize()
        # tolerance of the Gram tests: the float64 dot-product bound n eps |X|^T |Y|
        bound = A.n * 2.2e-16 * (np.abs(X).T @ np.abs(Y))
        ref = C_ref.cpu().numpy().reshape(p, q)
        got = C_na.cpu().numpy().reshape(p, q)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= 2 * bound)
        assert np.all(np.abs(got - X.T @ Y) <= bound)
    S.close()


def test_noalloc_gram_rejects_sizes_beyond_its_scratch():
    X = torch.zeros(10 * 65, dtype=torch.float64, device="cuda")
    C = torch.zeros(65 * 65, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="64"):
        ekcg.ekcg_gram_noalloc(10, X, 65, X, 1, C)
    # the C entry point itself refuses too (binding checks bypassed)
    st = ekcg.lib().ekcg_gram_noalloc(10, X.data_ptr(), 65, X.data_ptr(), 1, C.data_ptr(),
                                      None)
    assert st == ekcg.EKCG_EINVAL


def test_noalloc_gram_captures_into_a_cuda_graph_and_allocates_nothing():
    """After one warm-up call (which looks up the scratch address), a call changes the
    device's free memory by nothing, and the call captured into a CUDA graph replays
    correctly on new contents of X and Y."""
    n, p, q = 3000, 32, 16
    gen = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(n, p, dtype=torch.float64, device="cuda", generator=gen)
    Y = torch.randn(n, q, dtype=torch.float64, device="cuda", generator=gen)
    C = torch.empty(p * q, dtype=torch.float64, device="cuda")
    ekcg.ekcg_gram_noalloc(n, X, p, Y, q, C)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ekcg.ekcg_gram_noalloc(n, X, p, Y, q, C)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ekcg.ekcg_gram_noalloc(n, X, p, Y, q, C)
    for _ in range(2):
        X.copy_(torch.randn(n, p, dtype=torch.float64, device="cuda", generator=gen))
        Y.copy_(torch.randn(n, q, dtype=torch.float64, device="cuda", generator=gen))
        C.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        Xh, Yh = X.cpu().numpy(), Y.cpu().numpy()
        bound = n * 2.2e-16 * (np.abs(Xh).T @ np.abs(Yh))
        got = C.cpu().numpy().reshape(p, q)
        assert np.all(np.abs(got - Xh.T @ Yh) <= bound)
