"""Tensor-core split products (tcgen05, float64-accurate) against float64 references.

The CGS update OUT = Y - X C (Section 3.1: W <- W - Q C) and the Gram products C = X^T Y
(CGS coefficients Q^T (A W), the A-CholQR Gram W^T (A W)) run on the bf16 tensor cores as
sums of exact slice products.  Checks, through the C ABI:

* exactness: integer-valued X, C, Y whose product float64 represents exactly come out
  bit-exact (every slice, pair group, integer combination and scale must be right);
* accuracy on random data: |OUT - (Y - X C)| <= eps |Y| + 2 p eps (|X| |C|), the float64
  dot-product error bound, with Y - X C formed in float64 by NumPy and checked against an
  exact (fractions) evaluation on sampled entries;
* the float64-FMA kernel of the same entry point meets the same bound;
* whole solves with the split contraction against the FP64 oracle (iteration count within
  one, residual norms to 1e-6 over the first 20 iterations, x to 1e-8).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as wl
from oracle import ekcg_ref as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_10629_gb300 import ekcg  # noqa: E402

EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def solver():
    A = wl.stencil_matrix((45, 37))           # n = 1665: 13 tiles of 128 rows + 1 row
    S = ekcg.Solver(A, 16, wl.partition_boxes((45, 37), 16), max_s=4)
    yield S
    S.close()


def run_sub(S, X, C, Y, mode):
    p, q = C.shape
    out = torch.empty(X.shape[0] * q, dtype=torch.float64, device="cuda")
    ekcg.ekcg_sub_xc(S.ctx, dev(X), p, dev(C), dev(Y), q, out, mode)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(X.shape[0], q)


@pytest.mark.parametrize("p", [16, 32, 48, 64])
@pytest.mark.parametrize("q", [16, 32])
def test_split_update_exact_on_integers(solver, p, q):
    n = solver.n
    rng = np.random.default_rng(p * 100 + q)
    X = rng.integers(-1000, 1001, (n, p)).astype(np.float64)
    C = rng.integers(-1000, 1001, (p, q)).astype(np.float64)
    Y = rng.integers(-2**40, 2**40, (n, q)).astype(np.float64)
    X[5] = 0.0                                 # a zero row
    C[:, 3] = 0.0                              # a zero column
    ref = Y - X @ C                            # exact: every value is an integer < 2^53
    got = run_sub(solver, X, C, Y, "split")
    assert np.array_equal(got, ref)


def exact_sub(X, C, Y, i, q):
    return float(Fraction(Y[i, q]) - sum(Fraction(X[i, k]) * Fraction(C[k, q])
                                          for k in range(X.shape[1])))


@pytest.mark.parametrize("mode", ["split", "fp64"])
@pytest.mark.parametrize("p,q", [(16, 16), (32, 16), (64, 32), (32, 32), (48, 32)])
def test_update_within_float64_bound(solver, mode, p, q):
    n = solver.n
    rng = np.random.default_rng(7 * p + q)
    X = rng.standard_normal((n, p)) * np.exp(rng.uniform(-20, 20, (n, 1)))
    C = rng.standard_normal((p, q)) * np.exp(rng.uniform(-5, 5, (1, q)))
    Y = X @ C * (1 + 1e-9 * rng.standard_normal((n, q)))   # heavy cancellation, as in CGS
    got = run_sub(solver, X, C, Y, mode)
    ref = Y - X @ C
    bound = EPS * np.abs(Y) + 2 * p * EPS * (np.abs(X) @ np.abs(C))
    assert np.all(np.abs(got - ref) <= bound)
    # the NumPy reference itself against exact rational arithmetic on sampled entries
    for (i, qq) in [(0, 0), (n - 1, q - 1), (n // 2, q // 2), (777, 1)]:
        ex = exact_sub(X, C, Y, i, qq)
        assert abs(got[i, qq] - ex) <= bound[i, qq]


def test_split_update_rejects_other_shapes(solver):
    n = solver.n
    X = np.zeros((n, 24))
    C = np.zeros((24, 16))
    Y = np.zeros((n, 16))
    with pytest.raises(ekcg.EkcgError):
        run_sub(solver, X, C, Y, "split")
    with pytest.raises(ekcg.EkcgError):
        run_sub(solver, np.zeros((n, 16)), np.zeros((16, 8)), np.zeros((n, 8)), "split")


def run_gram(S, X, Y, mode):
    p, q = X.shape[1], Y.shape[1]
    out = torch.empty(p * q, dtype=torch.float64, device="cuda")
    ekcg.ekcg_gram_with(S.ctx, dev(X), p, dev(Y), q, out, mode)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(p, q)


@pytest.mark.parametrize("p", [16, 32, 48, 64])
@pytest.mark.parametrize("q", [16, 32])
def test_split_gram_exact_on_integers(solver, p, q):
    """C = X^T Y over 1665 rows (13 tiles of 128 rows and a ragged one): integer data whose
    inner products float64 represents exactly come out bit-exact."""
    n = solver.n
    rng = np.random.default_rng(p * 10 + q)
    X = rng.integers(-1000, 1001, (n, p)).astype(np.float64)
    Y = rng.integers(-1000, 1001, (n, q)).astype(np.float64)
    X[:, 1] = 0.0
    Y[200:700] = 0.0                            # whole tiles of zero rows in Y
    assert np.array_equal(run_gram(solver, X, Y, "split"), X.T @ Y)


@pytest.mark.parametrize("mode", ["split", "fp64"])
@pytest.mark.parametrize("p,q", [(16, 16), (32, 16), (64, 32), (32, 32), (48, 32)])
def test_gram_within_float64_bound(solver, mode, p, q):
    """|C - X^T Y| <= n eps |X|^T |Y| on data spanning 2^+-29 between rows and columns."""
    n = solver.n
    rng = np.random.default_rng(11 * p + q)
    X = rng.standard_normal((n, p)) * np.exp(rng.uniform(-20, 20, (n, 1)))
    Y = rng.standard_normal((n, q)) * np.exp(rng.uniform(-5, 5, (1, q)))
    got = run_gram(solver, X, Y, mode)
    ref = X.T @ Y
    bound = n * EPS * (np.abs(X).T @ np.abs(Y))
    assert np.all(np.abs(got - ref) <= bound)
    for (i, j) in [(0, 0), (p - 1, q - 1), (p // 2, 1)]:
        ex = float(sum(Fraction(X[k, i]) * Fraction(Y[k, j]) for k in range(n)))
        assert abs(got[i, j] - ex) <= bound[i, j]


def check_solve(A, b, part, t, s, variant="sre", basis="sstep", maxit=2000, mode="split"):
    ref = o.solve(A, b, part, t, s, tol=1e-8, maxit=maxit, variant=variant, basis=basis)
    S = ekcg.Solver(A, t, part, variant=variant, basis=basis, max_s=s,
                    max_basis_bytes=4 << 30, contraction=mode)
    x, it, hist, st = S.solve(dev(b), s=s, tol=1e-8, maxit=maxit)
    x = x.cpu().numpy()
    S.close()
    assert st == ref.status == o.OK, (st, ref.status)
    assert abs(it - ref.iters) <= 1, (it, ref.iters)
    m = min(21, len(hist), len(ref.hist))
    np.testing.assert_allclose(hist[:m], np.array(ref.hist[:m]), rtol=1e-6, atol=0)
    assert np.linalg.norm(b - A.to_scipy() @ x) <= 1.01e-8 * np.linalg.norm(b)
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("s", [1, 2, 4])
def test_split_solver_ani3d_t32(s):
    A = wl.stencil_matrix((24, 24, 24), aniso=(1.0, 1.0, 1e-3))
    check_solve(A, wl.rhs_uniform(A.n, 1), wl.partition_boxes((24, 24, 24), 32), 32, s)


@pytest.mark.parametrize("mode", ["split", "fp64"])
@pytest.mark.parametrize("variant,basis", [("sre2", "sstep"), ("msdo", "sstep"),
                                           ("msdo", "ca7")])
def test_split_solver_sky3d_t16(variant, basis, mode):
    """Sky3D-like 16^3, t = 16, s = 4.  (s-step SRE-CG with the two-block window is left
    out here: on this 1e3-contrast operator its residual norms jump by 2x-3x between
    iterations and neither float64 arithmetic on the GPU follows the oracle beyond about ten
    iterations; SRE-CG2 and MSDO-CG, which orthonormalise against every previous block,
    do.)"""
    A = wl.stencil_matrix((16, 16, 16), kappa=wl.kappa_skyscraper3d(16))
    check_solve(A, wl.rhs_uniform(A.n, 2), wl.partition_boxes((16, 16, 16), 16), 16, 4,
                variant, basis, mode=mode)


def test_split_solver_poisson2d_ragged():
    A = wl.stencil_matrix((45, 37))
    check_solve(A, wl.rhs_uniform(A.n, 11), wl.partition_boxes((45, 37), 16), 16, 2)
