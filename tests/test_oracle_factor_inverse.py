"""Pins of the oracle's second way to apply the A-CholQR factor (Section 3.1 writes
W R^{-1} and leaves the method open): the product with the explicit inverse.

* R^{-1} from the triangular solve against the identity: (W R^{-1}) R = W, and it equals
  the triangular-solve application to rounding on a well-conditioned factor.
* A planted mistake (the transposed inverse) fails the first pin.
* Whole solves started under factor_application("inverse") reproduce the default solves
  iterate for iterate in exact arithmetic: on Poisson 12 x 12 the iterates agree to 1e-10,
  and the solution is the Galerkin one (A-orthonormal basis, residual orthogonal to it).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import ekcg_ref as o


def test_inverse_application_matches_triangular_solve():
    rng = np.random.default_rng(3)
    B = rng.standard_normal((40, 8))
    R = np.linalg.cholesky(B.T @ B).T
    W = rng.standard_normal((100, 8))
    X = o.right_multiply_inverse(W, R)
    np.testing.assert_allclose(X @ R, W, rtol=0, atol=1e-12 * np.abs(W).max())
    np.testing.assert_allclose(X, o.right_solve_upper(W, R), rtol=0,
                               atol=1e-12 * np.abs(X).max())


def test_planted_transposed_inverse_fails():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((40, 8))
    R = np.linalg.cholesky(B.T @ B).T
    W = rng.standard_normal((100, 8))
    bad = W @ np.linalg.inv(R).T
    assert not np.allclose(bad @ R, W, atol=1e-8)


def test_inverse_solves_equal_default_solves():
    A = wl.stencil_matrix((12, 12))
    b = wl.rhs_uniform(A.n, 5)
    part = wl.partition_boxes((12, 12), 4)
    for variant, s in (("sre", 2), ("sre2", 3)):
        ref = o.solve(A, b, part, 4, s, tol=1e-10, maxit=200, variant=variant)
        with o.factor_application("inverse"):
            got = o.solve(A, b, part, 4, s, tol=1e-10, maxit=200, variant=variant)
        assert got.iters == ref.iters and got.status == ref.status == o.OK
        m = min(len(got.hist), len(ref.hist))
        # relative to the norm itself, and to rho_0 near the rounding floor of the last steps
        np.testing.assert_allclose(got.hist[:m], ref.hist[:m], rtol=1e-8,
                                   atol=1e-12 * ref.hist[0])
        np.testing.assert_allclose(got.x, ref.x, rtol=0, atol=1e-10 * np.abs(ref.x).max())
    # the mode is scoped: outside the block the default applies again
    assert o._FACTOR_APPLICATION[0] == "solve"


def test_inverse_mode_rejects_deflation():
    A = wl.stencil_matrix((8, 8))
    b = wl.rhs_uniform(A.n, 1)
    part = wl.partition_boxes((8, 8), 4)
    with o.factor_application("inverse"):
        with pytest.raises(ValueError):
            o.solve(A, b, part, 4, 1, deflate=True)
