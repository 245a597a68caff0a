"""Pins of the oracle's deflated A-CholQR (the rank-revealing breakdown handling): a
column whose Cholesky pivot fails the breakdown rule is dropped from the block instead of
stopping the solve.

* Cholesky with a dropped pivot: the kept part equals LAPACK's Cholesky of G without the
  dropped row and column.
* A right-hand side that vanishes on one of the t domains makes T(r_0) lose a column; the
  deflated solve must then be the solve on the t - 1 domains left (the empty domain's rows
  merged into a neighbour: r_0 is zero there, so T(r_0) is unchanged), iterate for
  iterate, for Algorithm 4 and Algorithm 3 (for Algorithm 6, which splits every new
  residual, the first iterate).
* Without rank loss, deflation changes nothing (bitwise).
* Planted mistakes fail a pin: the dropped column left in the block (dependent-column pin),
  the wrong column dropped (merge pin).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import ekcg_ref as o


def test_cholesky_with_dropped_pivot_matches_lapack_on_the_rest():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((7, 5))
    G = B.T @ B
    G = np.insert(np.insert(G, 2, 0.0, axis=0), 2, 0.0, axis=1)    # 6 x 6, row/col 2 zero
    R, dropped = o.cholesky_upper(G, 1e-14, deflate=True)
    assert dropped == [2]
    keep = [0, 1, 3, 4, 5]
    L = np.linalg.cholesky(G[np.ix_(keep, keep)])
    np.testing.assert_allclose(R[np.ix_(keep, keep)], L.T, rtol=1e-12, atol=1e-12)
    assert np.array_equal(R[2], np.eye(6)[2])
    with pytest.raises(o.Breakdown):
        o.cholesky_upper(np.zeros((3, 3)), 1e-14, deflate=True)
    with pytest.raises(o.Breakdown):
        o.cholesky_upper(G, 1e-14)                                   # no deflation: stop


def test_a_cholqr_with_a_dependent_column_drops_it():
    A = wl.stencil_matrix((9, 8)).to_scipy()
    rng = np.random.default_rng(1)
    W = rng.standard_normal((A.shape[0], 4))
    W[:, 3] = W[:, 0] - 2.0 * W[:, 1]                                # exactly dependent
    Wq, AWq = o.a_cholqr(W, A @ W, 1e-10, deflate=True)
    assert np.all(Wq[:, 3] == 0.0) and np.all(AWq[:, 3] == 0.0)
    np.testing.assert_allclose(Wq[:, :3].T @ (A @ Wq[:, :3]), np.eye(3), atol=1e-12)


def merged(part, d):
    """The partition with domain d merged into its neighbour and the labels compacted."""
    p = part.copy()
    p[p == d] = d - 1 if d > 0 else d + 1
    u = np.unique(p)
    return np.searchsorted(u, p).astype(np.int32), len(u)


@pytest.mark.parametrize("variant", ["sre", "sre2"])
@pytest.mark.parametrize("s", [1, 2])
def test_vanishing_domain_equals_solve_on_remaining_domains(variant, s):
    A = wl.stencil_matrix((16, 14))
    t = 4
    part = wl.partition_boxes((16, 14), t)
    b = wl.rhs_uniform(A.n, 5)
    b[part == 2] = 0.0
    ref = o.solve(A, b, part, t, s, tol=1e-10, maxit=500, variant=variant)
    assert ref.status == o.BREAKDOWN and ref.iters == 0               # without deflation
    got = o.solve(A, b, part, t, s, tol=1e-10, maxit=500, variant=variant, deflate=True,
                  record=True)
    p3, t3 = merged(part, 2)
    want = o.solve(A, b, p3, t3, s, tol=1e-10, maxit=500, variant=variant, record=True)
    assert got.status == want.status == o.OK and got.iters == want.iters
    for xg, xw in zip(got.xs, want.xs):
        assert np.linalg.norm(xg - xw) <= 1e-10 * max(np.linalg.norm(xw), 1.0)


@pytest.mark.parametrize("s", [1, 2])
def test_vanishing_domain_msdo_first_iteration_then_full_rank(s):
    """MSDO-CG (Algorithm 6) splits every new residual: T(r_0) loses the empty domain's
    column, so the first iterate equals the one on the t - 1 remaining domains; from then on
    r_k no longer vanishes there, T(r_k) has full rank again and the solve converges."""
    A = wl.stencil_matrix((16, 14))
    part = wl.partition_boxes((16, 14), 4)
    b = wl.rhs_uniform(A.n, 5)
    b[part == 2] = 0.0
    got = o.solve(A, b, part, 4, s, tol=1e-10, maxit=500, variant="msdo", deflate=True,
                  record=True)
    p3, t3 = merged(part, 2)
    want = o.solve(A, b, p3, t3, s, tol=1e-10, maxit=500, variant="msdo", record=True)
    assert got.status == o.OK
    assert np.linalg.norm(got.xs[1] - want.xs[1]) <= 1e-10 * np.linalg.norm(want.xs[1])
    assert np.linalg.norm(b - A.to_scipy() @ got.x) <= 1.01e-10 * np.linalg.norm(b)


def test_deflation_changes_nothing_without_rank_loss():
    A = wl.stencil_matrix((16, 14))
    part = wl.partition_boxes((16, 14), 4)
    b = wl.rhs_uniform(A.n, 6)
    a = o.solve(A, b, part, 4, 2, tol=1e-10, maxit=500)
    d = o.solve(A, b, part, 4, 2, tol=1e-10, maxit=500, deflate=True)
    assert a.iters == d.iters and np.array_equal(a.x, d.x) and a.hist == d.hist


def test_planted_mistake_dropped_column_kept_fails_the_dependent_column_pin(monkeypatch):
    """Keeping the deflated column (R_ii = 1 but the column not zeroed) leaves a nonzero,
    non-A-orthogonal column in the block."""
    orig = o.right_solve_upper
    monkeypatch.setattr(o, "right_solve_upper", lambda W, R, dropped=(): orig(W, R))
    A = wl.stencil_matrix((9, 8)).to_scipy()
    rng = np.random.default_rng(1)
    W = rng.standard_normal((A.shape[0], 4))
    W[:, 3] = W[:, 0] - 2.0 * W[:, 1]
    Wq, _ = o.a_cholqr(W, A @ W, 1e-10, deflate=True)
    assert not np.all(Wq[:, 3] == 0.0)


def test_planted_mistake_wrong_column_dropped_fails_the_merge_pin(monkeypatch):
    """Dropping the column after the failing pivot (an off-by-one) changes the iterates."""
    orig = o.right_solve_upper
    monkeypatch.setattr(o, "right_solve_upper",
                        lambda W, R, dropped=(): orig(W, R, [min(d + 1, W.shape[1] - 1)
                                                             for d in dropped]))
    A = wl.stencil_matrix((16, 14))
    part = wl.partition_boxes((16, 14), 4)
    b = wl.rhs_uniform(A.n, 5)
    b[part == 2] = 0.0
    p3, t3 = merged(part, 2)
    want = o.solve(A, b, p3, t3, 2, tol=1e-10, maxit=500, record=True)
    try:
        got = o.solve(A, b, part, 4, 2, tol=1e-10, maxit=500, deflate=True, record=True)
    except o.Breakdown:
        return
    same = got.iters == want.iters and all(
        np.linalg.norm(xg - xw) <= 1e-10 * max(np.linalg.norm(xw), 1.0)
        for xg, xw in zip(got.xs, want.xs))
    assert not same
