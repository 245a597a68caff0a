"""Planted mistakes: each test swaps one oracle step for a plausible wrong version (on the
CPU, inside the oracle only) and checks that the pins catch it.  This shows that the pins
constrain every step of the oracle, not just its final answer."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import ekcg_ref as o


def _problem():
    A = wl.stencil_matrix((12, 12))
    part = wl.partition_boxes((12, 12), 4)
    return A, wl.rhs_uniform(A.n, 0), part


def pins_hold():
    """A compact subset of the pins: t = s = 1 equals CG, enlarged Galerkin projection for
    s = 2, A-orthonormality, and the dense Cholesky solution."""
    A, b, part = _problem()
    Asp = A.to_scipy()
    try:
        # (1) t = s = 1 reproduces CG over 10 iterations
        ref = o.cg(A, b, tol=1e-14, maxit=10, record=True)
        res = o.solve(A, b, np.zeros(A.n, np.int32), 1, 1, tol=1e-14, maxit=10, record=True)
        for k in range(1, 11):
            if np.linalg.norm(res.xs[k] - ref.xs[k]) > 1e-10 * np.linalg.norm(ref.xs[k]):
                return False
        # (2) Galerkin over K_{2k,4}
        res = o.solve(A, b, part, 4, 2, tol=1e-14, maxit=3, record=True)
        Q = np.linalg.qr(o.split_T(b, part, 4))[0]
        B = Q
        for k in range(1, 4):
            while Q.shape[1] < 2 * k * 4:                  # K_{2k,4}: 2k blocks
                B = Asp @ B
                for _rep in range(2):
                    B = B - Q @ (Q.T @ B)
                B = np.linalg.qr(B)[0]
                Q = np.hstack([Q, B])
            xk = Q @ np.linalg.solve(Q.T @ (Asp @ Q), Q.T @ b)
            if np.linalg.norm(res.xs[k] - xk) > 1e-8 * np.linalg.norm(xk):
                return False
        # (3) A-orthonormal basis, (4) dense solve
        res = o.solve(A, b, part, 4, 2, tol=1e-10, maxit=200, variant="sre2", record=True)
        if res.status != o.OK or max(res.orth_loss[:5]) > 1e-11:
            return False
        x_star = sla.cho_solve(sla.cho_factor(Asp.toarray()), b)
        return np.linalg.norm(res.x - x_star) <= 1e-7 * np.linalg.norm(x_star)
    except (o.Breakdown, np.linalg.LinAlgError, ValueError, IndexError):
        return False


def test_unmodified_oracle_passes():
    assert pins_hold()


def test_euclidean_gram_in_cholqr_is_caught(monkeypatch):
    def bad(W, AW, tol):
        R = o.cholesky_upper(W.T @ W, tol)                # forgot A in the Gram
        return o.right_solve_upper(W, R), o.right_solve_upper(AW, R)
    monkeypatch.setattr(o, "a_cholqr", bad)
    assert not pins_hold()


def test_transposed_triangular_factor_is_caught(monkeypatch):
    monkeypatch.setattr(o, "right_solve_upper",
                        lambda W, R: sla.solve_triangular(R, W.T, trans="N", lower=False).T)
    assert not pins_hold()


def test_stale_AW_in_cgs_is_caught(monkeypatch):
    def bad(W, AW, Q, matmul):
        for _ in range(2):
            C = Q.T @ AW
            W = W - Q @ C                                  # A W never recomputed
        return W, AW
    monkeypatch.setattr(o, "cgs2_against", bad)
    assert not pins_hold()


def test_coefficient_rows_in_wrong_order_is_caught(monkeypatch):
    def bad(W, AW, Q, matmul):
        for _ in range(2):
            C = Q.T @ AW
            W = W - Q @ C[::-1]                            # rows of C in the wrong order
            AW = matmul(W)
        return W, AW
    monkeypatch.setattr(o, "cgs2_against", bad)
    assert not pins_hold()


def test_residual_sign_is_caught(monkeypatch):
    def bad(ctx, res, x, r, V, AV):
        alpha = V.T @ r
        x = x + V @ alpha
        r = r + AV @ alpha                                 # wrong sign
        return x, r, float(np.linalg.norm(r))
    monkeypatch.setattr(o, "_update", bad)
    assert not pins_hold()


def test_split_dropping_a_domain_is_caught(monkeypatch):
    real = o.split_T

    def bad(r, part, t):
        T = real(r, part, t)
        if t > 1:
            T[:, t - 1] = 0.0                              # last domain lost
        return T
    monkeypatch.setattr(o, "split_T", bad)
    assert not pins_hold()


def test_single_pass_cgs_loses_orthogonality_on_hard_problem(monkeypatch):
    """One CGS pass instead of two: invisible on easy problems, caught by the
    A-orthonormality pin on a skyscraper-like matrix (coefficient jumps 1 / 1e3)."""
    A = wl.stencil_matrix((8, 8, 8), kappa=wl.kappa_skyscraper3d(8, block=2))
    part = wl.partition_boxes((8, 8, 8), 8)
    b = wl.rhs_uniform(A.n, 0)

    def loss():
        res = o.solve(A, b, part, 8, 3, tol=1e-8, maxit=30, variant="sre2", record=True)
        return max(res.orth_loss[:6])

    good = loss()

    def bad(W, AW, Q, matmul):
        C = Q.T @ AW
        W = W - Q @ C
        return W, matmul(W)
    monkeypatch.setattr(o, "cgs2_against", bad)
    assert good <= 1e-11 and loss() > 1e-11
