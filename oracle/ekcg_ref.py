"""FP64 CPU oracle for the s-step enlarged Krylov subspace CG methods.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of `__graft_entry__` and the
CPU-baseline leg of `bench.py` may import this module.  The CUDA library never calls it,
shares no code with it, and does not fall back to it.

Plain, slow, obviously-correct NumPy/SciPy code in float64.  Each function follows the
paper (Moufawad, "Numerical Stability of s-step Enlarged Krylov Subspace Conjugate Gradient
methods", arXiv:1804.10629) step by step; the section / algorithm / equation it follows is
named in its docstring.  Library primitives used as steps: sparse matrix x dense block
(scipy.sparse), dense matrix products (NumPy/BLAS), Householder QR (numpy.linalg.qr) and
triangular solves (scipy.linalg.solve_triangular).

Everything works in the caller's (natural) row order.  The splitting operator T uses the
partition array directly: T(r)[i, part[i]] = r[i].  The domain permutation of Section 4
(rows reordered so that domains are contiguous) is a storage choice; `domain_perm` gives
the permutation the GPU library must reproduce.

Readings where the paper is silent or refers to the author's thesis:
  * CGS2 against Q (thesis Alg. 18, not printed): two passes of C = Q^T (A W),
    W <- W - Q C.  The A-inner products use a fresh sparse product A W of the current W in
    each pass (and one more after the second pass for the Gram matrix below).
  * A-CholQR (thesis Alg. 21): G = W^T (A W) = R^T R (upper Cholesky of the upper
    triangle of G), W <- W R^{-1}; the product A W is carried through the triangular
    factor, A W <- (A W) R^{-1}, and serves as the next candidate block A W_j and as the
    block A V of the residual update.
  * Pre-CholQR (thesis Alg. 23): thin Euclidean QR W = Z S with diag(S) > 0 first, then
    A-CholQR of Z (A Z = (A W) S^{-1}, again carried only through a triangular factor).
  * Why fresh products: carrying A W through the CGS updates as well (A W <- A W - (A Q) C)
    lets the error of A Q grow by the size of C at every block; on the skyscraper problem
    the A-orthogonality of s-step SRE-CG2 then decays to O(1) and the Gram matrix turns
    indefinite, whereas Section 4 reports s-step SRE-CG2 converging in k_s iterations on
    every test matrix.  `carried_cgs=True` keeps that carried form for comparison;
    `explicit_AW=True` also recomputes A W after the triangular factor.
  * Missing window blocks in the first iterations (W_{j-2} for j < 3) are skipped.
  * Stopping rule: while rho > tol*rho0 and iterations < maxit, rho = ||r_k||_2 of the
    recursively updated residual, checked once per s-step iteration.
  * Breakdown: a Cholesky pivot d_i <= breakdown_tol * |G_ii| (or a non-finite one) stops
    the solve with status BREAKDOWN and the current iterate.  With deflate=True (A-CholQR
    only) such a column is instead deflated, as enlarged CG deflates dependent directions
    (Section 2, the reference to ECG): it is dropped from the block (set to zero in W and
    A W, no Schur update from it), the other columns are A-orthonormalised among
    themselves, and the solve continues with fewer directions; a non-finite pivot, or a
    block whose columns are all deflated, is still a breakdown.
  * CA SRE-CG window: the last (s+1)t basis vectors; CA SRE-CG2 / (CA) MSDO-CG: all.
  * Inside a CA block V the columns are power-major: column p*t + i belongs to A^p W_i.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

OK = 0
MAXIT = 1
BREAKDOWN = -3

VARIANTS = ("sre", "sre2", "msdo")
BASES = ("sstep", "ca5", "ca7")
ORTHS = ("acholqr", "precholqr")


class Breakdown(Exception):
    """Raised when a Cholesky pivot fails the breakdown rule."""


@dataclasses.dataclass
class Result:
    x: np.ndarray
    iters: int
    hist: List[float]
    status: int
    xs: List[np.ndarray] = dataclasses.field(default_factory=list)       # x_0, x_1, ...
    orth_loss: List[float] = dataclasses.field(default_factory=list)     # max|Q^T A Q - I|
    pg_loss: List[float] = dataclasses.field(default_factory=list)       # ||V_k^T r_k|| / ||r_k||
    residuals: List[np.ndarray] = dataclasses.field(default_factory=list)  # r_0, r_1, ...
    basis: Optional[np.ndarray] = None   # stored Q at exit (full-history methods, record=True)
    spmm_count: int = 0


# ----------------------------------------------------------------------------------------
# Domain decomposition: permutation and the splitting operator T (Section 2, Section 4)
# ----------------------------------------------------------------------------------------

def domain_perm(part: np.ndarray) -> np.ndarray:
    """Row permutation that makes the t domains contiguous (Section 4: the matrix is
    reordered by the k-way partition).  Stable: rows keep their natural order inside a
    domain.  perm[i] = original row placed at position i."""
    return np.argsort(np.asarray(part), kind="stable").astype(np.int64)


def split_T(r: np.ndarray, part: np.ndarray, t: int) -> np.ndarray:
    """T(r) of Section 2: the n x t matrix whose column d is r restricted to domain d
    (the projection of r on the d-th domain), zero elsewhere."""
    n = r.shape[0]
    T = np.zeros((n, t))
    T[np.arange(n), np.asarray(part)] = r
    return T


# ----------------------------------------------------------------------------------------
# A-orthonormalisation (Section 3.1 and Section 4: CGS2 + A-CholQR or Pre-CholQR)
# ----------------------------------------------------------------------------------------

def cholesky_upper(G: np.ndarray, breakdown_tol: float, deflate: bool = False):
    """Upper Cholesky factor R (G = R^T R) from the upper triangle of G, right-looking.
    Breakdown rule: pivot d_i <= breakdown_tol*|G_ii| or non-finite.  With deflate=True a
    finite pivot that fails the rule drops column i instead: row i of R becomes e_i^T (no
    Schur update from it) and i is listed in the returned `dropped`; then (R, dropped) is
    returned, and a block with every column dropped is a breakdown."""
    m = G.shape[0]
    S = np.triu(np.array(G, dtype=np.float64))
    R = np.zeros((m, m))
    dropped = []
    for i in range(m):
        d = S[i, i]
        if not np.isfinite(d) or d <= breakdown_tol * abs(G[i, i]):
            if not deflate or not np.isfinite(d):
                raise Breakdown(f"pivot {i}: {d!r} vs G_ii {G[i, i]!r}")
            R[i, i] = 1.0
            dropped.append(i)
            continue
        R[i, i] = math.sqrt(d)
        R[i, i + 1:] = S[i, i + 1:] / R[i, i]
        S[i + 1:, i + 1:] -= np.triu(np.outer(R[i, i + 1:], R[i, i + 1:]))
    if not deflate:
        return R
    if len(dropped) == m:
        raise Breakdown("every column of the block deflated")
    return R, dropped


def right_solve_upper(W: np.ndarray, R: np.ndarray, dropped=()) -> np.ndarray:
    """W R^{-1} for upper-triangular R (solves X R = W); the columns in `dropped`
    (deflated by cholesky_upper) are set to zero."""
    X = sla.solve_triangular(R, W.T, trans="T", lower=False).T
    if len(dropped):
        X[:, list(dropped)] = 0.0
    return X


def right_multiply_inverse(W, R):
    """W R^{-1} by the explicit inverse of the upper-triangular R (R^{-1} from a triangular
    solve against the identity), then one matrix product: the other way to apply the
    factor of A-CholQR, which the paper leaves open (Section 3.1 writes W R^{-1})."""
    Rinv = sla.solve_triangular(R, np.eye(R.shape[0]), lower=False)
    return W @ Rinv


# How A-CholQR applies its factor: "solve" (a triangular solve, the default) or "inverse"
# (the product with R^{-1}).  Scoped by `factor_application`; read when a solve starts.
_FACTOR_APPLICATION = ["solve"]


class factor_application:
    """with factor_application("inverse"): solves started inside apply W R^{-1} as the
    product with the explicit inverse (without deflation)."""

    def __init__(self, mode):
        if mode not in ("solve", "inverse"):
            raise ValueError(mode)
        self.mode = mode

    def __enter__(self):
        self.prev = _FACTOR_APPLICATION[0]
        _FACTOR_APPLICATION[0] = self.mode
        return self

    def __exit__(self, *exc):
        _FACTOR_APPLICATION[0] = self.prev
        return False


def a_cholqr_inverse(W, AW, breakdown_tol):
    """A-CholQR applying its factor by the explicit inverse: G = W^T A W = R^T R,
    W <- W R^{-1}, A W <- (A W) R^{-1}."""
    R = cholesky_upper(W.T @ AW, breakdown_tol)
    return right_multiply_inverse(W, R), right_multiply_inverse(AW, R)


def a_cholqr(W, AW, breakdown_tol, deflate=False):
    """A-CholQR: G = W^T A W = R^T R, W <- W R^{-1} (and A W <- A W R^{-1}); with
    deflate=True the columns whose pivots fail the breakdown rule are dropped (zeroed)."""
    G = W.T @ AW
    if deflate:
        R, dropped = cholesky_upper(G, breakdown_tol, deflate=True)
        return right_solve_upper(W, R, dropped), right_solve_upper(AW, R, dropped)
    R = cholesky_upper(G, breakdown_tol)
    return right_solve_upper(W, R), right_solve_upper(AW, R)


def pre_cholqr(W, AW, breakdown_tol):
    """Pre-CholQR: Euclidean thin QR W = Z S (diag(S) > 0), then A-CholQR of Z."""
    Z, S = np.linalg.qr(W)
    sgn = np.where(np.diag(S) < 0, -1.0, 1.0)
    Z = Z * sgn
    S = S * sgn[:, None]
    dS = np.diag(S) ** 2
    gdiag = np.einsum("ij,ij->j", W, W)
    if not np.all(np.isfinite(dS)) or np.any(dS <= breakdown_tol * gdiag):
        raise Breakdown("Euclidean QR pivot")
    return a_cholqr(Z, right_solve_upper(AW, S), breakdown_tol)


def cgs2_against(W, AW, Q, matmul):
    """CGS2 A-orthonormalisation of W against the A-orthonormal Q: two passes of
    C = Q^T (A W), W <- W - Q C, where A W is a fresh sparse product of the current W
    (`AW` holds A W on entry; `matmul(X)` returns A X).  Returns W and A W."""
    for _ in range(2):
        C = Q.T @ AW
        W = W - Q @ C
        AW = matmul(W)
    return W, AW


def cgs2_against_carried(W, AW, Q, AQ):
    """CGS2 with A W carried by the same recurrence, A W <- A W - (A Q) C (the form whose
    A-orthogonality decays; kept for comparison only)."""
    for _ in range(2):
        C = Q.T @ AW
        W = W - Q @ C
        AW = AW - AQ @ C
    return W, AW


# ----------------------------------------------------------------------------------------
# Helpers shared by the solvers
# ----------------------------------------------------------------------------------------

class _Ctx:
    """Per-solve state: the operator, options, the optional split preconditioner and
    bookkeeping."""

    def __init__(self, A, part, t, orth, breakdown_tol, explicit_AW, record, carried_cgs=False,
                 precond=None, deflate=False):
        self.A = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
        self.part = np.asarray(part)
        self.t = t
        self.orth = orth
        self.tol_bd = breakdown_tol
        self.explicit = explicit_AW
        self.carried = carried_cgs
        self.record = record
        self.pre = precond
        self.deflate = deflate
        if deflate and orth != "acholqr":
            raise ValueError("deflation is defined for A-CholQR")
        self.inverse = _FACTOR_APPLICATION[0] == "inverse"
        if self.inverse and (deflate or orth != "acholqr"):
            raise ValueError("the explicit-inverse application is defined for A-CholQR")
        self.spmm = 0

    def matmul(self, W):
        self.spmm += 1
        return self.A @ W

    def first_block(self, r):
        """The block built from a residual: T(r), or with a split preconditioner
        M = L L^T, L^{-T} T(L^{-1} r) (Section 5, Algorithms 8-10)."""
        if self.pre is None:
            return split_T(r, self.part, self.t)
        return self.pre.solve_LT(split_T(self.pre.solve_L(r), self.part, self.t))

    def candidate(self, AW):
        """The next block from A W_{j-1}: A W_{j-1} itself, or M^{-1} A W_{j-1} with a
        split preconditioner (Section 5)."""
        if self.pre is None:
            return AW
        return self.pre.apply(AW)

    def self_orth(self, W, AW):
        if self.orth == "acholqr" and self.inverse:
            W, AW = a_cholqr_inverse(W, AW, self.tol_bd)
        elif self.orth == "acholqr":
            W, AW = (a_cholqr(W, AW, self.tol_bd, deflate=True) if self.deflate
                     else a_cholqr(W, AW, self.tol_bd))
        elif self.orth == "precholqr":
            W, AW = pre_cholqr(W, AW, self.tol_bd)
        else:
            raise ValueError(self.orth)
        if self.explicit:
            AW = self.A @ W
        return W, AW

    def against(self, W, AW, blocks):
        if isinstance(blocks, _Basis):
            if blocks.m == 0:
                return W, AW
            Q, AQ = blocks.Q, blocks.AQ
        else:
            if not blocks:
                return W, AW
            Q = np.hstack([b[0] for b in blocks])
            AQ = np.hstack([b[1] for b in blocks])
        if self.carried:
            return cgs2_against_carried(W, AW, Q, AQ)
        return cgs2_against(W, AW, Q, self.matmul)


class _Basis:
    """Stored basis vectors Q and their products A Q as contiguous n x m arrays (grown by
    doubling), so that a full-history solve does not re-concatenate Q every step."""

    def __init__(self, n):
        self.n = n
        self.m = 0
        self._Q = np.empty((n, 0))
        self._AQ = np.empty((n, 0))

    def append(self, W, AW):
        w = W.shape[1]
        if self.m + w > self._Q.shape[1]:
            cap = max(2 * self._Q.shape[1], self.m + w, 16)
            Q = np.empty((self.n, cap))
            AQ = np.empty((self.n, cap))
            Q[:, :self.m] = self._Q[:, :self.m]
            AQ[:, :self.m] = self._AQ[:, :self.m]
            self._Q, self._AQ = Q, AQ
        self._Q[:, self.m:self.m + w] = W
        self._AQ[:, self.m:self.m + w] = AW
        self.m += w

    @property
    def Q(self):
        return self._Q[:, :self.m]

    @property
    def AQ(self):
        return self._AQ[:, :self.m]

    def blocks(self, t):
        return [(self.Q[:, i:i + t], self.AQ[:, i:i + t]) for i in range(0, self.m, t)]


def _orth_loss_arrays(Q, AQ):
    return float(np.max(np.abs(Q.T @ AQ - np.eye(Q.shape[1]))))


def _orth_loss(blocks):
    if isinstance(blocks, _Basis):
        return _orth_loss_arrays(blocks.Q, blocks.AQ)
    Q = np.hstack([b[0] for b in blocks])
    AQ = np.hstack([b[1] for b in blocks])
    return _orth_loss_arrays(Q, AQ)


def _start(A, b, x0):
    Asp = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
    x = np.zeros_like(b, dtype=np.float64) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - Asp @ x
    return x, r, float(np.linalg.norm(r))


def _update(ctx, res, x, r, V, AV):
    """Lines 'alpha = V^T r_{k-1}; x_k = x_{k-1} + V alpha; r_k = r_{k-1} - AV alpha'."""
    alpha = V.T @ r
    x = x + V @ alpha
    r = r - AV @ alpha
    return x, r, float(np.linalg.norm(r))


def _finish(res, x, rho, rho0, tol, k):
    res.x = x
    res.iters = k - 1
    if res.status != BREAKDOWN:
        res.status = OK if rho <= tol * rho0 else MAXIT
    return res


def _record(ctx, res, x, r, V=None, blocks=None):
    if not ctx.record:
        return
    res.xs.append(x.copy())
    res.residuals.append(r.copy())
    if V is not None:
        nr = np.linalg.norm(r)
        res.pg_loss.append(float(np.linalg.norm(V.T @ r) / (nr if nr > 0 else 1.0)))
    if blocks is not None and (not isinstance(blocks, list) or blocks):
        res.orth_loss.append(_orth_loss(blocks))


# ----------------------------------------------------------------------------------------
# Classical CG (Section 2)
# ----------------------------------------------------------------------------------------

def cg(A, b, x0=None, tol=1e-8, maxit=10000, record=False) -> Result:
    """Conjugate Gradient as stated in Section 2: p_1 = r_0, p_k = r_{k-1} + beta_k p_{k-1},
    alpha_k = ||r_{k-1}||^2 / ||p_k||_A^2, beta_k = ||r_{k-1}||^2 / ||r_{k-2}||^2,
    x_k = x_{k-1} + alpha_k p_k, r_k = r_{k-1} - alpha_k A p_k; same stopping rule as the
    enlarged algorithms (rho = ||r_k||_2 > tol*rho_0 and k < k_max)."""
    Asp = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
    x, r, rho0 = _start(A, b, x0)
    res = Result(x=x, iters=0, hist=[rho0], status=OK)
    if record:
        res.xs.append(x.copy())
        res.residuals.append(r.copy())
    rho, k = rho0, 1
    p = None
    rr_prev = None
    kmax = maxit + 1
    while rho > tol * rho0 and k < kmax:
        rr = float(r @ r)
        p = r.copy() if k == 1 else r + (rr / rr_prev) * p
        Ap = Asp @ p
        alpha = rr / float(p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rr_prev = rr
        rho = float(np.linalg.norm(r))
        res.hist.append(rho)
        if record:
            res.xs.append(x.copy())
            res.residuals.append(r.copy())
        k += 1
    return _finish(res, x, rho, rho0, tol, k)


# ----------------------------------------------------------------------------------------
# s-step SRE-CG (Algorithm 4) and s-step SRE-CG2 (Algorithm 3)
# ----------------------------------------------------------------------------------------

def sstep_sre_cg(A, b, part, t, s, tol=1e-8, maxit=1000, x0=None, orth="acholqr",
                 full_history=False, breakdown_tol=1e-14, explicit_AW=False,
                 record=False, carried_cgs=False, precond=None, deflate=False) -> Result:
    """s-step SRE-CG (Algorithm 4); with full_history=True, s-step SRE-CG2 (Algorithm 3).

    Iteration k builds s blocks W_j..W_{j+s-1}, j = (k-1)s+1.  W_1 = T(r_0) is only
    A-orthonormalised against itself; every later W_j = A W_{j-1} is A-orthonormalised
    against W_{j-2}, W_{j-1} (Alg. 4) or against all previous blocks (Alg. 3), then against
    itself.  Then alpha = V^T r_{k-1}, x_k = x_{k-1} + V alpha, r_k = r_{k-1} - A V alpha.
    With a split preconditioner M = L L^T (`precond`, Algorithms 8 and 9): W_1 =
    L^{-T} T(L^{-1} r_0) and W_j = M^{-1} A W_{j-1}; the A-orthonormalisation and the
    updates are unchanged.
    """
    ctx = _Ctx(A, part, t, orth, breakdown_tol, explicit_AW, record, carried_cgs, precond,
               deflate)
    x, r, rho0 = _start(A, b, x0)
    res = Result(x=x, iters=0, hist=[rho0], status=OK)
    _record(ctx, res, x, r)
    r0 = r.copy()
    window = []                      # Alg. 4: (W, AW) of the last two blocks
    full = _Basis(b.shape[0])        # Alg. 3: all blocks
    last = None                      # (W_{j-1}, A W_{j-1})
    rho, k = rho0, 1
    kmax = maxit + 1
    try:
        while rho > tol * rho0 and k < kmax:
            Vb = []
            for i in range(s):
                if k == 1 and i == 0:
                    W = ctx.first_block(r0)
                    AW = ctx.matmul(W)
                else:
                    W = ctx.candidate(last[1])             # W_j = (M^{-1}) A W_{j-1}
                    AW = ctx.matmul(W)
                    W, AW = ctx.against(W, AW, full if full_history else window)
                W, AW = ctx.self_orth(W, AW)
                last = (W, AW)
                Vb.append(last)
                if full_history:
                    full.append(W, AW)
                else:
                    window = (window + [last])[-2:]
            V = np.hstack([v[0] for v in Vb])
            AV = np.hstack([v[1] for v in Vb])
            x, r, rho = _update(ctx, res, x, r, V, AV)
            res.hist.append(rho)
            _record(ctx, res, x, r, V, full if full_history else Vb)
            k += 1
    except Breakdown:
        res.status = BREAKDOWN
    res.spmm_count = ctx.spmm
    if record and full_history:
        res.basis = full.Q.copy()
    return _finish(res, x, rho, rho0, tol, k)


def sstep_sre_cg2(*args, **kw) -> Result:
    """s-step SRE-CG2 (Algorithm 3): Algorithm 4 with orthonormalisation against all Q."""
    kw["full_history"] = True
    return sstep_sre_cg(*args, **kw)


# ----------------------------------------------------------------------------------------
# s-step MSDO-CG (Algorithm 6, modified enlarged Krylov subspace of Section 3.2)
# ----------------------------------------------------------------------------------------

def sstep_msdo_cg(A, b, part, t, s, tol=1e-8, maxit=1000, x0=None, orth="acholqr",
                  breakdown_tol=1e-14, explicit_AW=False, record=False,
                  carried_cgs=False, precond=None, deflate=False) -> Result:
    """s-step MSDO-CG (Algorithm 6).  Iteration k: W_1 = T(r_{k-1}) A-orthonormalised
    against Q (k > 1) and itself; W_{i+1} = A W_i against Q and itself, i = 1..s-1; every
    block joins V and Q.  Then alpha = V^T r_{k-1} and the x / r updates.  With a split
    preconditioner (Algorithm 10): W_1 = L^{-T} T(L^{-1} r_{k-1}), W_{i+1} = M^{-1} A W_i."""
    ctx = _Ctx(A, part, t, orth, breakdown_tol, explicit_AW, record, carried_cgs, precond,
               deflate)
    x, r, rho0 = _start(A, b, x0)
    res = Result(x=x, iters=0, hist=[rho0], status=OK)
    _record(ctx, res, x, r)
    Qb = _Basis(b.shape[0])
    rho, k = rho0, 1
    kmax = maxit + 1
    try:
        while rho > tol * rho0 and k < kmax:
            Vb = []
            W = ctx.first_block(r)
            AW = ctx.matmul(W)
            W, AW = ctx.against(W, AW, Qb)
            W, AW = ctx.self_orth(W, AW)
            Vb.append((W, AW))
            Qb.append(W, AW)
            for i in range(1, s):
                W = ctx.candidate(Vb[-1][1])               # W_{i+1} = (M^{-1}) A W_i
                AW = ctx.matmul(W)
                W, AW = ctx.against(W, AW, Qb)
                W, AW = ctx.self_orth(W, AW)
                Vb.append((W, AW))
                Qb.append(W, AW)
            V = np.hstack([v[0] for v in Vb])
            AV = np.hstack([v[1] for v in Vb])
            x, r, rho = _update(ctx, res, x, r, V, AV)
            res.hist.append(rho)
            _record(ctx, res, x, r, V, Qb)
            k += 1
    except Breakdown:
        res.status = BREAKDOWN
    res.spmm_count = ctx.spmm
    if record:
        res.basis = Qb.Q.copy()
    return _finish(res, x, rho, rho0, tol, k)


# ----------------------------------------------------------------------------------------
# Communication-avoiding forms: CA-Arnoldi (Algorithm 5) and modified CA-Arnoldi (Alg. 7)
# ----------------------------------------------------------------------------------------

def _split_blocks(V, AV, t):
    return [(V[:, i:i + t], AV[:, i:i + t]) for i in range(0, V.shape[1], t)]


def ca_enlarged_cg(A, b, part, t, s, tol=1e-8, maxit=1000, x0=None, orth="acholqr",
                   variant="sre", arnoldi="alg7", breakdown_tol=1e-14, explicit_AW=False,
                   record=False, carried_cgs=False, precond=None, deflate=False) -> Result:
    """CA SRE-CG / CA SRE-CG2 / CA MSDO-CG: Algorithms 4 / 3 / 6 with the basis built by
    the CA-Arnoldi A-orthonormalisation (Algorithm 5, arnoldi='alg5') or the modified
    CA-Arnoldi (Algorithm 7, arnoldi='alg7').

    Algorithm 5: W_j = W_{j-1} (k = 1) or A W_{j-1} (k > 1); W_{j+i} = A W_{j+i-1} for
    i = 1..s-1; V = [W_j .. W_{j+s-1}] is A-orthonormalised against Q (k > 1), then itself.
    Algorithm 7: as Alg. 5, but W_j is first A-orthonormalised against Q (k > 1) and against
    itself before the powers are formed.
    Input block W_{j-1}: T(r_0) at k = 1, else the last t vectors of the previous V
    (SRE variants); T(r_{k-1}) at every k for MSDO, where W_j = W_{j-1} replaces
    W_j = A W_{j-1} (Section 3.2).
    Q: the last (s+1)t vectors (CA SRE-CG) or all previous vectors (CA SRE-CG2, CA MSDO-CG).
    With a split preconditioner (Section 5): every A W_{j+i-1} that forms a new block is
    replaced by M^{-1} A W_{j+i-1}, and the input block T(r) by L^{-T} T(L^{-1} r).
    """
    if variant not in VARIANTS or arnoldi not in ("alg5", "alg7"):
        raise ValueError((variant, arnoldi))
    ctx = _Ctx(A, part, t, orth, breakdown_tol, explicit_AW, record, carried_cgs, precond,
               deflate)
    x, r, rho0 = _start(A, b, x0)
    res = Result(x=x, iters=0, hist=[rho0], status=OK)
    _record(ctx, res, x, r)
    r0 = r.copy()
    window = []          # CA SRE-CG: t-wide column blocks of the last V's
    full = _Basis(b.shape[0])   # CA SRE-CG2 / CA MSDO-CG: all previous vectors
    last = None          # (W_{j-1}, A W_{j-1}) carried from the previous iteration
    rho, k = rho0, 1
    kmax = maxit + 1
    try:
        while rho > tol * rho0 and k < kmax:
            Qb = window[-(s + 1):] if variant == "sre" else full
            # first block W_j
            if variant == "msdo":
                Wj = ctx.first_block(r)
                AWj = ctx.matmul(Wj)
            elif k == 1:
                Wj = ctx.first_block(r0)
                AWj = ctx.matmul(Wj)
            else:
                Wj = ctx.candidate(last[1])                # W_j = (M^{-1}) A W_{j-1}
                AWj = ctx.matmul(Wj)
            if arnoldi == "alg7":
                if k > 1:
                    Wj, AWj = ctx.against(Wj, AWj, Qb)
                Wj, AWj = ctx.self_orth(Wj, AWj)
            Vb = [(Wj, AWj)]
            for i in range(1, s):
                W = ctx.candidate(Vb[-1][1])               # W_{j+i} = (M^{-1}) A W_{j+i-1}
                Vb.append((W, ctx.matmul(W)))
            V = np.hstack([v[0] for v in Vb])
            AV = np.hstack([v[1] for v in Vb])
            if k > 1:
                V, AV = ctx.against(V, AV, Qb)
            V, AV = ctx.self_orth(V, AV)
            newb = _split_blocks(V, AV, t)
            if variant == "sre":
                window = (window + newb)[-(2 * s + 1):]
            else:
                full.append(V, AV)
            last = newb[-1]
            x, r, rho = _update(ctx, res, x, r, V, AV)
            res.hist.append(rho)
            _record(ctx, res, x, r, V, full if variant != "sre" else newb)
            k += 1
    except Breakdown:
        res.status = BREAKDOWN
    res.spmm_count = ctx.spmm
    if record and variant != "sre":
        res.basis = full.Q.copy()
    return _finish(res, x, rho, rho0, tol, k)


# ----------------------------------------------------------------------------------------
# Restructured SRE-CG (Algorithm 2) and SRE-CG2 (Algorithm 1)
# ----------------------------------------------------------------------------------------

def restructured_sre_cg(A, b, part, t, s, tol=1e-8, maxit=1000, x0=None, orth="acholqr",
                        full_history=False, breakdown_tol=1e-14, record=False,
                        carried_cgs=False, deflate=False) -> Result:
    """Restructured SRE-CG (Algorithm 2; Algorithm 1 with full_history=True): build the s
    blocks as in Alg. 4 / Alg. 3, then s sequential updates alpha = W_i^T r_{i-1},
    x_i = x_{i-1} + W_i alpha, r_i = r_{i-1} - A W_i alpha.  The residual norm is checked
    once every s updates; `iters` counts those outer steps (k_s of Tables 2-3).  With
    record=True, `xs` holds every inner iterate x_0, x_1, x_2, ... (for s = 1 this is
    SRE-CG / SRE-CG2 itself)."""
    ctx = _Ctx(A, part, t, orth, breakdown_tol, False, record, carried_cgs, None, deflate)
    x, r, rho0 = _start(A, b, x0)
    res = Result(x=x, iters=0, hist=[rho0], status=OK)
    if record:
        res.xs.append(x.copy())
    r0 = r.copy()
    window = []
    full = _Basis(b.shape[0])
    last = None
    rho, k = rho0, 1
    kmax = maxit + 1
    try:
        while rho > tol * rho0 and k < kmax:
            Vb = []
            for i in range(s):
                if k == 1 and i == 0:
                    W = ctx.first_block(r0)
                    AW = ctx.matmul(W)
                else:
                    W = ctx.candidate(last[1])             # W_j = (M^{-1}) A W_{j-1}
                    AW = ctx.matmul(W)
                    W, AW = ctx.against(W, AW, full if full_history else window)
                W, AW = ctx.self_orth(W, AW)
                last = (W, AW)
                Vb.append(last)
                if full_history:
                    full.append(W, AW)
                else:
                    window = (window + [last])[-2:]
            for (W, AW) in Vb:
                alpha = W.T @ r
                x = x + W @ alpha
                r = r - AW @ alpha
                if record:
                    res.xs.append(x.copy())
            rho = float(np.linalg.norm(r))
            res.hist.append(rho)
            k += 1
    except Breakdown:
        res.status = BREAKDOWN
    res.spmm_count = ctx.spmm
    return _finish(res, x, rho, rho0, tol, k)


# ----------------------------------------------------------------------------------------
# Dispatcher
# ----------------------------------------------------------------------------------------

def solve(A, b, part, t, s, tol=1e-8, maxit=1000, x0=None, variant="sre", basis="sstep",
          orth="acholqr", breakdown_tol=1e-14, explicit_AW=False, record=False,
          carried_cgs=False, precond=None, deflate=False) -> Result:
    """Select the algorithm: basis 'sstep' -> Alg. 4 (sre) / Alg. 3 (sre2) / Alg. 6 (msdo);
    basis 'ca5' / 'ca7' -> the CA form of the variant with Alg. 5 / Alg. 7.  `precond`
    (e.g. BlockJacobi) gives the split preconditioned forms of Section 5 (Algorithms 8-10).
    deflate=True drops the columns whose A-CholQR pivots fail the breakdown rule.
    basis 'restructured' -> Alg. 2 (sre) / Alg. 1 (sre2)."""
    if basis == "restructured":
        if variant == "msdo" or precond is not None:
            raise ValueError("the restructured forms are Algorithms 1 and 2 (SRE-CG, SRE-CG2)")
        return restructured_sre_cg(A, b, part, t, s, tol, maxit, x0, orth, variant == "sre2",
                                   breakdown_tol, record, carried_cgs, deflate)
    if basis == "sstep":
        if variant == "msdo":
            return sstep_msdo_cg(A, b, part, t, s, tol, maxit, x0, orth, breakdown_tol,
                                 explicit_AW, record, carried_cgs, precond, deflate)
        return sstep_sre_cg(A, b, part, t, s, tol, maxit, x0, orth, variant == "sre2",
                            breakdown_tol, explicit_AW, record, carried_cgs, precond, deflate)
    return ca_enlarged_cg(A, b, part, t, s, tol, maxit, x0, orth, variant,
                          "alg5" if basis == "ca5" else "alg7", breakdown_tol, explicit_AW,
                          record, carried_cgs, precond, deflate)


# ----------------------------------------------------------------------------------------
# Split preconditioning (Section 5): block Jacobi M = L L^T, preconditioned CG
# ----------------------------------------------------------------------------------------

def ic0(Ad: np.ndarray) -> np.ndarray:
    """Incomplete Cholesky factor with zero fill-in of a dense SPD block: the lower
    triangular L with the sparsity pattern of tril(Ad), computed by the right-looking
    Cholesky elimination in which every update that falls outside the pattern is dropped
    (so (L L^T)_ij = Ad_ij on the pattern)."""
    n = Ad.shape[0]
    S = Ad != 0
    a = np.tril(np.asarray(Ad, dtype=np.float64)).copy()
    for k in range(n):
        if not (a[k, k] > 0):
            raise Breakdown(f"ic0 pivot {k}")
        a[k, k] = math.sqrt(a[k, k])
        rows = k + 1 + np.nonzero(S[k + 1:, k])[0]
        a[rows, k] /= a[k, k]
        for j in rows:
            ii = rows[rows >= j]
            ii = ii[S[ii, j]]
            a[ii, j] -= a[ii, k] * a[j, k]
    return a


class BlockJacobi:
    """Block Jacobi preconditioner M = L L^T of the preconditioned experiments of Section
    5: L is block diagonal over the domains of `bpart` (each row in one block), and L_i is
    the lower factor of the diagonal block A(D_i, D_i), either its complete Cholesky factor
    (factor='cholesky') or its incomplete Cholesky factor with zero fill-in (factor='ic0').
    solve_L / solve_LT / apply act on vectors or n x m blocks."""

    def __init__(self, A, bpart, factor="cholesky"):
        As = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
        bpart = np.asarray(bpart)
        self.n = As.shape[0]
        self.blocks = []
        for d in np.unique(bpart):
            idx = np.nonzero(bpart == d)[0]
            Ad = As[idx][:, idx].toarray()
            if factor == "cholesky":
                L = sla.cholesky(Ad, lower=True)
            elif factor == "ic0":
                L = ic0(Ad)
            else:
                raise ValueError(factor)
            self.blocks.append((idx, L))

    def solve_L(self, X):
        Y = np.array(X, dtype=np.float64, copy=True)
        for idx, L in self.blocks:
            Y[idx] = sla.solve_triangular(L, Y[idx], lower=True)
        return Y

    def solve_LT(self, X):
        Y = np.array(X, dtype=np.float64, copy=True)
        for idx, L in self.blocks:
            Y[idx] = sla.solve_triangular(L, Y[idx], lower=True, trans="T")
        return Y

    def apply(self, X):
        """M^{-1} X = L^{-T} L^{-1} X."""
        return self.solve_LT(self.solve_L(X))

    def L_dense(self):
        """The block diagonal factor L as a dense matrix (small test problems)."""
        L = np.zeros((self.n, self.n))
        for idx, Li in self.blocks:
            L[np.ix_(idx, idx)] = Li
        return L


def pcg(A, b, precond, x0=None, tol=1e-8, maxit=10000, record=False) -> Result:
    """Preconditioned CG as stated at the end of Section 6: p_1 = M^{-1} r_0,
    p_k = M^{-1} r_{k-1} + beta p_{k-1}, beta = rhat_{k-1} / rhat_{k-2} with
    rhat_k = r_k^T M^{-1} r_k, alpha = rhat_{k-1} / p^T A p, x_k = x_{k-1} + alpha p,
    r_k = r_{k-1} - alpha A p; stopping rule on ||r_k||_2 as for CG."""
    Asp = A.to_scipy() if hasattr(A, "to_scipy") else sp.csr_matrix(A)
    x, r, rho0 = _start(A, b, x0)
    res = Result(x=x, iters=0, hist=[rho0], status=OK)
    if record:
        res.xs.append(x.copy())
    z = precond.apply(r)
    rz = float(r @ z)
    rho, k = rho0, 1
    p = None
    rz_prev = None
    kmax = maxit + 1
    while rho > tol * rho0 and k < kmax:
        p = z.copy() if k == 1 else z + (rz / rz_prev) * p
        w = Asp @ p
        alpha = rz / float(p @ w)
        x = x + alpha * p
        r = r - alpha * w
        z = precond.apply(r)
        rz_prev, rz = rz, float(r @ z)
        rho = float(np.linalg.norm(r))
        res.hist.append(rho)
        if record:
            res.xs.append(x.copy())
        k += 1
    return _finish(res, x, rho, rho0, tol, k)


# ----------------------------------------------------------------------------------------
# Adjoint gradients of a solve (differentiable configuration; not in the paper)
# ----------------------------------------------------------------------------------------

def grad_A_values(A, lam, x):
    """dL/dA_ij = -lambda_i x_j for every stored nonzero (i, j) of A (CSR order), where
    x = A^{-1} b and lambda = A^{-1} dL/dx (A symmetric)."""
    out = np.empty(A.nnz)
    for i in range(A.n):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            out[k] = -lam[i] * x[A.colind[k]]
    return out


def diffusion2d_grad_logkappa(log_kappa, nx, ny, lam, x, ax=1.0, ay=1.0):
    """dL/dlog(kappa) for the 2D edge-form diffusion matrix
    A = sum_e w_e (e_p - e_q)(e_p - e_q)^T + sum_faces a kappa_p e_p e_p^T,
    w_e = a * 2 k_p k_q / (k_p + k_q): loop over edges and Dirichlet faces,
    dL/dw = -lambda^T (dA/dw) x, chained through dw/dk and dk/dlog k = k."""
    k = np.exp(np.asarray(log_kappa, dtype=np.float64).reshape(ny, nx))
    g = np.zeros((ny, nx))
    lam = np.asarray(lam).reshape(ny, nx)
    x = np.asarray(x).reshape(ny, nx)
    for j in range(ny):
        for i in range(nx):
            for (di, dj, a) in ((1, 0, ax), (0, 1, ay)):
                i2, j2 = i + di, j + dj
                if i2 < nx and j2 < ny:
                    kp, kq = k[j, i], k[j2, i2]
                    dLdw = -(lam[j, i] - lam[j2, i2]) * (x[j, i] - x[j2, i2])
                    g[j, i] += dLdw * a * 2.0 * kq * kq / (kp + kq) ** 2
                    g[j2, i2] += dLdw * a * 2.0 * kp * kp / (kp + kq) ** 2
            # Dirichlet faces: two per axis at the ends of the grid
            faces = (i == 0) + (i == nx - 1)
            g[j, i] += faces * ax * (-lam[j, i] * x[j, i])
            faces = (j == 0) + (j == ny - 1)
            g[j, i] += faces * ay * (-lam[j, i] * x[j, i])
    return (g * k).ravel()
