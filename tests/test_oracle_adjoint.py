"""Pins of the oracle's adjoint gradients: central finite differences of a dense float64
solve, and the closed form dL/db = lambda for the loss 0.5 ||x - x*||^2."""
import numpy as np
import scipy.linalg as sla

import workloads as wl
from oracle import ekcg_ref as o


def dense_solve(A, b):
    return sla.cho_solve(sla.cho_factor(A.to_scipy().toarray()), b)


def test_grad_values_and_b_by_finite_differences():
    N = 6
    A = wl.stencil_matrix((N, N), kappa=np.exp(wl.kappa_gaussian_field2d(N, 1, 2.0)))
    b = wl.rhs_uniform(A.n, 2)
    xt = wl.rhs_uniform(A.n, 3)

    def loss(val, bb):
        # a single perturbed entry makes A non-symmetric: general dense LU solve
        M = wl.CSR(A.n, A.rowptr, A.colind, val).to_scipy().toarray()
        return 0.5 * np.sum((np.linalg.solve(M, bb) - xt) ** 2)

    x = dense_solve(A, b)
    lam = dense_solve(A, x - xt)
    gv = o.grad_A_values(A, lam, x)
    h = 1e-6
    for k in [0, 3, 17, 40, A.nnz - 1]:
        e = np.zeros(A.nnz)
        e[k] = h
        fd = (loss(A.val + e, b) - loss(A.val - e, b)) / (2 * h)
        assert abs(gv[k] - fd) <= 1e-6 * max(1.0, abs(fd))
    for i in [0, 7, 35]:
        e = np.zeros(A.n)
        e[i] = h
        fd = (loss(A.val, b + e) - loss(A.val, b - e)) / (2 * h)
        assert abs(lam[i] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_grad_logkappa_by_finite_differences():
    nx, ny = 7, 5
    lk = np.random.default_rng(0).standard_normal(nx * ny)
    b = np.ones(nx * ny)
    xt = wl.rhs_uniform(nx * ny, 4)

    def loss(l):
        A = wl.stencil_matrix((nx, ny), kappa=np.exp(l).reshape(ny, nx), aniso=(1.0, 0.3))
        return 0.5 * np.sum((dense_solve(A, b) - xt) ** 2)

    A = wl.stencil_matrix((nx, ny), kappa=np.exp(lk).reshape(ny, nx), aniso=(1.0, 0.3))
    x = dense_solve(A, b)
    lam = dense_solve(A, x - xt)
    g = o.diffusion2d_grad_logkappa(lk, nx, ny, lam, x, 1.0, 0.3)
    h = 1e-6
    for p in range(nx * ny):
        e = np.zeros(nx * ny)
        e[p] = h
        fd = (loss(lk + e) - loss(lk - e)) / (2 * h)
        assert abs(g[p] - fd) <= 1e-7 * max(1.0, abs(fd)), (p, g[p], fd)
