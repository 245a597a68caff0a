"""Adjoint gradients of the enlarged solve (torch.autograd) against float64 dense
references: the analytic gradient from a dense Cholesky solve, and central finite
differences of the dense loss, on small grids."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import ekcg_ref as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_10629_gb300 import autograd as ag  # noqa: E402
from paper_1804_10629_gb300 import ekcg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()


def dense_solve(A, b):
    return sla.cho_solve(sla.cho_factor(A.to_scipy().toarray()), b)


def test_diffusion2d_values_match_generator():
    N = 12
    lk = wl.kappa_gaussian_field2d(N, seed=4, corr=3.0)
    A = wl.stencil_matrix((N, N), kappa=np.exp(lk))
    S = ekcg.Solver(A, 4, wl.partition_boxes((N, N), 4), max_s=3)
    val = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    ekcg.ekcg_diffusion2d_values(S.ctx, N, N, 1.0, 1.0,
                                 torch.as_tensor(lk, device="cuda"), val)
    np.testing.assert_allclose(val.cpu().numpy(), A.val, rtol=1e-14, atol=0)
    S.close()


def test_grad_b_and_values_match_dense_adjoint():
    N = 10
    A = wl.stencil_matrix((N, N), kappa=np.exp(wl.kappa_gaussian_field2d(N, 5, 3.0)))
    part = wl.partition_boxes((N, N), 4)
    b = wl.rhs_uniform(A.n, 6)
    xt = wl.rhs_uniform(A.n, 7)
    S = ekcg.Solver(A, 4, part, max_s=3)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    vt = torch.tensor(A.val, device="cuda", requires_grad=True)
    x = ag.enlarged_solve(bt, vt, S, s=3, tol=1e-12)
    loss = 0.5 * ((x - torch.as_tensor(xt, device="cuda")) ** 2).sum()
    loss.backward()
    # dense float64 reference: x = A^{-1} b, lambda = A^{-1}(x - xt), dL/dA_ij = -lambda_i x_j
    xd = dense_solve(A, b)
    lam = dense_solve(A, xd - xt)
    dval = o.grad_A_values(A, lam, xd)
    np.testing.assert_allclose(bt.grad.cpu().numpy(), lam, rtol=0, atol=1e-8 * np.abs(lam).max())
    np.testing.assert_allclose(vt.grad.cpu().numpy(), dval, rtol=0,
                               atol=1e-8 * np.abs(dval).max())
    S.close()


def test_grad_logkappa_matches_finite_differences():
    N = 8
    lk0 = wl.kappa_gaussian_field2d(N, 4, 2.0)
    b = np.ones(N * N)
    target = dense_solve(wl.stencil_matrix((N, N), kappa=np.exp(
        wl.kappa_gaussian_field2d(N, 5, 2.0))), b)

    def loss_dense(lk):
        x = dense_solve(wl.stencil_matrix((N, N), kappa=np.exp(lk)), b)
        return 0.5 * np.sum((x - target) ** 2)

    A = wl.stencil_matrix((N, N), kappa=np.exp(lk0))
    S = ekcg.Solver(A, 4, wl.partition_boxes((N, N), 4), max_s=3)
    lkt = torch.tensor(lk0.ravel(), device="cuda", requires_grad=True)
    x = ag.diffusion2d_solve(lkt, torch.as_tensor(b, device="cuda"), S, N, N, s=3, tol=1e-13)
    loss = 0.5 * ((x - torch.as_tensor(target, device="cuda")) ** 2).sum()
    loss.backward()
    g = lkt.grad.cpu().numpy()
    assert abs(loss.item() - loss_dense(lk0.ravel())) <= 1e-10 * max(1.0, loss.item())
    xd = dense_solve(A, b)
    g_or = o.diffusion2d_grad_logkappa(lk0.ravel(), N, N, dense_solve(A, xd - target), xd)
    np.testing.assert_allclose(g, g_or, rtol=0, atol=1e-8 * np.abs(g_or).max())
    h = 1e-5
    rng = np.random.default_rng(0)
    for p in rng.choice(N * N, 12, replace=False):
        e = np.zeros(N * N)
        e[p] = h
        fd = (loss_dense(lk0.ravel() + e) - loss_dense(lk0.ravel() - e)) / (2 * h)
        assert abs(g[p] - fd) <= 1e-6 * np.abs(g).max() + 1e-8 * abs(fd), (p, g[p], fd)
    S.close()


@pytest.mark.slow
def test_differentiable_workload_full_size_against_oracle_record():
    """The differentiable configuration at its full size (512^2, kappa = exp of a Gaussian
    random field with correlation length 16, t = 16, s = 3, tol 1e-8): the solve for the
    target x* (field seed 5, b = 1), the forward solve x (field seed 4, b = 1), the adjoint
    solve A lambda = x - x* and dL/dlog kappa, each against the oracle's whole-solve record
    (tests/golden/oracle_counts.json, written by the oracle only): iteration counts within
    the spread of oracle solves whose right-hand side was perturbed at the rounding level
    (the counts are chaotic in rounding at this size), widened by one; the first 21
    residual norms to 1e-6, the true relative residual, and x, lambda
    and the gradient at 256 sampled rows (float64 tolerances relative to the max-norm of
    the oracle's vector: 1e-8 for x*, x and lambda, 1e-7 for the gradient, a product of
    two solutions)."""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_counts.json")))
    key = "diff2d/N512/t16/s3/sre/sstep/fp64"
    N, t, s = 512, 16, 3
    lk = wl.kappa_gaussian_field2d(N, seed=4, corr=16.0)
    lk_star = wl.kappa_gaussian_field2d(N, seed=5, corr=16.0)
    A = wl.stencil_matrix((N, N), kappa=np.exp(lk))
    A_star = wl.stencil_matrix((N, N), kappa=np.exp(lk_star))
    part = wl.partition_boxes((N, N), t)
    S = ekcg.Solver(A, t, part, max_s=s)
    val = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    one = torch.ones(N * N, dtype=torch.float64, device="cuda")

    def spread(which):
        pre = f"{key}/{which}/perturbed/"
        return [gold[f"{key}/{which}"]["iters"]] + [v["iters"] for k, v in gold.items()
                                                    if k.startswith(pre)]

    def solve(log_k, rhs, which, Amat, rhs_np):
        rec = gold[f"{key}/{which}"]
        ekcg.ekcg_diffusion2d_values(S.ctx, N, N, 1.0, 1.0,
                                     torch.as_tensor(log_k.ravel(), device="cuda"), val)
        ekcg.ekcg_update_values(S.ctx, val)
        x, it, hist, st = S.solve(rhs, s=s, tol=1e-8, maxit=5000)
        counts = spread(which)
        assert st == 0 and min(counts) - 1 <= it <= max(counts) + 1, (it, counts)
        np.testing.assert_allclose(hist[:21], rec["hist"][:21], rtol=1e-6)
        xh = x.cpu().numpy()
        assert (np.linalg.norm(rhs_np - Amat.to_scipy() @ xh) <= 1.01e-8 *
                np.linalg.norm(rhs_np))
        ref = np.array(rec["x"]["values"])
        rows = np.array(gold[key + "/grad_logkappa"]["rows"])
        assert np.max(np.abs(xh[rows] - ref)) <= 1e-8 * rec["x"]["norminf"]
        return x, xh

    xs, xsh = solve(lk_star, one, "target", A_star, np.ones(N * N))
    x, xh = solve(lk, one, "forward", A, np.ones(N * N))
    g = x - xs
    lam, lamh = solve(lk, g.contiguous(), "adjoint", A, g.cpu().numpy())
    glk = torch.empty(N * N, dtype=torch.float64, device="cuda")
    ekcg.ekcg_diffusion2d_grad_logkappa(S.ctx, N, N, 1.0, 1.0,
                                        torch.as_tensor(lk.ravel(), device="cuda"), lam, x, glk)
    rec = gold[key + "/grad_logkappa"]
    rows = np.array(rec["rows"])
    got = glk.cpu().numpy()[rows]
    assert np.max(np.abs(got - np.array(rec["values"]))) <= 1e-7 * rec["norminf"]
    np.testing.assert_allclose(0.5 * float((g * g).sum()), rec["loss"], rtol=1e-7)
    S.close()
