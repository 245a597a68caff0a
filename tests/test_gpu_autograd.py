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
    solve A lambda = x - x* and dL/dlog kappa, against the oracle's records
    (tests/golden/oracle_counts.json, written by the oracle only).

    This workload is sensitive to rounding: with b multiplied by (1 + 1e-15 xi) the oracle's
    own residual norms move by about 2e-6 at the third s-step iteration and by tens of
    percent from the fourth ("perturbed_hist" records), and its iteration counts spread
    ("perturbed" records).  So the bars are:
    * iteration counts within the oracle's perturbation spread, widened by one;
    * residual norm k within max(1e-6, twice the oracle's perturbation spread at k), up to
      the first iteration that the perturbation moves by more than 1e-3;
    * the true relative residual <= 1.01e-8 (the solutions themselves are what is unique);
    * x, x* and lambda at 256 sampled rows within the bound that any two solutions with
      those residuals obey, |u - v| <= ||u - v||_2 <= (||r_u|| + ||r_v||) / lambda_min(A)
      (lambda_min by shift-invert Lanczos), the adjoint's right-hand side difference
      included;
    * the gradient kernel at full size: the GPU's dL/dlog kappa equals the oracle's
      formula applied to the GPU's own x and lambda (sampled rows, 1e-12 of the max-norm);
    * the loss within the bound implied by the bounds on x - x*."""
    import json
    from scipy.sparse.linalg import eigsh
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
    rows = np.array(gold[key + "/grad_logkappa"]["rows"])

    def lam_min(Amat):
        return float(eigsh(Amat.to_scipy().tocsc(), k=1, sigma=0, which="LM",
                           return_eigenvectors=False)[0])

    def spread(which):
        pre = f"{key}/{which}/perturbed/"
        return [gold[f"{key}/{which}"]["iters"]] + [v["iters"] for k, v in gold.items()
                                                    if k.startswith(pre)]

    def hist_tol(which):
        """The oracle's norms, the tolerance (twice its perturbation spread, at least
        1e-6), and how many of them to compare: those before the first one that the
        perturbation moves by more than 1e-3 (past it the history is chaotic and a few
        seeds do not bound it)."""
        base = np.array(gold[f"{key}/{which}"]["hist"][:21])
        pre = f"{key}/{which}/perturbed_hist/"
        pert = [np.array(v["hist"][:21]) for k, v in gold.items() if k.startswith(pre)]
        assert len(pert) >= 2, which
        dev = np.max([np.abs(h - base) / base for h in pert], axis=0)
        chaotic = np.nonzero(dev > 1e-3)[0]
        return base, np.maximum(1e-6, 2.0 * dev), int(chaotic[0]) if len(chaotic) else 21

    def solve(log_k, rhs, which, Amat, rhs_np):
        rec = gold[f"{key}/{which}"]
        ekcg.ekcg_diffusion2d_values(S.ctx, N, N, 1.0, 1.0,
                                     torch.as_tensor(log_k.ravel(), device="cuda"), val)
        ekcg.ekcg_update_values(S.ctx, val)
        x, it, hist, st = S.solve(rhs, s=s, tol=1e-8, maxit=5000)
        counts = spread(which)
        assert st == 0 and min(counts) - 1 <= it <= max(counts) + 1, (it, counts)
        xh = x.cpu().numpy()
        res = float(np.linalg.norm(rhs_np - Amat.to_scipy() @ xh))
        assert res <= 1.01e-8 * np.linalg.norm(rhs_np)
        return x, xh, np.array(hist), res

    # target and forward: histories against the oracle's perturbation spread
    lmin_star, lmin = lam_min(A_star), lam_min(A)
    xs, xsh, hs, res_s = solve(lk_star, one, "target", A_star, np.ones(N * N))
    x, xh, hx, res_x = solve(lk, one, "forward", A, np.ones(N * N))
    for which, h in (("target", hs), ("forward", hx)):
        base, tol, kc = hist_tol(which)
        assert kc >= 3, (which, kc)
        m = min(len(h), len(base), kc)
        assert np.all(np.abs(h[:m] - base[:m]) <= tol[:m] * base[:m]), (which, h[:m], base[:m])
    nb = float(np.sqrt(N * N))
    bound_s = (res_s + gold[key + "/target"]["relres"] * nb) / lmin_star
    bound_x = (res_x + gold[key + "/forward"]["relres"] * nb) / lmin
    assert np.max(np.abs(xsh[rows] - np.array(gold[key + "/target"]["x"]["values"]))) <= bound_s
    assert np.max(np.abs(xh[rows] - np.array(gold[key + "/forward"]["x"]["values"]))) <= bound_x
    # adjoint: its right-hand side is the GPU's x - x*, within bound_x + bound_s of the
    # oracle's (whose norm is sqrt(2 loss))
    g = x - xs
    gh = g.cpu().numpy()
    dg = bound_x + bound_s
    loss_o = gold[key + "/grad_logkappa"]["loss"]
    ng_o = np.sqrt(2.0 * loss_o)
    lam, lamh, hl, res_l = solve(lk, g.contiguous(), "adjoint", A, gh)
    assert abs(hl[0] - gold[key + "/adjoint"]["hist"][0]) <= dg + 1e-6 * hl[0]
    bound_l = (res_l + gold[key + "/adjoint"]["relres"] * ng_o + dg) / lmin
    assert np.max(np.abs(lamh[rows] - np.array(gold[key + "/adjoint"]["x"]["values"]))) <= bound_l
    # the gradient kernel at full size, on the GPU's own lambda and x
    glk = torch.empty(N * N, dtype=torch.float64, device="cuda")
    ekcg.ekcg_diffusion2d_grad_logkappa(S.ctx, N, N, 1.0, 1.0,
                                        torch.as_tensor(lk.ravel(), device="cuda"), lam, x, glk)
    ref = o.diffusion2d_grad_logkappa(lk.ravel(), N, N, lamh, xh)
    got = glk.cpu().numpy()
    assert np.max(np.abs(got[rows] - ref[rows])) <= 1e-12 * np.max(np.abs(ref))
    # the loss 0.5 ||g||^2 against the oracle's
    ng = float(np.linalg.norm(gh))
    assert abs(0.5 * ng * ng - loss_o) <= (ng + 0.5 * dg) * dg + 1e-12 * loss_o
    S.close()
