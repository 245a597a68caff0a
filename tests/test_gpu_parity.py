"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (stated with the method's target): the partition permutation and T(r) are
bit-exact; the iteration count is within +-1 s-step iteration; per-iteration residual norms
agree to 1e-6 relative over the first 20 iterations; x agrees to 1e-8 relative; the true
relative residual ||b - A x|| / ||b|| is <= tol (1e-8), up to the 1% slack of the
recursive-vs-true residual gap.
"""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import ekcg_ref as o

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_10629_gb300 import ekcg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not os.path.exists(ekcg.LIB_PATH):
        from paper_1804_10629_gb300 import build
        build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def relres(A, b, x):
    return np.linalg.norm(b - A.to_scipy() @ x) / np.linalg.norm(b)


def check_parity(A, b, part, t, s, variant="sre", basis="sstep", orth="acholqr", tol=1e-8,
                 maxit=2000, x_tol=1e-8):
    ref = o.solve(A, b, part, t, s, tol=tol, maxit=maxit, variant=variant, basis=basis,
                  orth=orth)
    S = ekcg.Solver(A, t, part, variant=variant, basis=basis, orth=orth, max_s=max(s, 1),
                    max_basis_bytes=8 << 30)
    x, it, hist, st = S.solve(dev(b), s=s, tol=tol, maxit=maxit)
    x = x.cpu().numpy()
    S.close()
    assert st == ref.status, (st, ref.status)
    assert abs(it - ref.iters) <= 1, (it, ref.iters)
    m = min(21, len(hist), len(ref.hist))
    h_ref = np.array(ref.hist[:m])
    np.testing.assert_allclose(hist[:m], h_ref, rtol=1e-6, atol=0)
    if ref.status == o.OK:
        assert relres(A, b, x) <= tol * 1.01
        assert np.linalg.norm(x - ref.x) <= x_tol * np.linalg.norm(ref.x)
    return it, ref.iters


# ----------------------------------------------------------------------------------------
# Bit-exact integer / copy work
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["strips", "boxes3d", "random"])
def test_perm_and_split_T_bit_exact(kind):
    if kind == "strips":
        p = wl.poisson2d(100, 4)
        A, part, t = p.A, p.part, 4
    elif kind == "boxes3d":
        A = wl.stencil_matrix((32, 32, 32), aniso=(1, 1, 1e-3))
        t = 32
        part = wl.partition_boxes((32, 32, 32), t)
    else:
        A = wl.stencil_matrix((45, 37))
        t = 7
        part = np.random.default_rng(3).integers(0, t, A.n).astype(np.int32)
    S = ekcg.Solver(A, t, part, max_s=1)
    perm = S.perm()
    assert np.array_equal(perm, o.domain_perm(part))
    r = np.random.default_rng(1).standard_normal(A.n)
    rp = dev(r[perm])
    T = torch.empty(A.n * t, dtype=torch.float64, device="cuda")
    ekcg.ekcg_split_T(S.ctx, rp, T)
    ref = o.split_T(r, part, t)[perm]
    assert np.array_equal(T.cpu().numpy().reshape(A.n, t), ref)
    # permute both ways
    y = torch.empty_like(rp)
    ekcg.ekcg_permute(S.ctx, dev(r), y, 0)
    assert np.array_equal(y.cpu().numpy(), r[perm])
    z = torch.empty_like(rp)
    ekcg.ekcg_permute(S.ctx, y, z, 1)
    assert np.array_equal(z.cpu().numpy(), r)
    S.close()


@pytest.mark.parametrize("w", [1, 3, 4, 16, 32])
def test_spmm_matches_scipy(w):
    A = wl.stencil_matrix((23, 19, 11), kappa=wl.kappa_skyscraper3d(23)[:11, :19, :23])
    part = wl.partition_boxes((23, 19, 11), 8)
    S = ekcg.Solver(A, 8, part, max_s=1)
    perm = S.perm()
    Ap = A.to_scipy()[perm][:, perm]
    W = np.random.default_rng(w).standard_normal((A.n, w))
    U = torch.empty(A.n * w, dtype=torch.float64, device="cuda")
    ekcg.ekcg_spmm(S.ctx, dev(W), U, w)
    ref = Ap @ W
    got = U.cpu().numpy().reshape(A.n, w)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    S.close()


@pytest.mark.parametrize("p,q", [(64, 32), (32, 32), (16, 16), (48, 8), (64, 1), (48, 1), (256, 1),
                                 (256, 16)])
def test_gram_entry_matches_numpy(p, q):
    """C = X^T Y over n = 1665 rows (ragged against the 32-row stages), tolerance
    n * eps * |X|^T |Y| (the float64 dot-product error bound)."""
    A = wl.stencil_matrix((45, 37))
    S = ekcg.Solver(A, 16, wl.partition_boxes((45, 37), 16), max_s=4)
    rng = np.random.default_rng(p * 1000 + q)
    X = rng.standard_normal((A.n, p))
    Y = rng.standard_normal((A.n, q))
    C = torch.empty(p * q, dtype=torch.float64, device="cuda")
    ekcg.ekcg_gram(S.ctx, dev(X), p, dev(Y), q, C)
    bound = A.n * 2.2e-16 * (np.abs(X).T @ np.abs(Y))
    assert np.all(np.abs(C.cpu().numpy().reshape(p, q) - X.T @ Y) <= bound)
    S.close()


# ----------------------------------------------------------------------------------------
# Solver parity (ragged sizes: n = 45*37 = 1665 rows is not a multiple of any tile)
# ----------------------------------------------------------------------------------------

def ragged_problem(t=4):
    A = wl.stencil_matrix((45, 37))
    return A, wl.rhs_uniform(A.n, 11), wl.partition_boxes((45, 37), t)


@pytest.mark.parametrize("variant,basis", [("sre", "sstep"), ("sre2", "sstep"),
                                           ("msdo", "sstep"), ("sre", "ca7"),
                                           ("sre2", "ca7"), ("msdo", "ca7"),
                                           ("sre", "ca5"), ("sre2", "ca5"),
                                           ("msdo", "ca5")])
@pytest.mark.parametrize("s", [1, 2, 3])
def test_solver_parity_ragged(variant, basis, s):
    A, b, part = ragged_problem()
    check_parity(A, b, part, 4, s, variant, basis)


@pytest.mark.parametrize("variant", ["sre", "sre2"])
@pytest.mark.parametrize("s", [1, 2, 3])
def test_restructured_parity(variant, s):
    """Restructured SRE-CG / SRE-CG2 (Algorithms 2 / 1): the s-step basis, then s sequential
    block updates per outer iteration, against the oracle's restructured form."""
    A, b, part = ragged_problem()
    check_parity(A, b, part, 4, s, variant, "restructured")


def test_restructured_msdo_is_rejected():
    A, b, part = ragged_problem()
    with pytest.raises(Exception):
        ekcg.Solver(A, 4, part, variant="msdo", basis="restructured", max_s=2)


@pytest.mark.parametrize("variant", ["sre", "sre2", "msdo"])
@pytest.mark.parametrize("s", [1, 2])
@pytest.mark.parametrize("basis", ["sstep", "ca5", "ca7"])
def test_block_jacobi_parity(variant, s, basis):
    """Split preconditioned s-step and CA forms (Section 5, Algorithms 8-10; in the CA
    forms every power M^{-1} A W) with block Jacobi IC(0) over 16 boxes inside the 4
    domains, against the oracle (its own IC(0) and triangular solves)."""
    A, b, part = ragged_problem()
    bpart = wl.partition_boxes((45, 37), 16)
    M = o.BlockJacobi(A, bpart, "ic0")
    ref = o.solve(A, b, part, 4, s, tol=1e-8, maxit=2000, variant=variant, basis=basis,
                  precond=M)
    S = ekcg.Solver(A, 4, part, variant=variant, basis=basis, max_s=s,
                    max_basis_bytes=8 << 30)
    S.set_block_jacobi(bpart)
    x, it, hist, st = S.solve(dev(b), s=s, tol=1e-8, maxit=2000)
    x = x.cpu().numpy()
    S.close()
    assert st == ref.status == o.OK, (st, ref.status)
    assert abs(it - ref.iters) <= 1, (it, ref.iters)
    m = min(21, len(hist), len(ref.hist))
    np.testing.assert_allclose(hist[:m], np.array(ref.hist[:m]), rtol=1e-6, atol=0)
    assert relres(A, b, x) <= 1e-8 * 1.01
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_block_jacobi_rejections():
    A, b, part = ragged_problem()
    S = ekcg.Solver(A, 4, part, max_s=2)
    with pytest.raises(ekcg.EkcgError):        # blocks across the 4 domains
        S.set_block_jacobi(wl.partition_strips(A.n, 3))
    S.set_block_jacobi(wl.partition_boxes((45, 37), 16))
    S.set_block_jacobi(None)                   # removed: the plain solve again
    x, it, hist, st = S.solve(dev(b), s=2, tol=1e-8, maxit=2000)
    ref = o.solve(A, b, part, 4, 2, tol=1e-8, maxit=2000)
    assert st == 0 and abs(it - ref.iters) <= 1
    S.close()
    F = ekcg.Solver(A, 4, part, precision="fp32_ir", max_s=2)
    with pytest.raises(ekcg.EkcgError):
        F.set_block_jacobi(wl.partition_boxes((45, 37), 16))
    F.close()
    R = ekcg.Solver(A, 4, part, basis="restructured", max_s=2)
    with pytest.raises(ekcg.EkcgError):
        R.set_block_jacobi(wl.partition_boxes((45, 37), 16))
    R.close()


@pytest.mark.parametrize("variant", ["sre", "sre2", "msdo"])
def test_precholqr_parity(variant):
    A, b, part = ragged_problem(t=8)
    check_parity(A, b, part, 8, 2, variant, "sstep", "precholqr")


def test_poisson2d_config_parity():
    """Poisson2D 100x100, 4 strips, s = 2, tol 1e-8, plain FP64."""
    p = wl.poisson2d(100, 4, seed=0)
    check_parity(p.A, p.b, p.part, 4, 2)


def test_t1_is_cg():
    A = wl.stencil_matrix((40, 40))
    b = wl.rhs_uniform(A.n, 2)
    part = np.zeros(A.n, np.int32)
    ref = o.cg(A, b, tol=1e-8, maxit=2000)
    S = ekcg.Solver(A, 1, part, max_s=1)
    x, it, hist, st = S.solve(dev(b), s=1, tol=1e-8, maxit=2000)
    assert st == 0 and abs(it - ref.iters) <= 1
    np.testing.assert_allclose(hist[:21], ref.hist[:21], rtol=1e-6)
    S.close()


@pytest.mark.parametrize("s", [1, 2, 4])
def test_ani3d_small_parity(s):
    """Ani3D-like operator (7-point, coefficients 1, 1, 1e-3) on 24^3 with t = 32 boxes."""
    A = wl.stencil_matrix((24, 24, 24), aniso=(1.0, 1.0, 1e-3))
    part = wl.partition_boxes((24, 24, 24), 32)
    b = wl.rhs_uniform(A.n, 1)
    check_parity(A, b, part, 32, s)


@pytest.mark.parametrize("variant", ["sre", "sre2", "msdo"])
def test_ca7_s8_t32_gram_256(variant):
    """CA forms with the modified CA-Arnoldi (Algorithm 7) at s = 8, t = 32: every
    iteration A-orthonormalises an n x 256 block V = [W, A W, ..., A^7 W], so the A-CholQR
    Gram is 256 x 256 (the largest the library takes).  At s = 8 the power basis is
    numerically rank deficient (Section 4: the CA forms lose stability as s grows); on the
    Ani3D-like operator on 10^3 boxes the oracle's max|Q^T A Q - I| grows from 1e-5 to
    3e-2 within three iterations and the Cholesky pivot test stops the solve.  The GPU must
    stop the same way at the same iteration (within one), agree on the residual norms while
    the basis is still A-orthonormal (iterations 1 and 2) and return the same last complete
    iterate.  Tolerance 1e-4: the oracle's own basis is A-orthonormal only to 1e-5 - 7e-5 in
    these iterations, and rounding differences in V^T A V enter the residual norms scaled
    by that loss (two float64 implementations agree to a few 1e-6 here)."""
    A = wl.stencil_matrix((10, 10, 10), aniso=(1.0, 1.0, 1e-3))
    part = wl.partition_boxes((10, 10, 10), 32)
    b = wl.rhs_uniform(A.n, 1)
    ref = o.solve(A, b, part, 32, 8, tol=1e-8, maxit=100, variant=variant, basis="ca7")
    assert ref.status == o.BREAKDOWN
    S = ekcg.Solver(A, 32, part, variant=variant, basis="ca7", max_s=8,
                    max_basis_bytes=1 << 30)
    x, it, hist, st = S.solve(dev(b), s=8, tol=1e-8, maxit=100)
    S.close()
    assert st == ekcg.EKCG_EBREAKDOWN
    assert abs(it - ref.iters) <= 1, (it, ref.iters)
    np.testing.assert_allclose(hist[:3], ref.hist[:3], rtol=1e-4)
    if it == ref.iters:
        x = x.cpu().numpy()
        assert np.linalg.norm(x - ref.x) <= 1e-4 * np.linalg.norm(ref.x)


def test_sky3d_small_parity():
    A = wl.stencil_matrix((16, 16, 16), kappa=wl.kappa_skyscraper3d(16))
    part = wl.partition_boxes((16, 16, 16), 16)
    b = wl.rhs_uniform(A.n, 2)
    check_parity(A, b, part, 16, 4, "sre2")


# ----------------------------------------------------------------------------------------
# Edge cases and status codes
# ----------------------------------------------------------------------------------------

def test_edge_cases():
    A, b, part = ragged_problem()
    S = ekcg.Solver(A, 4, part, max_s=4)
    # b = 0: rho_0 = 0, nothing to do
    x, it, hist, st = S.solve(dev(np.zeros(A.n)), s=2)
    assert st == 0 and it == 0 and float(x.abs().max()) == 0.0 and hist[0] == 0.0
    # maxit = 0
    x, it, hist, st = S.solve(dev(b), s=2, maxit=0)
    assert st == ekcg.EKCG_MAXIT and it == 0
    # maxit reached
    x, it, hist, st = S.solve(dev(b), s=2, maxit=3)
    assert st == ekcg.EKCG_MAXIT and it == 3 and len(hist) == 4
    ref = o.solve(A, b, part, 4, 2, maxit=3)
    np.testing.assert_allclose(x.cpu().numpy(), ref.x, rtol=0, atol=1e-10 * np.linalg.norm(ref.x))
    # warm start: the tolerance is relative to ||r_0|| of that solve (Algorithm 4 line 1)
    x1, it1, _, st1 = S.solve(dev(b), s=2, tol=1e-6)
    x2, it2, h2, st2 = S.solve(dev(b), x0=x1, s=2, tol=1e-2)
    ref = o.solve(A, b, part, 4, 2, tol=1e-2, x0=x1.cpu().numpy())
    assert st1 == 0 and st2 == 0 and abs(it2 - ref.iters) <= 1
    np.testing.assert_allclose(h2[0], ref.hist[0], rtol=1e-6)
    # NaN right-hand side
    bn = b.copy()
    bn[5] = np.nan
    with pytest.raises(ekcg.EkcgError) as e:
        S.solve(dev(bn), s=2)
    assert e.value.status == ekcg.EKCG_EINVAL
    # s beyond max_s
    with pytest.raises(ekcg.EkcgError):
        S.solve(dev(b), s=5)
    # breakdown: r_0 vanishes on one domain -> T(r_0) has a zero column
    bz = b.copy()
    bz[part == 2] = 0.0
    x, it, hist, st = S.solve(dev(bz), s=2)
    ref = o.solve(A, bz, part, 4, 2)
    assert st == ekcg.EKCG_EBREAKDOWN == ref.status and it == 0 == ref.iters
    S.close()


def test_setup_rejects_bad_input():
    A, b, part = ragged_problem()
    bad = part.copy()
    bad[0] = 9
    with pytest.raises(ekcg.EkcgError):
        ekcg.Solver(A, 4, bad)
    empty = part.copy()
    empty[empty == 3] = 2
    with pytest.raises(ekcg.EkcgError):
        ekcg.Solver(A, 4, empty)
    with pytest.raises(ekcg.EkcgError):
        ekcg.Solver(A, 64, wl.partition_boxes((45, 37), 64), max_s=8)   # s*t > 256
    col = A.colind.copy()
    col[1] = col[2]          # unsorted / duplicate column
    A2 = wl.CSR(A.n, A.rowptr, col, A.val)
    with pytest.raises(ekcg.EkcgError):
        ekcg.Solver(A2, 4, part)


def test_host_solve_matches_device_solve_and_is_deterministic():
    A, b, part = ragged_problem()
    S = ekcg.Solver(A, 4, part, max_s=2)
    xd, itd, hd, _ = S.solve(dev(b), s=2)
    xd2, _, hd2, _ = S.solve(dev(b), s=2)
    xh, ith, hh, _ = S.solve_host(b, s=2)
    assert itd == ith
    assert np.array_equal(xd.cpu().numpy(), xh) and np.array_equal(hd, hh)
    assert np.array_equal(xd.cpu().numpy(), xd2.cpu().numpy()) and np.array_equal(hd, hd2)
    S.close()


# ----------------------------------------------------------------------------------------
# Mixed precision: float32 inner solves inside float64 iterative refinement
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["sre", "sre2"])
def test_fp32_ir_reaches_fp64_accuracy(variant):
    A = wl.stencil_matrix((16, 16, 16), kappa=wl.kappa_skyscraper3d(16))
    part = wl.partition_boxes((16, 16, 16), 16)
    b = wl.rhs_uniform(A.n, 2)
    ref = o.solve(A, b, part, 16, 4, tol=1e-8, maxit=1000, variant=variant)
    S = ekcg.Solver(A, 16, part, variant=variant, precision="fp32_ir", max_s=4,
                    max_basis_bytes=4 << 30)
    x, it, hist, st = S.solve(dev(b), s=4, tol=1e-8, maxit=5000)
    x = x.cpu().numpy()
    assert st == 0
    assert relres(A, b, x) <= 1e-8 * 1.01
    # both satisfy relres <= 1e-8: ||x - x_ref|| <= kappa * 2e-8 ||x||, kappa <= 1e5 here
    assert np.linalg.norm(x - ref.x) <= 2e-3 * np.linalg.norm(ref.x)
    S.close()


@pytest.mark.parametrize("orth", ["acholqr", "precholqr"])
def test_fp32_ir_upper_gram_orthonormalisations(orth):
    """The float32 path forms the A-CholQR Gram W^T (A W) and the Pre-CholQR Gram W^T W
    upper-triangle only (float-float accumulation) for block widths 16 and 32: both
    orthonormalisations reach the float64 tolerance on a t = 16 Sky3D-like case."""
    A = wl.stencil_matrix((16, 16, 16), kappa=wl.kappa_skyscraper3d(16))
    part = wl.partition_boxes((16, 16, 16), 16)
    b = wl.rhs_uniform(A.n, 3)
    S = ekcg.Solver(A, 16, part, orth=orth, precision="fp32_ir", max_s=2)
    x, it, hist, st = S.solve(dev(b), s=2, tol=1e-8, maxit=5000)
    assert st == 0
    assert relres(A, b, x.cpu().numpy()) <= 1e-8 * 1.01
    S.close()


@pytest.mark.parametrize("s", [1, 2])
def test_fp32_ir_ani3d_t32(s):
    """t = 32 exercises the float32 register-row update (P = 64 window, P = 32 triangular)
    and the warp-tile float32 Gram (64 x 32 coefficients, 32 x 32 float-float Gram)."""
    A = wl.stencil_matrix((24, 24, 24), aniso=(1.0, 1.0, 1e-3))
    part = wl.partition_boxes((24, 24, 24), 32)
    b = wl.rhs_uniform(A.n, 1)
    ref = o.solve(A, b, part, 32, s, tol=1e-8, maxit=1000)
    S = ekcg.Solver(A, 32, part, precision="fp32_ir", max_s=s)
    x, it, hist, st = S.solve(dev(b), s=s, tol=1e-8, maxit=5000)
    x = x.cpu().numpy()
    assert st == 0
    assert relres(A, b, x) <= 1e-8 * 1.01
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    # both relres <= 1e-8: ||x - x_ref|| / ||x_ref|| <= 2e-8 kappa
    assert np.linalg.norm(x - ref.x) <= 2e-8 * lam[-1] / lam[0] * np.linalg.norm(ref.x)
    S.close()


# ----------------------------------------------------------------------------------------
# Full-size Ani3D-like 128^3 (the benchmark's launch configuration), sampled checks
# ----------------------------------------------------------------------------------------

@pytest.mark.slow
def test_ani3d_full_size_sampled():
    """At n = 2,097,152 the oracle cannot finish a whole solve in test time: it runs the
    first 3 s-step iterations (rho_1..rho_3 compared to 1e-6) and the final GPU iterate is
    checked by a property that holds at any size, the true relative residual."""
    p = wl.ani3d(128, 32, seed=1)
    S = ekcg.Solver(p.A, 32, p.part, max_s=2)
    perm = S.perm()
    assert np.array_equal(perm, o.domain_perm(p.part))
    x, it, hist, st = S.solve(dev(p.b), s=2, tol=1e-8, maxit=5000)
    assert st == 0
    assert relres(p.A, p.b, x.cpu().numpy()) <= 1e-8 * 1.01
    ref = o.solve(p.A, p.b, p.part, 32, 2, tol=1e-8, maxit=3)
    np.testing.assert_allclose(hist[:4], ref.hist[:4], rtol=1e-6)
    # whole-solve oracle record (tests/golden/make_oracle_counts.py, oracle only)
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_counts.json")))
    g = gold["ani3d/t32/s2/sre/sstep/fp64"]
    assert abs(it - g["iters"]) <= 1
    np.testing.assert_allclose(hist[:21], g["hist"][:21], rtol=1e-6)
    S.close()


@pytest.mark.slow
@pytest.mark.parametrize("s", [1, 4, 8])
def test_ani3d_full_size_other_s_against_oracle_records(s):
    """Ani3D-like 128^3, t = 32, s = 1, 4, 8 (the configuration's other s values): the
    iteration count within one of the oracle's whole-solve record (tests/golden/
    oracle_counts.json, written by the oracle only), the first 21 residual norms to 1e-6
    and the true relative residual."""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_counts.json")))
    g = gold[f"ani3d/t32/s{s}/sre/sstep/fp64"]
    p = wl.ani3d(128, 32, seed=1)
    S = ekcg.Solver(p.A, 32, p.part, max_s=s)
    x, it, hist, st = S.solve(dev(p.b), s=s, tol=1e-8, maxit=5000)
    assert st == 0
    assert abs(it - g["iters"]) <= 1, (it, g["iters"])
    np.testing.assert_allclose(hist[:21], g["hist"][:21], rtol=1e-6)
    assert relres(p.A, p.b, x.cpu().numpy()) <= 1e-8 * 1.01
    S.close()


@pytest.mark.slow
def test_sky3d_full_size_against_oracle_record():
    """Sky3D-like 96^3 (coefficient 1 / 1e3 on 8^3 blocks), t = 16, s = 4, float64: the
    iteration count within one of the oracle's whole-solve record
    (tests/golden/oracle_counts.json, written by the oracle only), the first 21 residual
    norms to 1e-6 and the true relative residual."""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_counts.json")))
    key = "sky3d/t16/s4/sre/sstep/fp64"
    g = gold[key]
    p = wl.sky3d(96, 16, seed=2)
    S = ekcg.Solver(p.A, 16, p.part, max_s=4)
    x, it, hist, st = S.solve(dev(p.b), s=4, tol=1e-8, maxit=5000)
    assert st == 0
    assert abs(it - g["iters"]) <= 1, (it, g["iters"])
    np.testing.assert_allclose(hist[:21], g["hist"][:21], rtol=1e-6)
    assert relres(p.A, p.b, x.cpu().numpy()) <= 1e-8 * 1.01
    S.close()


@pytest.mark.slow
def test_sky3d_full_size_perturbed_counts_within_oracle_spread():
    """The Sky3D-like count is sensitive to rounding: with b multiplied entrywise by
    (1 + 1e-15 xi) the oracle itself takes 452 - 457 iterations (tests/golden/
    oracle_counts.json, "perturbed" records, written by the oracle only; the same range
    with A-CholQR applying its factor by the explicit inverse, "inverse" records).  With
    the same perturbations, the float64-FMA contraction's counts must lie within that
    spread widened by one.  (The default tensor-core contraction passes the unperturbed
    test above; its perturbed counts reach up to four above the oracle's range, an open
    finding reported with the measurements, not a bar this test sets.)"""
    import json
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "oracle_counts.json")))
    key = "sky3d/t16/s4/sre/sstep/fp64"
    seeds = sorted(int(k.rsplit("/", 1)[1]) for k in gold if k.startswith(key + "/perturbed/"))
    counts = [gold[key]["iters"]] + [gold[f"{key}/perturbed/{sd}"]["iters"] for sd in seeds]
    counts += [v["iters"] for k, v in gold.items() if k.startswith(key + "/inverse")]
    p = wl.sky3d(96, 16, seed=2)
    S = ekcg.Solver(p.A, 16, p.part, max_s=4, contraction="fp64")
    got = []
    for sd in seeds:
        b = p.b * (1.0 + 1e-15 * np.random.default_rng(sd).standard_normal(p.A.n))
        x, it, hist, st = S.solve(dev(b), s=4, tol=1e-8, maxit=5000)
        assert st == 0
        got.append(it)
    S.close()
    assert all(min(counts) - 1 <= it <= max(counts) + 1 for it in got), (got, counts)


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    """The bulk-copy stages wait on mbarriers with a cycle limit.  A stage that never
    completes (16 bytes expected, no copy issued) must end in EKCG_ETIMEOUT, not a hang, and
    a solve afterwards must still succeed."""
    assert ekcg.ekcg_wait_selftest(1 << 20) == ekcg.EKCG_ETIMEOUT
    assert ekcg.ekcg_wait_selftest(0) == ekcg.EKCG_EINVAL
    A, b, part = ragged_problem(4)
    S = ekcg.Solver(A, 4, part, max_s=2)
    x, it, hist, st = S.solve(dev(b), s=2, tol=1e-8, maxit=500)
    assert st == 0 and relres(A, b, x.cpu().numpy()) <= 1e-8 * 1.01
    S.close()


# ----------------------------------------------------------------------------------------
# Rank-revealing A-CholQR: deflation of dependent directions instead of breakdown
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["sre", "sre2", "msdo"])
@pytest.mark.parametrize("s", [1, 2])
def test_deflation_vanishing_domain_against_oracle(variant, s):
    """b vanishes on one of the t = 4 domains, so T(r_0) has a zero column: with
    deflate = True the GPU drops it as the oracle does and the solve converges (without
    deflation both stop with a breakdown, test_edge_cases)."""
    A, b, part = ragged_problem()
    b = b.copy()
    b[part == 2] = 0.0
    ref = o.solve(A, b, part, 4, s, tol=1e-8, maxit=2000, variant=variant, deflate=True)
    S = ekcg.Solver(A, 4, part, variant=variant, max_s=s, max_basis_bytes=8 << 30,
                    deflate=True)
    x, it, hist, st = S.solve(dev(b), s=s, tol=1e-8, maxit=2000)
    ndef = S.deflated_columns()
    S.close()
    assert st == ref.status == o.OK and ndef >= 1
    assert abs(it - ref.iters) <= 1, (it, ref.iters)
    m = min(21, len(hist), len(ref.hist))
    np.testing.assert_allclose(hist[:m], ref.hist[:m], rtol=1e-6)
    x = x.cpu().numpy()
    assert relres(A, b, x) <= 1e-8 * 1.01
    assert np.linalg.norm(x - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_deflation_needs_acholqr():
    A, b, part = ragged_problem()
    with pytest.raises(ekcg.EkcgError):
        ekcg.Solver(A, 4, part, orth="precholqr", deflate=True)


# ----------------------------------------------------------------------------------------
# Device-side convergence (the `while` line of Algorithms 3 / 4 tested on the device)
# ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("basis,s", [("sstep", 1), ("sstep", 2), ("sstep", 3),
                                     ("sstep", 4), ("restructured", 2)])
def test_device_loop_matches_host_loop_bitwise(basis, s):
    """The graph of conditional iterations launches the host loop's kernels in the host
    loop's order: x, the iteration count and every residual norm are bitwise the same;
    the iterations after the window fills ran on the device."""
    A, b, part = ragged_problem()
    S = ekcg.Solver(A, 4, part, basis=basis, max_s=s)
    S.set_device_loop(True)
    xd, itd, hd, std = S.solve(dev(b), s=s, tol=1e-8, maxit=2000)
    on_dev = S.device_loop_iters()
    S.set_device_loop(False)
    xh, ith, hh, sth = S.solve(dev(b), s=s, tol=1e-8, maxit=2000)
    assert S.device_loop_iters() == 0
    S.close()
    assert std == sth == 0 and itd == ith
    assert on_dev == itd - (2 if s == 1 else 1)
    assert np.array_equal(xd.cpu().numpy(), xh.cpu().numpy())
    assert np.array_equal(hd, hh)


@pytest.mark.parametrize("maxit", [2, 3, 9, 10, 11, 17])
def test_device_loop_stops_at_maxit(maxit):
    """maxit reached inside a batch of graph iterations: status EKCG_MAXIT, exactly maxit
    iterations, maxit + 1 residual norms, the iterate of the host loop."""
    A, b, part = ragged_problem()
    S = ekcg.Solver(A, 4, part, max_s=2)
    x, it, hist, st = S.solve(dev(b), s=2, tol=1e-8, maxit=maxit)
    S.set_device_loop(False)
    xh, ith, hh, sth = S.solve(dev(b), s=2, tol=1e-8, maxit=maxit)
    S.close()
    assert st == sth == ekcg.EKCG_MAXIT and it == ith == maxit and len(hist) == maxit + 1
    assert np.array_equal(x.cpu().numpy(), xh.cpu().numpy()) and np.array_equal(hist, hh)
